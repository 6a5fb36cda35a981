// Exact adjoint P^T of the Siddon projector: f_j = sum_i a_ij g_i with the same a_ij.
//
// The paper replaces the adjoint by the closed form of Eq. (3) because a ray-driven
// scatter would make threads collide on voxels (Section 2.2.2). Here the exact transpose
// is computed as a gather: each thread owns one (x, y) voxel column and a chunk of ZC
// consecutive z voxels and, for every view, visits exactly the rays that can cross it.
// The geometry separates: ray (u, v) meets column (ix, iy) over a tau interval [ta, tb]
// that depends on u only, and meets z slab k over an interval that depends on v only, so
//   a_ij = |D - S| * max(0, min(tb, tz1(v)) - max(ta, tz0(v))).
// Candidate imager columns u come from the shadow of the voxel column's corners. For one
// u, almost every row whose ray reaches slab k stays inside it across the whole column
// and so has weight (tb - ta): those rows form a contiguous range and are summed at once
// from per-column prefix sums over rows (k_row_prefix); only the rows whose ray crosses
// a z plane inside the column (about 0.1 per plane at the paper's sizes) are evaluated
// one by one. The factor |D - S| is folded into the table, which holds for every row m
// the pair (prefix of the rows below m, value of row m): one 8-byte load per plane gives
// both the window's prefix and its straddling row. Every crossing parameter
// uses the same helper expressions as the projector, so both operators use the same
// FP32 weights. No atomics: the result is independent of scheduling.
#include "cbct_internal.cuh"

#include <type_traits>

namespace cbct {

// Thread mapping: each warp takes an 8 x 4 patch of voxel columns, and a block of NT
// threads stacks them into a 16 x (NT / 8) tile. Lanes whose columns are close in both x
// and y read nearby table entries in every view (a voxel's imager column moves with x at
// some views and with y at others): an 8 x 4 patch touches 10 sectors per table request
// where a 32 x 1 row touched 16, and the warps of a block share their lines in L1. Larger
// blocks share more of each view's table lines and pay where the grid is large (16-voxel
// chunks on the paper's finest grid, kernel alone: 128 threads 1.80 ms, 256 1.72 ms, 512
// (16 x 32 columns) 1.70 ms, 1024 1.72 ms); on coarser grids they leave too few blocks,
// and 128 threads are kept.
constexpr int BP_THREADS = 128;                 // the block size of the coarser grids
constexpr int BP_BIG_THREADS = 512;             // with 16-voxel chunks
constexpr int BP_WX = 8, BP_WY = 4;             // warp patch
constexpr int BP_BX = 16;                       // block tile along x (two patches)
template <int NT> constexpr int bp_by() { return BP_WY * (NT / 64); } // block tile along y
constexpr int BP_BY = bp_by<BP_THREADS>();

// resident blocks per SM the register budget of the 16-voxel chunks is sized for (64
// registers, no spills)
#ifndef CBCT_BP_Z16_BLOCKS
#define CBCT_BP_Z16_BLOCKS 8
#endif

// z voxels per thread. 16 halves the per-visit setup and the plane shared by two chunks,
// but doubles a thread's work: it pays only where the grid still fills many waves of the
// resident slots (at least six of 8 blocks per SM); measured 2.35 -> 2.26 ms for the paper's
// 512x512x70 grid and 2.01 -> 1.87 ms for 512x512x128, while 256x256x64 (under two waves)
// and 256x256x35 (a ragged last chunk) lose 1-4%. Otherwise 8, halved while the grid has
// fewer than 4 blocks per SM.
static int bp_zchunk(const GeomDev &G)
{
    const long long tiles = (long long)((G.nx + BP_BX - 1) / BP_BX) * ((G.ny + BP_BY - 1) / BP_BY);
    const long long sms = device_sm_count();
    if (tiles * ((G.nz + 15) / 16) >= 6LL * CBCT_BP_Z16_BLOCKS * sms) return 16;
    const long long want = 4LL * sms;
    int zc = 8;
    while (zc > 1 && tiles * ((G.nz + zc - 1) / zc) < want) zc >>= 1;
    return zc;
}

int backproject_max_blocks(const GeomDev &G)
{
    return ((G.nx + BP_BX - 1) / BP_BX) * ((G.ny + BP_BY - 1) / BP_BY) * G.nz; // one z voxel per thread
}

// threads per block of a launch with z chunk zc
static int bp_threads(int zc) { return zc >= 16 ? BP_BIG_THREADS : BP_THREADS; }

int backproject_num_blocks(const GeomDev &G)
{
    const int zc = bp_zchunk(G);
    const int by = bp_threads(zc) == BP_BIG_THREADS ? bp_by<BP_BIG_THREADS>() : BP_BY;
    return ((G.nx + BP_BX - 1) / BP_BX) * ((G.ny + by - 1) / by) * ((G.nz + zc - 1) / zc);
}

// Rows whose ray, while inside the column (tau in [ta, tb], 1/(tc+ta) = A, 1/(tc+tb) = B),
// reaches the plane z = zp: v (tc + tau) = zp for some tau, i.e. v between zp*A and zp*B.
// Returned as a widened integer row range (may extend outside [0, nv-1]).
__device__ __forceinline__ void straddle_rows(const GeomDev &G, float zp, float A, float B, int &lo, int &hi)
{
    const float v0 = zp * A, v1 = zp * B;
    const float lim = (float)(G.nv + 1);
    const float flo = fminf(fmaxf(fmaf(fminf(v0, v1) - G.v_first, G.inv_dv, -1e-3f), -2.0f), lim);
    const float fhi = fminf(fmaxf(fmaf(fmaxf(v0, v1) - G.v_first, G.inv_dv, 1e-3f), -2.0f), lim);
    lo = (int)ceilf(flo);
    hi = (int)floorf(fhi);
}

// The straddling row of a plane window [a, b) (b <= a + 1; table entry T = (P[a], g[a]))
// split at the plane: its weighted value g (0 if the window is empty) times the part of
// [ta, tb] below and above the plane z = zp.
__device__ __forceinline__ void plane_split(const GeomDev &G, const float *s_invv, float2 T, int a, int b, float zp,
                                            float ta, float tb, float &g, float &below, float &above)
{
    g = b > a ? T.y : 0.0f;
    const float iw = s_invv[min(a, G.nv - 1)];
    const float scl = fminf(fmaxf(tau_zplane(zp, iw, G.tc), ta), tb);
    const float wlo = scl - ta, whi = tb - scl;
    const bool up = iw > 0.0f; // z grows along the ray (v >= 0)
    below = g * (up ? wlo : whi);
    above = g * (up ? whi : wlo);
}

// For a window on the imager (a <= nv - 1: the row exists; `in`: row a lies in the window,
// i.e. b > a): the weighted value of the straddling row times the part of [ta, tb] that
// lies below the plane z = zp (0 if the window is empty). UP = +1 / -1: the caller knows
// that a row in the window has v > 0 / v < 0 (its ray rises / falls), so the direction
// test is dropped; UP = 0 tests it.
template <int UP>
__device__ __forceinline__ float plane_below(const float *s_invv, float tc, float2 T, int a, bool in, float zp,
                                             float ta, float tb)
{
    const float g = in ? T.y : 0.0f;
    const float iw = s_invv[a];
    const float scl = fminf(fmaxf(tau_zplane(zp, iw, tc), ta), tb);
    const bool up = UP > 0 ? true : UP < 0 ? false : iw > 0.0f;
    return g * (up ? scl - ta : tb - scl);
}

// Rows reaching plane zp inside the column lie in the window [a, b) of imager rows (at
// most one row when the caller's `simple` test holds); a and b are clamped to [0, nv] so
// that the table entry col[a * nu] exists (the table is [view][row 0..nv][column]).
__device__ __forceinline__ void plane_window(const GeomDev &G, float zp, float A, float B, float c0, float c1,
                                             int &a, int &b)
{
    const float v0 = zp * A, v1 = zp * B;
    const float nvf = (float)G.nv;
    const float fa = fminf(fmaxf(fmaf(fminf(v0, v1), G.inv_dv, c0), 0.0f), nvf);
    const float fb = fminf(fmaxf(fmaf(fmaxf(v0, v1), G.inv_dv, c1), -1.0f), nvf - 1.0f);
    a = ceil_small(fa);
    b = floor_small(fb) + 1;
}

// Register budget of the 8-voxel chunks: 9 resident blocks of 128 threads (56 registers, no
// spills) instead of the 5 that 88 registers allowed; measured 2.96 -> 2.34 ms for one P^T
// of the paper grid through the public call, bit-identical results. Shorter chunks keep
// the compiler's choice (fewer registers there cost more than they gain).
#ifndef CBCT_BP_MIN_BLOCKS
#define CBCT_BP_MIN_BLOCKS 9
#endif
template <int ZC, bool FLAT, int NT>
__global__ void __launch_bounds__(NT, ZC >= 16 ? CBCT_BP_Z16_BLOCKS * 128 / NT : ZC >= 8 ? CBCT_BP_MIN_BLOCKS : 1)
k_backproject(GeomDev G, const float2 *__restrict__ ps, float *__restrict__ out, int sx, int sy, int sz,
              float *__restrict__ out2, double *__restrict__ partials)
{
    extern __shared__ float s_invv[]; // 1 / v per imager row
    __shared__ double s_warp[NT / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < G.nv; i += NT) {
        const float v = imager_v(G, i);
        s_invv[i] = v != 0.0f ? __frcp_rn(v) : 1e30f;
    }
    __syncthreads();

    const int ix = blockIdx.x * BP_BX + (warp & 1) * BP_WX + lane % BP_WX;
    const int iy = blockIdx.y * bp_by<NT>() + (warp >> 1) * BP_WY + lane / BP_WX;
    const int iz0 = blockIdx.z * ZC;
    const bool ok = ix < G.nx && iy < G.ny;
    float acc[ZC];
#pragma unroll
    for (int z = 0; z < ZC; ++z) acc[z] = 0.0f;

    if (ok) {
        const float xl = plane_at(ix, G.dx, G.x0), xh = plane_at(ix + 1, G.dx, G.x0);
        const float yl = plane_at(iy, G.dy, G.y0), yh = plane_at(iy + 1, G.dy, G.y0);
        float zp[ZC + 1], zs[ZC + 1];
#pragma unroll
        for (int z = 0; z <= ZC; ++z) {
            zp[z] = plane_at(iz0 + z, G.dz, G.z0);
            zs[z] = zp[z] * G.inv_dv;
        }
        const int nzc = min(ZC, G.nz - iz0); // valid voxels in this chunk
        const float ztop = plane_at(iz0 + nzc, G.dz, G.z0), zs_top = ztop * G.inv_dv; // the chunk's top plane
        const float zabs = fmaxf(fabsf(zp[0]), fabsf(ztop));
        const size_t view_stride = ((size_t)G.nv + 1) * G.nu;
        const float c0 = fmaf(-G.v_first, G.inv_dv, -1e-3f), c1 = fmaf(-G.v_first, G.inv_dv, 1e-3f);

        // imager columns in the shadow of the voxel column in view k (its corners' u)
        auto shadow = [&](int k, int &lo, int &hi) {
            const float2 cs = G.cs[k];
            float umin = 3.0e38f, umax = -3.0e38f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float px = (c & 1) ? xh : xl, py = (c & 2) ? yh : yl;
                const float a = fmaf(-px, cs.y, py * cs.x);
                const float w = G.sad - fmaf(px, cs.x, py * cs.y);
                const float u = G.sdd * __fdividef(a, w);
                umin = fminf(umin, u);
                umax = fmaxf(umax, u);
            }
            lo = max(0, (int)ceilf(fmaf(umin - G.u_first, G.inv_du, -1e-3f)));
            hi = min(G.nu - 1, (int)floorf(fmaf(umax - G.u_first, G.inv_du, 1e-3f)));
        };
        // all rows of imager column iu in view k that cross this voxel column
        auto visit = [&](int k, int iu) {
                const float4 r4 = __ldg(G.ray4 + k * G.nu + iu); // (dxr, dyr, qx, qy)
                const float2 r2 = __ldg(G.ray2 + k * G.nu + iu); // (1/dxr, 1/dyr)
                const float t0 = tau_plane(xl, r4.z, r2.x), t1 = tau_plane(xh, r4.z, r2.x);
                const float t2 = tau_plane(yl, r4.w, r2.y), t3 = tau_plane(yh, r4.w, r2.y);
                const float ta = fmaxf(fminf(t0, t1), fminf(t2, t3));
                const float tb = fminf(fmaxf(t0, t1), fmaxf(t2, t3));
                if (!(tb > ta)) return;
                const float A = __fdividef(1.0f, G.tc + ta), B = __fdividef(1.0f, G.tc + tb);
                const float wfull = tb - ta;
                const float2 *col = ps + (size_t)k * view_stride + iu; // prefix m at col[m * nu]
                // Plane z = zp is reached by the rows with v between zp*A and zp*B. While that
                // window is shorter than a row pitch and adjacent planes' windows are apart,
                // every row crosses at most one plane inside the column (the usual case).
                const float span = zabs * (A - B) * G.inv_dv;
                const bool simple = span + 3e-3f < 1.0f && fmaf(G.dz * B, G.inv_dv, -span) > 3e-3f;
                // row-window bounds at the lowest and highest plane of the chunk (monotone
                // in the plane height, so these bound every plane's window)
                const float fa_lo = fmaf(zs[0], zs[0] >= 0.0f ? B : A, c0);
                const float fb_hi = fmaf(zs_top, zs_top >= 0.0f ? A : B, c1);
                if (simple && fa_lo >= 0.0f && fb_hi <= (float)(G.nv - 1)) {
                    // every window lies on the imager: no clamping. Slab z receives the rows
                    // strictly between the windows of planes z and z + 1 at weight tb - ta,
                    // P[a_{z+1}] - P[a_z] - g_z, the part of plane z's straddling row above
                    // the plane, g_z (tb - ta) - below_z, and the part of plane z + 1's
                    // straddling row below it, below_{z+1}; together
                    //     (tb - ta) (P[a_{z+1}] - P[a_z]) + below_{z+1} - below_z.
                    // The window of plane zp spans rows v in [zp B, zp A] above z = 0 and
                    // [zp A, zp B] below; a chunk whose planes all lie on one side (all but
                    // one chunk of a column) fixes that choice for the whole visit. Its
                    // windows' rows then also share the sign of v (below: the test that
                    // picks the side keeps every window a thousandth of a row pitch or more
                    // away from v = 0), so the split needs no per-row direction test.
                    auto planes = [&](auto side) {
                        constexpr int S = decltype(side)::value; // +1 / -1: every plane at z > 0 / < 0
                        auto bounds = [&](float zsv, float &lo_f, float &hi_f) {
                            const bool pos = S > 0 || (S == 0 && zsv >= 0.0f);
                            lo_f = pos ? B : A;
                            hi_f = pos ? A : B;
                        };
                        // The window is [a, b) with a = ceil(xa), b = floor(xb) + 1; row a is in it
                        // iff floor(xb) >= a, i.e. xb >= a (a is an integer), so b is not formed.
                        float lo_f, hi_f;
                        bounds(zs[0], lo_f, hi_f);
                        int a = ceil_small(fmaf(zs[0], lo_f, c0));
                        bool in = fmaf(zs[0], hi_f, c1) >= (float)a;
                        float2 T = __ldg(col + a * G.nu); // (nv + 1) * nu < 2^31: 32-bit offsets
                        float Pprev = T.x, bprev = plane_below<S>(s_invv, G.tc, T, a, in, zp[0], ta, tb);
#pragma unroll
                        for (int z = 0; z < ZC; ++z) {
                            if (z >= nzc) break;
                            bounds(zs[z + 1], lo_f, hi_f);
                            a = ceil_small(fmaf(zs[z + 1], lo_f, c0));
                            in = fmaf(zs[z + 1], hi_f, c1) >= (float)a;
                            T = __ldg(col + a * G.nu);
                            const float below = plane_below<S>(s_invv, G.tc, T, a, in, zp[z + 1], ta, tb);
                            acc[z] += fmaf(wfull, T.x - Pprev, below - bprev);
                            Pprev = T.x;
                            bprev = below;
                        }
                    };
                    // Side +1: the window of the lowest plane, hence of every plane, starts
                    // at a row with v / dv >= zs[0] B - 1e-3 > 0; side -1: every window ends
                    // at a row with v / dv <= zs_top B + 1e-3 < 0. Otherwise (a chunk that
                    // meets or nearly meets z = 0) both the side and the direction are
                    // decided per plane, which gives the same bounds for the planes at z >= 0.
                    if (zs[0] * B > 2e-3f) planes(std::integral_constant<int, 1>());
                    else if (zs_top * B < -2e-3f) planes(std::integral_constant<int, -1>());
                    else planes(std::integral_constant<int, 0>());
                } else if (simple) {
                    // windows may leave the imager: clamped to [0, nv]
                    int a, b;
                    plane_window(G, zp[0], A, B, c0, c1, a, b);
                    float2 T = __ldg(col + a * G.nu);
                    float g, below, above;
                    plane_split(G, s_invv, T, a, b, zp[0], ta, tb, g, below, above);
                    acc[0] += above;
                    float Pprev = T.x, gprev = g;
#pragma unroll
                    for (int z = 0; z < ZC; ++z) {
                        if (z >= nzc) break;
                        plane_window(G, zp[z + 1], A, B, c0, c1, a, b);
                        T = __ldg(col + a * G.nu);
                        plane_split(G, s_invv, T, a, b, zp[z + 1], ta, tb, g, below, above);
                        acc[z] = fmaf(wfull, (T.x - Pprev) - gprev, acc[z]) + below;
                        if (z + 1 < ZC && z + 1 < nzc) acc[z + 1] += above;
                        Pprev = T.x;
                        gprev = g;
                    }
                } else {
                    int lo_p, hi_p;
                    straddle_rows(G, zp[0], A, B, lo_p, hi_p);
#pragma unroll
                    for (int z = 0; z < ZC; ++z) {
                        if (z >= nzc) break;
                        int lo_n, hi_n;
                        straddle_rows(G, zp[z + 1], A, B, lo_n, hi_n);
                        float a = acc[z];
                        const int f0 = max(hi_p + 1, 0), f1 = min(lo_n - 1, G.nv - 1);
                        if (f0 <= f1) {
                            const float P1 = __ldg(col + (f1 + 1) * G.nu).x, P0 = __ldg(col + f0 * G.nu).x;
                            a = fmaf(wfull, P1 - P0, a);
                        }
                        // rows that cross a z plane inside the column: exact overlap
                        const int r0 = max(lo_p, 0), r1 = min(hi_n, G.nv - 1);
                        for (int iv = r0; iv <= r1; ++iv) {
                            if (iv == f0 && f0 <= f1) { // already counted
                                iv = f1;
                                continue;
                            }
                            const float iw = s_invv[iv];
                            const float s0 = tau_zplane(zp[z], iw, G.tc), s1 = tau_zplane(zp[z + 1], iw, G.tc);
                            const float lo = fmaxf(ta, fminf(s0, s1)), hi = fminf(tb, fmaxf(s0, s1));
                            if (hi > lo) a = fmaf(__ldg(col + iv * G.nu).y, hi - lo, a);
                        }
                        acc[z] = a;
                        lo_p = lo_n;
                        hi_p = hi_n;
                    }
                }
        };
        if (FLAT) {
            // Each lane walks its own list of candidates (view, imager column) across all
            // views in one loop, so a warp runs for the longest per-lane total instead of the
            // widest shadow in every view: fewer idle lanes where shadows are ~1 column wide.
            int k = -1, iu = 0, iu_hi = -1;
            for (;;) {
                while (iu > iu_hi && k < G.nviews) // next view with a non-empty shadow
                    if (++k < G.nviews) shadow(k, iu, iu_hi);
                if (k >= G.nviews) break;
                visit(k, iu++);
            }
        } else {
            for (int k = 0; k < G.nviews; ++k) {
                int lo, hi;
                shadow(k, lo, hi);
                for (int iu = lo; iu <= hi; ++iu) visit(k, iu);
            }
        }
    }

    double red = 0.0;
    if (ok) {
        const long long base = (long long)ix * sx + (long long)iy * sy;
#pragma unroll
        for (int z = 0; z < ZC; ++z) {
            if (iz0 + z < G.nz) {
                const long long o = base + (long long)(iz0 + z) * sz;
                out[o] = acc[z];
                if (out2) out2[o] = acc[z];
                red += (double)acc[z] * (double)acc[z];
            }
        }
    }
    if (partials) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) red += __shfl_down_sync(0xffffffffu, red, o);
        if ((tid & 31) == 0) s_warp[tid >> 5] = red;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < NT / 32; ++w) t += s_warp[w];
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
}

cbct_status launch_backproject(const GeomDev &G, const float2 *ps, float *out, long long sx, long long sy,
                               long long sz, float *out2, double *partials, cudaStream_t st)
{
    const int zc = bp_zchunk(G);
    const int nt = bp_threads(zc);
    const int by = nt == BP_BIG_THREADS ? bp_by<BP_BIG_THREADS>() : BP_BY;
    dim3 block(nt);
    dim3 grid((G.nx + BP_BX - 1) / BP_BX, (G.ny + by - 1) / by, (G.nz + zc - 1) / zc);
    const size_t smem = sizeof(float) * G.nv;
    const int isx = (int)sx, isy = (int)sy, isz = (int)sz;
    ProfToken tok = prof_start(CBCT_KERNEL_BACKPROJECT, st);
    // flatten the candidate loop where a voxel column's shadow spans about one imager
    // column (its diagonal, magnified at the rotation axis, below 1.5 pixels)
    const bool flat = sqrtf(G.dx * G.dx + G.dy * G.dy) * (G.sdd / G.sad) < 1.5f * G.du;
#define CBCT_BP_LAUNCH(Z, NT)                                                                                    \
    if (flat) k_backproject<Z, true, NT><<<grid, block, smem, st>>>(G, ps, out, isx, isy, isz, out2, partials);    \
    else k_backproject<Z, false, NT><<<grid, block, smem, st>>>(G, ps, out, isx, isy, isz, out2, partials)
    switch (zc) {
    case 16: CBCT_BP_LAUNCH(16, BP_BIG_THREADS); break;
    case 8: CBCT_BP_LAUNCH(8, BP_THREADS); break;
    case 4: CBCT_BP_LAUNCH(4, BP_THREADS); break;
    case 2: CBCT_BP_LAUNCH(2, BP_THREADS); break;
    default: CBCT_BP_LAUNCH(1, BP_THREADS); break;
    }
#undef CBCT_BP_LAUNCH
    prof_stop(tok, st);
    note_launch();
    return check_cuda(cudaGetLastError(), "backproject launch");
}

// Prefix sums over imager rows of every (view k, imager column iu), stored row-major like
// the projections so that neighbouring lanes (columns) touch neighbouring addresses:
// ps[k][m][iu] = (P_m, w(m) g[k][m][iu]) for m = 0..nv, where P_m = sum_{iv < m} w(iv)
// g[k][iv][iu] and the second member is row m's own weighted value (0 at m = nv), with
// w = |D - S| if `prescale` (folds the ray length into the adjoint's input) and 1
// otherwise. The running sums are compensated (Neumaier) and rounded to FP32 once per
// entry, so a difference of two prefixes carries at most two roundings of the prefixes'
// magnitude. A block covers 32 columns (lanes, coalesced reads) of one view; its 16 warps
// take consecutive row chunks: pass 1 sums each chunk, the chunk offsets come from shared
// memory, pass 2 writes.
constexpr int PREFIX_WARPS = 16;

// Compensated FP32 summation (Neumaier): s + c carries the running sum to about twice
// FP32's precision. (FP64 arithmetic is much slower on this part.)
__device__ __forceinline__ void comp_add(float &s, float &c, float v)
{
    const float t = s + v;
    const bool s_big = fabsf(s) >= fabsf(v);
    c += ((s_big ? s : v) - t) + (s_big ? v : s);
    s = t;
}

template <typename T>
__global__ void __launch_bounds__(32 * PREFIX_WARPS)
k_row_prefix(GeomDev G, const T *__restrict__ g, float2 *__restrict__ ps, int prescale)
{
    __shared__ float2 s_tot[PREFIX_WARPS][32];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int k = blockIdx.y, iu = blockIdx.x * 32 + lane;
    const bool ok = iu < G.nu;
    const int chunk = (G.nv + PREFIX_WARPS - 1) / PREFIX_WARPS;
    const int r0 = min(G.nv, w * chunk), r1 = min(G.nv, r0 + chunk);
    float dxr = 0.f, dyr = 0.f;
    if (prescale && ok) {
        const float4 r4 = __ldg(G.ray4 + k * G.nu + iu);
        dxr = r4.x;
        dyr = r4.y;
    }
    const T *src = g + (size_t)k * G.nv * G.nu + iu;
    float ts = 0.0f, tc = 0.0f;
    if (ok)
        for (int iv = r0; iv < r1; ++iv) {
            float val = load_as_float(src + (size_t)iv * G.nu);
            if (prescale) val *= ray_length(dxr, dyr, imager_v(G, iv));
            comp_add(ts, tc, val);
        }
    s_tot[w][lane] = make_float2(ts, tc);
    __syncthreads();
    float rs = 0.0f, rc = 0.0f; // the chunks before this warp's
    for (int c = 0; c < w; ++c) {
        const float2 t = s_tot[c][lane];
        comp_add(rs, rc, t.x);
        rc += t.y;
    }
    if (!ok) return;
    float2 *dst = ps + (size_t)k * ((size_t)G.nv + 1) * G.nu + iu; // entry m at dst[m * nu]
    for (int iv = r0; iv < r1; ++iv) {
        float val = load_as_float(src + (size_t)iv * G.nu);
        if (prescale) val *= ray_length(dxr, dyr, imager_v(G, iv));
        dst[(size_t)iv * G.nu] = make_float2(rs + rc, val);
        comp_add(rs, rc, val);
    }
    if (w == PREFIX_WARPS - 1) dst[(size_t)G.nv * G.nu] = make_float2(rs + rc, 0.0f); // all rows
}

cbct_status launch_row_prefix(const GeomDev &G, const void *g, float2 *ps, int prescale, cudaStream_t st, int storage)
{
    dim3 grid((G.nu + 31) / 32, G.nviews), block(32, PREFIX_WARPS);
    if (storage == ST_BF16)
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_row_prefix<__nv_bfloat16><<<grid, block, 0, st>>>(G, static_cast<const __nv_bfloat16 *>(g), ps, prescale));
    else if (storage == ST_F16)
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_row_prefix<__half><<<grid, block, 0, st>>>(G, static_cast<const __half *>(g), ps, prescale));
    else
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_row_prefix<float><<<grid, block, 0, st>>>(G, static_cast<const float *>(g), ps, prescale));
    return check_cuda(cudaGetLastError(), "row prefix launch");
}

// The paper's own backprojector, Eq. (3): voxel-driven, for every view the imager value at
// the point u* where the ray through the voxel centre x meets the imager is taken by
// bilinear interpolation (zero outside the imager) and weighted by
// (dx dy dz / (du dv)) L^3(u*) / (L0 l^2(x)) with L0 = sdd, l = |x - S|, L = |u* - S|.
// With w the distance of x from the source along the central ray, L = l sdd / w, so the
// weight is (dx dy dz / (du dv)) l sdd^2 / w^3. It approximates the exact adjoint
// (Appendix 2). Thread per voxel, lanes along x (public x-fastest layout).
__global__ void __launch_bounds__(128)
k_backproject_eq3(GeomDev G, const float *__restrict__ g, float *__restrict__ f, float pref)
{
    const int ix = blockIdx.x * 32 + threadIdx.x, iy = blockIdx.y * 4 + threadIdx.y, iz = blockIdx.z;
    if (ix >= G.nx || iy >= G.ny) return;
    const float px = fmaf((float)ix + 0.5f, G.dx, G.x0);
    const float py = fmaf((float)iy + 0.5f, G.dy, G.y0);
    const float pz = fmaf((float)iz + 0.5f, G.dz, G.z0);
    const float sdd2 = G.sdd * G.sdd;
    float acc = 0.0f;
    for (int k = 0; k < G.nviews; ++k) {
        const float2 cs = G.cs[k];
        const float w = G.sad - fmaf(px, cs.x, py * cs.y);
        const float inv_w = 1.0f / w;
        const float u = G.sdd * fmaf(-px, cs.y, py * cs.x) * inv_w;
        const float v = G.sdd * pz * inv_w;
        const float fu = (u - G.u_first) * G.inv_du, fv = (v - G.v_first) * G.inv_dv;
        const float flu = floorf(fu), flv = floorf(fv);
        const int i0 = (int)flu, j0 = (int)flv;
        const float wu = fu - flu, wv = fv - flv;
        const float *gk = g + (size_t)k * G.nv * G.nu;
        float val = 0.0f;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const int iu = i0 + a, iv = j0 + b;
                if (iu >= 0 && iu < G.nu && iv >= 0 && iv < G.nv)
                    val = fmaf((a ? wu : 1.0f - wu) * (b ? wv : 1.0f - wv), __ldg(gk + (size_t)iv * G.nu + iu), val);
            }
        const float dxs = fmaf(-G.sad, cs.x, px), dys = fmaf(-G.sad, cs.y, py);
        const float l = sqrtf(fmaf(dxs, dxs, fmaf(dys, dys, pz * pz)));
        acc = fmaf(pref * l * sdd2 * inv_w * inv_w * inv_w, val, acc);
    }
    f[((size_t)iz * G.ny + iy) * G.nx + ix] = acc;
}

cbct_status launch_backproject_eq3(const GeomDev &G, const float *g, float *f, float pref, cudaStream_t st)
{
    dim3 grid((G.nx + 31) / 32, (G.ny + 3) / 4, G.nz), block(32, 4);
    CBCT_TIMED(CBCT_KERNEL_BACKPROJECT, st, k_backproject_eq3<<<grid, block, 0, st>>>(G, g, f, pref));
    return check_cuda(cudaGetLastError(), "backproject_eq3 launch");
}

} // namespace cbct
