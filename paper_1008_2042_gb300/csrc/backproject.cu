// Exact adjoint P^T of the Siddon projector: f_j = sum_i a_ij g_i with the same a_ij.
//
// The paper replaces the adjoint by the closed form of Eq. (3) because a ray-driven
// scatter would make threads collide on voxels (Section 2.2.2). Here the exact transpose
// is computed as a gather instead: each thread owns one (x, y) voxel column and a chunk
// of ZC consecutive z voxels, and for every view enumerates exactly the rays that can
// cross it. The geometry separates: ray (u, v) meets column (ix, iy) over a tau interval
// [ta, tb] that depends on u only, and meets z slab k over an interval that depends on v
// only, so
//   a_ij = |D - S| * max(0, min(tb, tz1(v)) - max(ta, tz0(v))).
// The candidate columns u come from the shadow of the column's four corners, the
// candidate rows of each (u, slab) pair from the slab's z range seen over [ta, tb]. The
// factor |D - S| is folded into the input beforehand (k_prescale, or the projector's
// prescaled epilogue inside CGLS). Every crossing parameter is computed with the same
// helper expressions as the projector, so both operators use the same FP32 weights.
// No atomics: the result is independent of scheduling. Lanes of a warp are adjacent x
// voxels, which see adjacent imager columns of the same rows: loads coalesce.
#include "cbct_internal.cuh"

namespace cbct {

constexpr int BP_TX = 32, BP_TY = 4;

static int bp_zchunk(const GeomDev &G)
{
    const long long tiles = (long long)((G.nx + BP_TX - 1) / BP_TX) * ((G.ny + BP_TY - 1) / BP_TY);
    const long long want = 4LL * device_sm_count();
    int zc = 8;
    while (zc > 1 && tiles * ((G.nz + zc - 1) / zc) < want) zc >>= 1;
    return zc;
}

int backproject_num_blocks(const GeomDev &G)
{
    const int zc = bp_zchunk(G);
    return ((G.nx + BP_TX - 1) / BP_TX) * ((G.ny + BP_TY - 1) / BP_TY) * ((G.nz + zc - 1) / zc);
}

template <int ZC>
__global__ void __launch_bounds__(BP_TX *BP_TY)
k_backproject(GeomDev G, const float *__restrict__ gt, float *__restrict__ out, long long sx,
              long long sy, long long sz, float *__restrict__ out2, double *__restrict__ partials)
{
    extern __shared__ float s_invv[]; // 1 / v per imager row
    __shared__ double s_warp[BP_TX * BP_TY / 32];
    const int tid = threadIdx.y * BP_TX + threadIdx.x;
    for (int i = tid; i < G.nv; i += BP_TX * BP_TY) {
        const float v = imager_v(G, i);
        s_invv[i] = v != 0.0f ? __frcp_rn(v) : 1e30f;
    }
    __syncthreads();

    const int ix = blockIdx.x * BP_TX + threadIdx.x;
    const int iy = blockIdx.y * BP_TY + threadIdx.y;
    const int iz0 = blockIdx.z * ZC;
    const bool ok = ix < G.nx && iy < G.ny;
    float acc[ZC];
#pragma unroll
    for (int z = 0; z < ZC; ++z) acc[z] = 0.0f;

    if (ok) {
        const float xl = plane_at(ix, G.dx, G.x0), xh = plane_at(ix + 1, G.dx, G.x0);
        const float yl = plane_at(iy, G.dy, G.y0), yh = plane_at(iy + 1, G.dy, G.y0);
        float zp[ZC + 1];
#pragma unroll
        for (int z = 0; z <= ZC; ++z) zp[z] = plane_at(iz0 + z, G.dz, G.z0);
        const int nzc = min(ZC, G.nz - iz0); // valid voxels in this chunk

        for (int k = 0; k < G.nviews; ++k) {
            const float2 cs = G.cs[k];
            // shadow of the column on the imager: u of its four corners
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
            const int iu_lo = max(0, (int)ceilf(fmaf(umin - G.u_first, G.inv_du, -1e-3f)));
            const int iu_hi = min(G.nu - 1, (int)floorf(fmaf(umax - G.u_first, G.inv_du, 1e-3f)));
            const float *gk = gt + (size_t)k * G.nv * G.nu;

            for (int iu = iu_lo; iu <= iu_hi; ++iu) {
                float dxr, dyr, qx, qy;
                ray_xy(G, cs.x, cs.y, imager_u(G, iu), dxr, dyr, qx, qy);
                const float inv_x = safe_rcp(dxr), inv_y = safe_rcp(dyr);
                const float t0 = tau_plane(xl, qx, inv_x), t1 = tau_plane(xh, qx, inv_x);
                const float t2 = tau_plane(yl, qy, inv_y), t3 = tau_plane(yh, qy, inv_y);
                const float ta = fmaxf(fminf(t0, t1), fminf(t2, t3));
                const float tb = fminf(fmaxf(t0, t1), fmaxf(t2, t3));
                if (!(tb > ta)) continue;
                // rows whose ray reaches slab [zl, zh] while inside the column:
                // v (tc + tau) in [zl, zh] for some tau in [ta, tb]
                const float A = __frcp_rn(G.tc + ta), B = __frcp_rn(G.tc + tb);
                const float *gcol = gk + iu;
#pragma unroll
                for (int z = 0; z < ZC; ++z) {
                    if (z >= nzc) break;
                    const float zl = zp[z], zh = zp[z + 1];
                    const float vlo = fminf(zl * A, zl * B), vhi = fmaxf(zh * A, zh * B);
                    const int iv_lo = max(0, (int)ceilf(fmaf(vlo - G.v_first, G.inv_dv, -1e-3f)));
                    const int iv_hi = min(G.nv - 1, (int)floorf(fmaf(vhi - G.v_first, G.inv_dv, 1e-3f)));
                    float a = acc[z];
                    for (int iv = iv_lo; iv <= iv_hi; ++iv) {
                        const float iw = s_invv[iv];
                        const float s0 = tau_zplane(zl, iw, G.tc), s1 = tau_zplane(zh, iw, G.tc);
                        const float lo = fmaxf(ta, fminf(s0, s1)), hi = fminf(tb, fmaxf(s0, s1));
                        if (hi > lo) a = fmaf(__ldg(gcol + (size_t)iv * G.nu), hi - lo, a);
                    }
                    acc[z] = a;
                }
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
            for (int w = 0; w < BP_TX * BP_TY / 32; ++w) t += s_warp[w];
            partials[((size_t)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x] = t;
        }
    }
}

cbct_status launch_backproject(const GeomDev &G, const float *gt, float *out, long long sx,
                               long long sy, long long sz, float *out2, double *partials,
                               cudaStream_t st)
{
    const int zc = bp_zchunk(G);
    dim3 block(BP_TX, BP_TY);
    dim3 grid((G.nx + BP_TX - 1) / BP_TX, (G.ny + BP_TY - 1) / BP_TY, (G.nz + zc - 1) / zc);
    const size_t smem = sizeof(float) * G.nv;
    ProfToken tok = prof_start(CBCT_KERNEL_BACKPROJECT, st);
    switch (zc) {
    case 8: k_backproject<8><<<grid, block, smem, st>>>(G, gt, out, sx, sy, sz, out2, partials); break;
    case 4: k_backproject<4><<<grid, block, smem, st>>>(G, gt, out, sx, sy, sz, out2, partials); break;
    case 2: k_backproject<2><<<grid, block, smem, st>>>(G, gt, out, sx, sy, sz, out2, partials); break;
    default: k_backproject<1><<<grid, block, smem, st>>>(G, gt, out, sx, sy, sz, out2, partials); break;
    }
    prof_stop(tok, st);
    note_launch();
    return check_cuda(cudaGetLastError(), "backproject launch");
}

// gt = g * |D - S| per pixel: folds the ray length into the adjoint's input.
__global__ void k_prescale(GeomDev G, const float *__restrict__ g, float *__restrict__ gt)
{
    const size_t n = (size_t)G.nviews * G.nv * G.nu;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const int iu = (int)(i % G.nu);
        const int iv = (int)((i / G.nu) % G.nv);
        const int k = (int)(i / ((size_t)G.nu * G.nv));
        const float2 cs = G.cs[k];
        float dxr, dyr, qx, qy;
        ray_xy(G, cs.x, cs.y, imager_u(G, iu), dxr, dyr, qx, qy);
        gt[i] = g[i] * ray_length(dxr, dyr, imager_v(G, iv));
    }
}

cbct_status launch_prescale(const GeomDev &G, const float *g, float *gt, cudaStream_t st)
{
    const size_t n = (size_t)G.nviews * G.nv * G.nu;
    const int threads = 256;
    const long long want = (long long)((n + threads - 1) / threads);
    const int blocks = (int)(want < 8LL * device_sm_count() * 8 ? want : 8LL * device_sm_count() * 8);
    CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_prescale<<<blocks > 0 ? blocks : 1, threads, 0, st>>>(G, g, gt));
    return check_cuda(cudaGetLastError(), "prescale launch");
}

} // namespace cbct
