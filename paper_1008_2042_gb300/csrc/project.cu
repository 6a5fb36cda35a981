// Forward projector P (Eq. (1), Section 2.2.1: one ray per imager pixel, Siddon's exact
// ray tracing, g_i = sum_j a_ij f_j with a_ij the length of ray i inside voxel j).
//
// GB300 mapping. All rays of one view that hit the same imager column u share their
// transverse path through the (x, y) voxel columns; the imager row v only tilts them in
// z. A block owns one (view, column) pair and its threads own the imager rows. The
// block first computes the shared transverse Siddon trace once, cooperatively, into
// shared memory (a parallel merge of the x-plane and y-plane crossing lists). Each lane
// then walks that list, reading the voxel of its own z slab in every column; with the
// iteration's z-fastest volume layout the 32 lanes of a warp read a few consecutive
// floats of one column, one or two 32-byte sectors per load. Columns are processed in
// unrolled groups whose loads are all in flight together; the rare columns in which a
// lane crosses a z plane are corrected afterwards. Accumulation is FP32; the epilogue can
// scale by |D - S|, form the CGLS residual and reduce squared norms in FP64 into one
// partial per block; the output is stored as FP32, BF16 or FP16.
#include <cfloat>

#include "cbct_internal.cuh"

namespace cbct {

constexpr int PROJ_THREADS = 192; // threads per block; each thread walks two imager rows
constexpr float P_INF = 3.0e38f;

// threads of a block (a multiple of 32, every lane present for warp votes) and the imager
// rows one block covers (two per thread)
static inline int proj_threads(const GeomDev &G)
{
    const int rows = G.nv < 2 * PROJ_THREADS ? G.nv : 2 * PROJ_THREADS;
    const int t = (((rows + 1) / 2 + 31) / 32) * 32;
    return t < PROJ_THREADS ? t : PROJ_THREADS;
}

int project_num_blocks(const GeomDev &G)
{
    const int rows = 2 * proj_threads(G);
    return G.nviews * G.nu * ((G.nv + rows - 1) / rows);
}

// Number of column segments a lane processes per unrolled group.
constexpr int SEG_GROUP = 16;

__device__ __forceinline__ int lower_count(const float *a, int n, float t) // # a[i] < t
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] < t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__device__ __forceinline__ int upper_count(const float *a, int n, float t) // # a[i] <= t
{
    int lo = 0, hi = n;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (a[mid] <= t) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

static inline int seg_capacity(const GeomDev &G)
{
    return ((G.nx + G.ny + 3 + SEG_GROUP - 1) / SEG_GROUP + 1) * SEG_GROUP;
}

// Shared memory of one block: the two crossing lists, then (16-byte aligned) per segment
// its end tau, its column offset and the packed record used by the walk.
static inline int seg_offset(const GeomDev &G) { return ((G.nx + G.ny + 2 + 3) / 4) * 4; }

// z-lines of one group of columns, staged in shared memory as adjacent-voxel pairs
// (f[k], f[k+1]) indexed [k][column in group], the column pitch odd to spread banks.
constexpr int LINE_PITCH = SEG_GROUP + 1;

static inline int line_pairs(const GeomDev &G) { return G.nz > 1 ? G.nz - 1 : 1; }

static inline size_t project_smem(const GeomDev &G)
{
    return sizeof(float) * (size_t)seg_offset(G) + (sizeof(float) + sizeof(int) + sizeof(float4)) * (size_t)seg_capacity(G) +
           sizeof(float2) * 2 * (size_t)line_pairs(G) * LINE_PITCH;
}

size_t project_smem_bytes(const GeomDev &G) { return project_smem(G); }

__device__ __forceinline__ void cp_async4(float *smem_dst, const float *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One block per (view, imager column, chunk of rows), volume z-contiguous (sz = 1).
// Phase 1 (whole block): the transverse Siddon trace of the column's rays — the
// crossings with the x planes and with the y planes are each increasing in tau, so every
// crossing's position in the merged order is its own index plus the number of crossings
// of the other family before it (binary search); this yields the list of (x, y) voxel
// columns the rays visit and the tau at which each is left. For every segment the block
// also stores its length, 1 / length and its start relative to its group.
// Phase 2 (one lane per imager row): walk the list in groups of SEG_GROUP columns. In a
// group a lane crosses at most one z plane (else an exact sequential walk is used): it
// reads the voxel pair (kb, kb + 1) around its current and next slab in every column and
// splits each column's length at its crossing with a saturated FMA. No branch and no
// integer or compare instruction is spent per column.
template <int MODE, typename TP>
__global__ void __launch_bounds__(PROJ_THREADS, 4)
k_project(GeomDev G, const float *__restrict__ f, int sx, int sy, const float *__restrict__ y,
          TP *__restrict__ out, double *__restrict__ partials, float count_thr, const Scalars *__restrict__ sc)
{
    extern __shared__ float smem[];
    __shared__ double s_warp[PROJ_THREADS / 32];
    float *sA = smem;                      // x-plane crossings, in ray order
    float *sB = sA + (G.nx + 1);           // y-plane crossings
    const int cap = ((G.nx + G.ny + 3 + SEG_GROUP - 1) / SEG_GROUP + 1) * SEG_GROUP;
    float *sEnd = smem + ((G.nx + G.ny + 2 + 3) / 4) * 4; // tau at which segment j ends
    int *sCol = reinterpret_cast<int *>(sEnd + cap);      // voxel-column offset of segment j
    float4 *sSeg = reinterpret_cast<float4 *>(sCol + cap); // (column bits, length, 1/length, start term)
    float2 *sPair = reinterpret_cast<float2 *>(sSeg + cap); // two staged groups of z-line pairs
    const int npair = G.nz > 1 ? G.nz - 1 : 1;

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int view = blockIdx.x / G.nu;
    const int iu = blockIdx.x - view * G.nu;

    // ---- transverse ray, shared by every row ----
    const float2 cs = G.cs[view];
    float dxr, dyr, qx, qy;
    ray_xy(G, cs.x, cs.y, imager_u(G, iu), dxr, dyr, qx, qy);
    const float inv_x = safe_rcp(dxr), inv_y = safe_rcp(dyr);
    const float xa = tau_plane(G.x0, qx, inv_x), xb = tau_plane(plane_at(G.nx, G.dx, G.x0), qx, inv_x);
    const float ya = tau_plane(G.y0, qy, inv_y), yb = tau_plane(plane_at(G.ny, G.dy, G.y0), qy, inv_y);
    const float tau_in = fmaxf(fmaxf(fminf(xa, xb), fminf(ya, yb)), -G.tc);
    const float tau_out = fminf(fminf(fmaxf(xa, xb), fmaxf(ya, yb)), 1.0f - G.tc);
    const bool hit = tau_in < tau_out;
    const int sxs = dxr > 0.0f ? 1 : -1, sys = dyr > 0.0f ? 1 : -1;

    // ---- phase 1: crossings of each plane family, then their merged order ----
    int a_le = 0, a_in = 0, b_le = 0, b_in = 0;
    for (int a0 = 0; a0 <= G.nx; a0 += nthr) {
        const int a = a0 + tid;
        bool le = false, in = false;
        if (a <= G.nx && hit && dxr != 0.0f) {
            const float t = tau_plane(plane_at(dxr > 0.0f ? a : G.nx - a, G.dx, G.x0), qx, inv_x);
            sA[a] = t;
            le = t <= tau_in;
            in = t > tau_in && t < tau_out;
        }
        a_le += __syncthreads_count(le);
        a_in += __syncthreads_count(in);
    }
    for (int b0 = 0; b0 <= G.ny; b0 += nthr) {
        const int b = b0 + tid;
        bool le = false, in = false;
        if (b <= G.ny && hit && dyr != 0.0f) {
            const float t = tau_plane(plane_at(dyr > 0.0f ? b : G.ny - b, G.dy, G.y0), qy, inv_y);
            sB[b] = t;
            le = t <= tau_in;
            in = t > tau_in && t < tau_out;
        }
        b_le += __syncthreads_count(le);
        b_in += __syncthreads_count(in);
    }
    const float *LA = sA + a_le, *LB = sB + b_le;
    const int nA = a_in, nB = b_in, nseg = nA + nB + 1;
    // the column entered first contains the midpoint of the first segment
    float e0 = tau_out;
    if (nA) e0 = fminf(e0, LA[0]);
    if (nB) e0 = fminf(e0, LB[0]);
    const float tm = 0.5f * (tau_in + e0);
    const int ix_e = min(max((int)floorf((fmaf(tm, dxr, qx) - G.x0) / G.dx), 0), G.nx - 1);
    const int iy_e = min(max((int)floorf((fmaf(tm, dyr, qy) - G.y0) / G.dy), 0), G.ny - 1);
    for (int i = tid; i < nA; i += nthr) {
        const float t = LA[i];
        const int nb = lower_count(LB, nB, t), r = i + nb;
        const int cx = min(max(ix_e + sxs * (i + 1), 0), G.nx - 1), cy = min(max(iy_e + sys * nb, 0), G.ny - 1);
        sEnd[r] = t;
        sCol[r + 1] = cx * sx + cy * sy;
    }
    for (int j = tid; j < nB; j += nthr) {
        const float t = LB[j];
        const int na = upper_count(LA, nA, t), r = j + na;
        const int cx = min(max(ix_e + sxs * na, 0), G.nx - 1), cy = min(max(iy_e + sys * (j + 1), 0), G.ny - 1);
        sEnd[r] = t;
        sCol[r + 1] = cx * sx + cy * sy;
    }
    const int col0 = ix_e * sx + iy_e * sy;
    if (tid == 0) {
        sCol[0] = col0;
        sEnd[nseg - 1] = tau_out;
    }
    for (int q = nseg + tid; q < cap; q += nthr) { // zero-length padding up to whole groups
        sEnd[q] = tau_out;
        sCol[q] = col0;
    }
    __syncthreads();
    for (int q = tid; q < cap; q += nthr) {
        const float e = sEnd[q];
        const float st = q ? sEnd[q - 1] : tau_in;
        const int qg = q - q % SEG_GROUP;
        const float g0 = qg ? sEnd[qg - 1] : tau_in; // start of q's group
        const float len = e - st;
        const float ia = len > 0.0f ? __frcp_rn(len) : 0.0f;
        sSeg[q] = make_float4(__int_as_float(sCol[q]), len, ia, -(st - g0) * ia);
    }
    __syncthreads();

    // ---- phase 2: per-row z state (two rows per thread: iv[0] and iv[1] = iv[0] + nthr) ----
    constexpr int R = 2;
    int iv[R], skz[R], kz[R];
    float inv_v[R], tzn[R], L[R], acc[R];
    bool ok[R], active[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        iv[r] = blockIdx.y * (R * nthr) + r * nthr + tid;
        ok[r] = iv[r] < G.nv;
        const float v = imager_v(G, iv[r]);
        inv_v[r] = v != 0.0f ? __frcp_rn(v) : 1e30f;
        skz[r] = v >= 0.0f ? 1 : -1;
        kz[r] = (int)floorf((v * (G.tc + tau_in) - G.z0) / G.dz);
        active[r] = hit && ok[r] && kz[r] >= 0 && kz[r] < G.nz;
        tzn[r] = active[r] ? tau_zplane(plane_at(kz[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc) : P_INF;
        if (active[r] && tzn[r] <= tau_in) { // the entry point already lies past that plane
            kz[r] += skz[r];
            active[r] = (unsigned)kz[r] < (unsigned)G.nz;
            tzn[r] = active[r] ? tau_zplane(plane_at(kz[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc) : P_INF;
        }
        L[r] = ray_length(dxr, dyr, v);
        acc[r] = 0.0f;
    }

    int cnt = 0;
    if (hit && MODE == PM_COUNT) {
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float thr_tau = count_thr / L[r];
            float s0 = tau_in;
            for (int j = 0; j < nseg; ++j) {
                const float e = sEnd[j];
                float sl = s0;
                while (tzn[r] < e) {
                    cnt += (tzn[r] - sl) > thr_tau;
                    sl = tzn[r];
                    kz[r] += skz[r];
                    active[r] = (unsigned)kz[r] < (unsigned)G.nz;
                    tzn[r] = active[r] ? tau_zplane(plane_at(kz[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc) : P_INF;
                }
                if (active[r]) cnt += (e - sl) > thr_tau;
                s0 = e;
            }
        }
    } else if (hit) {
        // Stage the z-lines of each group of columns into shared memory one group ahead
        // (cp.async), then let every row read its voxel pair there.
        const int nchunk = (nseg + SEG_GROUP - 1) / SEG_GROUP;
        const int line_elems = SEG_GROUP * G.nz;
        const int u0 = tid / G.nz, k0 = tid - u0 * G.nz;
        const int du = nthr / G.nz, dk = nthr - du * G.nz;
        auto fill = [&](int chunk, int buf) {
            float2 *dst = sPair + buf * npair * LINE_PITCH;
            const float4 *seg = sSeg + chunk * SEG_GROUP;
            int u = u0, k = k0;
            for (int idx = tid; idx < line_elems; idx += nthr) {
                const float *src = f + __float_as_int(seg[u].x) + k;
                if (k < npair) cp_async4(&dst[k * LINE_PITCH + u].x, src);   // first of pair k
                if (k >= 1) cp_async4(&dst[(k - 1) * LINE_PITCH + u].y, src); // second of pair k - 1
                k += dk;
                u += du;
                if (k >= G.nz) {
                    k -= G.nz;
                    ++u;
                }
            }
            cp_async_commit();
        };
        fill(0, 0);
        float g0 = tau_in;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int j = ch * SEG_GROUP;
            if (ch + 1 < nchunk) {
                fill(ch + 1, (ch + 1) & 1);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const float2 *pairs = sPair + (ch & 1) * npair * LINE_PITCH;
            const float gend = sEnd[j + SEG_GROUP - 1];
            int knew[R];
            bool anew[R];
            float tz2[R];
            bool dense = false;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                knew[r] = kz[r] + skz[r];
                anew[r] = active[r] && (unsigned)knew[r] < (unsigned)G.nz;
                // the crossing after tzn, to detect two crossings inside one group
                tz2[r] = (tzn[r] < gend && anew[r])
                             ? tau_zplane(plane_at(knew[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc) : P_INF;
                dense = dense || tz2[r] < gend;
            }
            if (G.nz >= 2 && !__any_sync(0xffffffffu, dense)) {
                // voxel pair (kb, kb + 1) holding a row's current slab kz and next slab knew
                const float2 *base[R];
                float m_lo[R], m_hi[R], sg[R], hg[R], dt[R], acc_lo[R], acc_hi[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    int kb = anew[r] ? min(kz[r], knew[r]) : (active[r] ? (skz[r] > 0 ? kz[r] - 1 : kz[r]) : 0);
                    kb = min(max(kb, 0), G.nz - 2);
                    const bool lo_old = kb == kz[r];
                    m_lo[r] = ((lo_old && active[r]) || (kb == knew[r] && anew[r])) ? 1.0f : 0.0f;
                    m_hi[r] = ((kb + 1 == kz[r] && active[r]) || (kb + 1 == knew[r] && anew[r])) ? 1.0f : 0.0f;
                    // the lower voxel takes the part before the crossing if it is the current slab
                    sg[r] = lo_old ? 1.0f : -1.0f;
                    hg[r] = lo_old ? 0.0f : 1.0f;
                    dt[r] = fminf(tzn[r], 1e30f) - g0;
                    base[r] = pairs + kb * LINE_PITCH;
                    acc_lo[r] = 0.0f;
                    acc_hi[r] = 0.0f;
                }
#pragma unroll
                for (int u = 0; u < SEG_GROUP; ++u) {
                    const float4 sg4 = sSeg[j + u]; // (column, length, 1/length, start term)
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float flo = __saturatef(fmaf(sg[r], fmaf(dt[r], sg4.z, sg4.w), hg[r]));
                        const float wlo = sg4.y * flo, whi = sg4.y - wlo;
                        const float2 v = base[r][u];
                        acc_lo[r] = fmaf(v.x, wlo, acc_lo[r]);
                        acc_hi[r] = fmaf(v.y, whi, acc_hi[r]);
                    }
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    acc[r] = fmaf(m_lo[r], acc_lo[r], fmaf(m_hi[r], acc_hi[r], acc[r]));
                    if (tzn[r] < gend) {
                        kz[r] = knew[r];
                        active[r] = anew[r];
                        tzn[r] = tz2[r];
                    }
                }
            } else {
                // a row crosses several z planes in this group (or nz = 1): walk it exactly
#pragma unroll
                for (int r = 0; r < R; ++r) {
#pragma unroll 1
                    for (int u = 0; u < SEG_GROUP; ++u) {
                        const float e = sEnd[j + u];
                        float sl = u ? sEnd[j + u - 1] : g0;
                        while (tzn[r] < e) {
                            if (active[r])
                                acc[r] = fmaf(kz[r] < npair ? pairs[kz[r] * LINE_PITCH + u].x
                                                            : pairs[(kz[r] - 1) * LINE_PITCH + u].y,
                                              tzn[r] - sl, acc[r]);
                            sl = tzn[r];
                            kz[r] += skz[r];
                            active[r] = (unsigned)kz[r] < (unsigned)G.nz;
                            tzn[r] = active[r] ? tau_zplane(plane_at(kz[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc)
                                               : P_INF;
                        }
                        if (active[r])
                            acc[r] = fmaf(kz[r] < npair ? pairs[kz[r] * LINE_PITCH + u].x
                                                        : pairs[(kz[r] - 1) * LINE_PITCH + u].y,
                                          e - sl, acc[r]);
                    }
                }
            }
            g0 = gend;
            __syncthreads();
        }
    }

    // ---- epilogue ----
    double red = 0.0;
    const float kappa = (MODE == PM_Q_SCALED) ? (float)sc->kappa : 1.0f;
    constexpr bool PRESCALE = sizeof(TP) == 4;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        if (!ok[r]) continue;
        const size_t idx = ((size_t)view * G.nv + iv[r]) * G.nu + iu;
        const float q = acc[r] * L[r];
        // FP32 storage keeps |D - S| folded into r and q (the adjoint then needs no
        // per-sample rescale); 16-bit storage keeps the bare values
        const float s = PRESCALE ? L[r] : 1.0f;
        if (MODE == PM_PLAIN) {
            store_from_float(out + idx, q);
        } else if (MODE == PM_Q_SCALED) {
            store_from_float(out + idx, q * s * kappa);
            red += (double)q * (double)q;
        } else if (MODE == PM_RESID) {
            const float rr = __ldg(y + idx) - q;
            store_from_float(out + idx, rr * s);
            red += (double)rr * (double)rr;
        }
    }
    if (MODE == PM_COUNT) red = (double)cnt;
    if (MODE != PM_PLAIN) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) red += __shfl_down_sync(0xffffffffu, red, o);
        if ((tid & 31) == 0) s_warp[tid >> 5] = red;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < (nthr + 31) / 32; ++w) t += s_warp[w];
            partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
}

// per-device record of the shared-memory opt-in, one per kernel instantiation
template <int MODE, typename TP> static std::atomic<unsigned long long> g_project_optin{0};

template <int MODE, typename TP> static cbct_status project_optin()
{
    cudaError_t e = smem_optin_once(k_project<MODE, TP>, 200 * 1024, g_project_optin<MODE, TP>);
    return e == cudaSuccess ? CBCT_OK : check_cuda(e, "project attribute");
}

template <int MODE, typename TP>
static cbct_status launch_project_t(const GeomDev &G, const float *f, int isx, int isy, const float *y, void *out,
                                   double *partials, float count_thr, const Scalars *sc, dim3 grid, int threads,
                                   size_t smem, cudaStream_t st)
{
    {
        cbct_status a = project_optin<MODE, TP>();
        if (a != CBCT_OK) return a;
    }
    k_project<MODE, TP><<<grid, threads, smem, st>>>(G, f, isx, isy, y, static_cast<TP *>(out),
                                                    partials, count_thr, sc);
    return CBCT_OK;
}

cbct_status project_prepare()
{
    cbct_status r = CBCT_OK;
    if (r == CBCT_OK) r = project_optin<PM_PLAIN, float>();
    if (r == CBCT_OK) r = project_optin<PM_PLAIN, __nv_bfloat16>();
    if (r == CBCT_OK) r = project_optin<PM_PLAIN, __half>();
    if (r == CBCT_OK) r = project_optin<PM_COUNT, float>();
    if (r == CBCT_OK) r = project_optin<PM_Q_SCALED, float>();
    if (r == CBCT_OK) r = project_optin<PM_Q_SCALED, __nv_bfloat16>();
    if (r == CBCT_OK) r = project_optin<PM_Q_SCALED, __half>();
    if (r == CBCT_OK) r = project_optin<PM_RESID, float>();
    if (r == CBCT_OK) r = project_optin<PM_RESID, __nv_bfloat16>();
    if (r == CBCT_OK) r = project_optin<PM_RESID, __half>();
    return r;
}

cbct_status launch_project(const GeomDev &G, const float *f, long long sx, long long sy,
                           long long sz, const float *y, void *out, int mode,
                           double *partials, float count_thr, cudaStream_t st, int storage, const Scalars *sc)
{
    const int threads = proj_threads(G); // 2 rows each
    dim3 grid((unsigned)(G.nviews * G.nu), (unsigned)((G.nv + 2 * threads - 1) / (2 * threads)));
    const size_t smem = project_smem(G);
    if (smem > 200 * 1024)
        return set_error(CBCT_ERR_UNSUPPORTED, "project: grid too large for the projector's shared memory (nx + ny and nz)");
    if (sz != 1) return set_error(CBCT_ERR_INVALID_ARG, "project: the volume must be z-contiguous");
    const int isx = (int)sx, isy = (int)sy;
    cbct_status r = CBCT_OK;
    ProfToken tok = prof_start(CBCT_KERNEL_PROJECT, st);
    if (mode == PM_PLAIN) {
        if (storage == ST_BF16)
            r = launch_project_t<PM_PLAIN, __nv_bfloat16>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else if (storage == ST_F16)
            r = launch_project_t<PM_PLAIN, __half>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else
            r = launch_project_t<PM_PLAIN, float>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
    } else if (mode == PM_COUNT) {
        r = launch_project_t<PM_COUNT, float>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
    } else if (mode == PM_Q_SCALED) {
        if (storage == ST_BF16)
            r = launch_project_t<PM_Q_SCALED, __nv_bfloat16>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else if (storage == ST_F16)
            r = launch_project_t<PM_Q_SCALED, __half>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else
            r = launch_project_t<PM_Q_SCALED, float>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
    } else {
        if (storage == ST_BF16)
            r = launch_project_t<PM_RESID, __nv_bfloat16>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else if (storage == ST_F16)
            r = launch_project_t<PM_RESID, __half>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
        else
            r = launch_project_t<PM_RESID, float>(G, f, isx, isy, y, out, partials, count_thr, sc, grid, threads, smem, st);
    }
    prof_stop(tok, st);
    note_launch();
    if (r != CBCT_OK) return r;
    return check_cuda(cudaGetLastError(), "project launch");
}

} // namespace cbct
