// CGLS (Appendix 1), Algorithm A2 (Section 2.1) and the coarse-to-fine multigrid
// (Section 2.2.3), plus the public entry points that wrap the operators.
//
// The whole iteration stays on the device: CGLS inner products are reduced in FP64 into
// device-resident scalars (one partial per producer block, then one finalising block
// in a fixed order, so results are deterministic), and the vector updates read their
// step sizes from there. The host only enqueues kernels; it reads one status word at
// the end. The A2 momentum coefficients do not depend on the data and are computed on
// the host.
#include <cmath>
#include <cstring>
#include <memory>
#include <utility>
#include <vector>

#include "cbct_internal.cuh"

namespace cbct {

// ------------------------------------------------------------------------------------
// Reductions and vector updates
// ------------------------------------------------------------------------------------

// scale_q: q is about to be stored in FP16, so keep kappa = 1 / sqrt(gamma) (||kappa p|| >= 1
// and kappa q stays O(1)); otherwise kappa = 1.
__global__ void __launch_bounds__(1024) k_finalize(const double *__restrict__ partials, int n,
                                                   Scalars *sc, int op, int scale_q)
{
    __shared__ double s[32];
    double t = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) t += partials[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += s[w];
        if (!isfinite(sum)) sc->flags |= 1u;
        if (op == FIN_GAMMA || op == FIN_BETA) {
            if (op == FIN_BETA) sc->beta = sc->gamma > 0.0 ? sum / sc->gamma : 0.0;
            sc->gamma = sum;
            sc->kappa = (scale_q && sum > 0.0 && isfinite(sum)) ? 1.0 / sqrt(sum) : 1.0;
        } else if (op == FIN_ALPHA) {
            sc->delta = sum;
            sc->alpha = (sc->gamma > 0.0 && sum > 0.0) ? sc->gamma / sum : 0.0;
        } else {
            sc->rr = sum;
        }
    }
}

static cbct_status finalize(const double *partials, int n, Scalars *sc, int op, cudaStream_t st, int scale_q = 0)
{
    CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_finalize<<<1, 1024, 0, st>>>(partials, n, sc, op, scale_q));
    return check_cuda(cudaGetLastError(), "finalize launch");
}

static int vec_blocks(size_t n)
{
    const size_t per = 256 * 4;
    size_t b = (n + per - 1) / per;
    const size_t cap = 16ull * device_sm_count();
    if (b > cap) b = cap;
    return b < 1 ? 1 : (int)b;
}

// Four consecutive values as FP32 (one 16-byte or 8-byte load) and back.
__device__ __forceinline__ float4 load4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void store4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float4 load4(const __nv_bfloat16 *p)
{
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store4(__nv_bfloat16 *p, float4 v)
{
    uint2 raw;
    *reinterpret_cast<__nv_bfloat162 *>(&raw.x) = __floats2bfloat162_rn(v.x, v.y);
    *reinterpret_cast<__nv_bfloat162 *>(&raw.y) = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<uint2 *>(p) = raw;
}
__device__ __forceinline__ float4 load4(const __half *p)
{
    const uint2 raw = *reinterpret_cast<const uint2 *>(p);
    const float2 a = __half22float2(*reinterpret_cast<const __half2 *>(&raw.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2 *>(&raw.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void store4(__half *p, float4 v)
{
    uint2 raw;
    *reinterpret_cast<__half2 *>(&raw.x) = __floats2half2_rn(v.x, v.y);
    *reinterpret_cast<__half2 *>(&raw.y) = __floats2half2_rn(v.z, v.w);
    *reinterpret_cast<uint2 *>(p) = raw;
}

// r -= alpha q, with q stored as kappa q: r -= (alpha / kappa) q_stored. FP32 arithmetic,
// r and q in the storage type T (both buffers 256-byte aligned).
template <typename T>
__global__ void k_update_r(T *__restrict__ r, const T *__restrict__ q, const Scalars *sc, size_t n)
{
    const float a = (float)(sc->alpha / sc->kappa);
    const size_t n4 = n / 4;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 rv = load4(r + 4 * i);
        const float4 qv = load4(q + 4 * i);
        rv.x = fmaf(-a, qv.x, rv.x);
        rv.y = fmaf(-a, qv.y, rv.y);
        rv.z = fmaf(-a, qv.z, rv.z);
        rv.w = fmaf(-a, qv.w, rv.w);
        store4(r + 4 * i, rv);
    }
    for (size_t i = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float rv = fmaf(-a, load_as_float(q + i), load_as_float(r + i));
        store_from_float(r + i, rv);
    }
}

static cbct_status launch_update_r(void *r, const void *q, const Scalars *sc, size_t n, int storage, cudaStream_t st)
{
    if (storage == ST_BF16)
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_update_r<<<vec_blocks(n), 256, 0, st>>>(static_cast<__nv_bfloat16 *>(r),
                                                             static_cast<const __nv_bfloat16 *>(q), sc, n));
    else if (storage == ST_F16)
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_update_r<<<vec_blocks(n), 256, 0, st>>>(static_cast<__half *>(r), static_cast<const __half *>(q),
                                                             sc, n));
    else
        CBCT_TIMED(CBCT_KERNEL_OTHER, st,
                   k_update_r<<<vec_blocks(n), 256, 0, st>>>(static_cast<float *>(r), static_cast<const float *>(q), sc, n));
    return check_cuda(cudaGetLastError(), "update launch");
}

// x += alpha p; and if with_p: p = s + beta p
__global__ void k_update_xp(float *__restrict__ x, float *__restrict__ p, const float *__restrict__ s,
                            const Scalars *sc, size_t n, int with_p)
{
    const float a = (float)sc->alpha, b = (float)sc->beta;
    const size_t n4 = n / 4;
    float4 *x4 = reinterpret_cast<float4 *>(x);
    float4 *p4 = reinterpret_cast<float4 *>(p);
    const float4 *s4 = reinterpret_cast<const float4 *>(s);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        float4 xv = x4[i];
        float4 pv = p4[i];
        xv.x = fmaf(a, pv.x, xv.x);
        xv.y = fmaf(a, pv.y, xv.y);
        xv.z = fmaf(a, pv.z, xv.z);
        xv.w = fmaf(a, pv.w, xv.w);
        x4[i] = xv;
        if (with_p) {
            const float4 sv = s4[i];
            pv.x = fmaf(b, pv.x, sv.x);
            pv.y = fmaf(b, pv.y, sv.y);
            pv.z = fmaf(b, pv.z, sv.z);
            pv.w = fmaf(b, pv.w, sv.w);
            p4[i] = pv;
        }
    }
    for (size_t i = 4 * n4 + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float pv = p[i];
        x[i] = fmaf(a, pv, x[i]);
        if (with_p) p[i] = fmaf(b, pv, s[i]);
    }
}

// ------------------------------------------------------------------------------------
// Layout conversion: public x-fastest [z][y][x] <-> internal z-fastest [y][x][z]
// ------------------------------------------------------------------------------------

__global__ void k_pub_to_int(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz)
{
    __shared__ float t[32][33];
    const int xb = blockIdx.x * 32, zb = blockIdx.y * 32, y = blockIdx.z;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int z = zb + j, x = xb + threadIdx.x;
        if (z < nz && x < nx) t[j][threadIdx.x] = in[((size_t)z * ny + y) * nx + x];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int x = xb + j, z = zb + threadIdx.x;
        if (z < nz && x < nx) out[((size_t)y * nx + x) * nz + z] = t[threadIdx.x][j];
    }
}

__global__ void k_int_to_pub(const float *__restrict__ in, float *__restrict__ out, int nx, int ny, int nz)
{
    __shared__ float t[32][33];
    const int xb = blockIdx.x * 32, zb = blockIdx.y * 32, y = blockIdx.z;
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int x = xb + j, z = zb + threadIdx.x;
        if (z < nz && x < nx) t[j][threadIdx.x] = in[((size_t)y * nx + x) * nz + z];
    }
    __syncthreads();
    for (int j = threadIdx.y; j < 32; j += 8) {
        const int z = zb + j, x = xb + threadIdx.x;
        if (z < nz && x < nx) out[((size_t)z * ny + y) * nx + x] = t[threadIdx.x][j];
    }
}

cbct_status transpose(const float *in, float *out, int nx, int ny, int nz, bool to_internal,
                      cudaStream_t st)
{
    dim3 grid((nx + 31) / 32, (nz + 31) / 32, ny), block(32, 8);
    if (to_internal) CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_pub_to_int<<<grid, block, 0, st>>>(in, out, nx, ny, nz));
    else CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_int_to_pub<<<grid, block, 0, st>>>(in, out, nx, ny, nz));
    return check_cuda(cudaGetLastError(), "transpose launch");
}

// ------------------------------------------------------------------------------------
// Multigrid transfer (Section 2.2.3). layout 0: x-fastest, 1: z-fastest.
// ------------------------------------------------------------------------------------

struct Grid3 {
    int n[3];
    float h[3];
};

__device__ __forceinline__ void unflatten(size_t i, const int n[3], int layout, int c[3])
{
    if (layout == 0) {
        c[0] = (int)(i % n[0]);
        c[1] = (int)((i / n[0]) % n[1]);
        c[2] = (int)(i / ((size_t)n[0] * n[1]));
    } else {
        c[2] = (int)(i % n[2]);
        c[0] = (int)((i / n[2]) % n[0]);
        c[1] = (int)(i / ((size_t)n[2] * n[0]));
    }
}

__device__ __forceinline__ size_t flatten(const int n[3], int layout, int x, int y, int z)
{
    return layout == 0 ? ((size_t)z * n[1] + y) * n[0] + x : ((size_t)y * n[0] + x) * n[2] + z;
}

__global__ void k_prolong(Grid3 cg, const float *__restrict__ fc, Grid3 fg, float *__restrict__ ff, int layout)
{
    const size_t N = (size_t)fg.n[0] * fg.n[1] * fg.n[2];
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        int c[3], i0[3], i1[3];
        float w[3];
        unflatten(i, fg.n, layout, c);
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            // fine voxel centre in coarse index units, clamped to the coarse centres' hull
            const float pos = (c[a] + 0.5f - 0.5f * fg.n[a]) * fg.h[a];
            float xi = pos / cg.h[a] + 0.5f * cg.n[a] - 0.5f;
            xi = fminf(fmaxf(xi, 0.0f), (float)(cg.n[a] - 1));
            i0[a] = min((int)floorf(xi), cg.n[a] - 1);
            i1[a] = min(i0[a] + 1, cg.n[a] - 1);
            w[a] = xi - i0[a];
        }
        float acc = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int jx = (q & 1) ? i1[0] : i0[0], jy = (q & 2) ? i1[1] : i0[1], jz = (q & 4) ? i1[2] : i0[2];
            const float wt = ((q & 1) ? w[0] : 1.0f - w[0]) * ((q & 2) ? w[1] : 1.0f - w[1]) *
                             ((q & 4) ? w[2] : 1.0f - w[2]);
            acc = fmaf(wt, __ldg(fc + flatten(cg.n, layout, jx, jy, jz)), acc);
        }
        ff[i] = acc;
    }
}

// Each coarse voxel: mean of the fine voxels whose centres fall inside it. The owning
// coarse index of a fine centre is floor((pos - origin_c) / h_c), evaluated in FP64.
__global__ void k_restrict(Grid3 fg, const float *__restrict__ ff, Grid3 cg, float *__restrict__ fc,
                           double fh0, double fh1, double fh2, double ch0, double ch1, double ch2, int layout)
{
    const size_t N = (size_t)cg.n[0] * cg.n[1] * cg.n[2];
    const double fh[3] = {fh0, fh1, fh2}, ch[3] = {ch0, ch1, ch2};
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (size_t)gridDim.x * blockDim.x) {
        int c[3], lo[3], hi[3];
        unflatten(i, cg.n, layout, c);
        bool empty = false;
        for (int a = 0; a < 3; ++a) {
            // candidate fine indices around the coarse voxel, then exact ownership test
            const double ratio = ch[a] / fh[a];
            const double first = (c[a] * ch[a] - 0.5 * cg.n[a] * ch[a] + 0.5 * fg.n[a] * fh[a]) / fh[a] - 0.5;
            lo[a] = max(0, (int)floor(first) - 1);
            hi[a] = min(fg.n[a] - 1, (int)ceil(first + ratio) + 1);
            int l2 = hi[a] + 1, h2 = lo[a] - 1;
            for (int j = lo[a]; j <= hi[a]; ++j) {
                const double pos = -0.5 * fg.n[a] * fh[a] + (j + 0.5) * fh[a];
                const int own = (int)floor((pos + 0.5 * cg.n[a] * ch[a]) / ch[a]);
                if (own == c[a]) {
                    l2 = min(l2, j);
                    h2 = max(h2, j);
                }
            }
            lo[a] = l2;
            hi[a] = h2;
            if (l2 > h2) empty = true;
        }
        float out = 0.0f;
        if (!empty) {
            double s = 0.0;
            for (int z = lo[2]; z <= hi[2]; ++z)
                for (int y = lo[1]; y <= hi[1]; ++y)
                    for (int x = lo[0]; x <= hi[0]; ++x) s += ff[flatten(fg.n, layout, x, y, z)];
            const double cnt = (double)(hi[0] - lo[0] + 1) * (hi[1] - lo[1] + 1) * (hi[2] - lo[2] + 1);
            out = (float)(s / cnt);
        }
        fc[i] = out;
    }
}

static Grid3 grid3(int nx, int ny, int nz, double dx, double dy, double dz)
{
    Grid3 g;
    g.n[0] = nx; g.n[1] = ny; g.n[2] = nz;
    g.h[0] = (float)dx; g.h[1] = (float)dy; g.h[2] = (float)dz;
    return g;
}

static cbct_status launch_prolong(const Grid3 &cg, const float *fc, const Grid3 &fg, float *ff, int layout,
                                  cudaStream_t st)
{
    const size_t N = (size_t)fg.n[0] * fg.n[1] * fg.n[2];
    CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_prolong<<<vec_blocks(N), 256, 0, st>>>(cg, fc, fg, ff, layout));
    return check_cuda(cudaGetLastError(), "prolong launch");
}

// ------------------------------------------------------------------------------------
// Workspace
// ------------------------------------------------------------------------------------

struct Work {
    float *X, *X2, *P, *S, *Fa, *Fb; // X, X2: the CGLS iterate and the next momentum point
    void *R, *Q; // residual and projected search direction: n_views*nv*nu values of the storage type
    float2 *PS; // row prefix sums of the prescaled residual, input of the adjoint
    void *TR[MAX_LEVELS]; // per level: the projector's trace table (internal layout strides)
    double *partials;
    Scalars *sc;
};

static size_t prefix_elems(const cbct_geometry_desc &d) { return (size_t)d.n_views * d.nu * ((size_t)d.nv + 1); }

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static size_t max_partials(const cbct_geometry *g)
{
    GeomDev G = level_geom(g, 0);
    size_t a = (size_t)project_num_blocks(G);
    // backprojection blocks are most numerous with one z voxel per thread at the finest grid
    size_t b = (size_t)backproject_max_blocks(G);
    return a > b ? a : b;
}

static size_t work_layout(const cbct_geometry *g, char *base, Work *w)
{
    const cbct_geometry_desc &d = g->desc;
    const size_t N = (size_t)d.nx * d.ny * d.nz, M = (size_t)d.n_views * d.nv * d.nu;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char *p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t VB = 4 * N + PROJECT_VOLUME_SLACK; // volumes the projector may read past the end
    float *X = (float *)take(VB), *X2 = (float *)take(VB), *P = (float *)take(VB), *S = (float *)take(VB);
    float *Fa = (float *)take(VB), *Fb = (float *)take(VB);
    void *R = take(4 * M), *Q = take(4 * M); // sized for FP32, the widest storage type
    float2 *PS = (float2 *)take(sizeof(float2) * prefix_elems(d));
    void *TR[MAX_LEVELS];
    for (int lev = 0; lev < MAX_LEVELS; ++lev) TR[lev] = take(trace_table_bytes(level_geom(g, lev)));
    double *partials = (double *)take(sizeof(double) * max_partials(g));
    Scalars *sc = (Scalars *)take(sizeof(Scalars));
    if (w) {
        *w = Work{X, X2, P, S, Fa, Fb, R, Q, PS, {}, partials, sc};
        for (int lev = 0; lev < MAX_LEVELS; ++lev) w->TR[lev] = TR[lev];
    }
    return off;
}

static cbct_status get_work(cbct_geometry *g, void *ws, size_t ws_bytes, Work *w)
{
    const size_t need = work_layout(g, nullptr, nullptr);
    if (ws) {
        if (ws_bytes < need)
            return set_error(CBCT_ERR_OUT_OF_MEMORY, "workspace too small: %zu < %zu bytes", ws_bytes, need);
        if (((uintptr_t)ws & 255) != 0) return set_error(CBCT_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
        work_layout(g, (char *)ws, w);
        return CBCT_OK;
    }
    if (!g->d_ws || g->ws_bytes < need) {
        if (g->d_ws) {
            cudaDeviceSynchronize();
            cudaFree(g->d_ws);
            g->d_ws = nullptr;
            g->ws_bytes = 0;
        }
        cudaError_t e = cudaMalloc(&g->d_ws, need);
        if (e != cudaSuccess) return check_cuda(e, "workspace allocation");
        g->ws_bytes = need;
    }
    work_layout(g, (char *)g->d_ws, w);
    return CBCT_OK;
}

// ------------------------------------------------------------------------------------
// CGLS (Appendix 1) on the internal layout; x is read and updated in place.
// ------------------------------------------------------------------------------------

#define TRY(expr)                                                                                  \
    do {                                                                                           \
        cbct_status _s = (expr);                                                                   \
        if (_s != CBCT_OK) return _s;                                                              \
    } while (0)

static cbct_status run_cgls(const GeomDev &G, const float *y, float *x, int n_iter, const Work &w, int storage,
                            const void *traces, cudaStream_t st)
{
    const long long sz = 1, sx = G.nz, sy = (long long)G.nx * G.nz;
    const size_t N = (size_t)G.nx * G.ny * G.nz, M = (size_t)G.nviews * G.nv * G.nu;
    const int nbp = project_num_blocks(G), nbb = backproject_num_blocks(G);
    // FP32 storage holds |D-S| r and |D-S| q; 16-bit storage holds r and kappa q and the
    // row prefix applies |D-S|. Only FP16 needs kappa (BF16 has FP32's exponent range).
    const int prescale = storage == ST_F32 ? 0 : 1;
    const int scale_q = storage == ST_F16 ? 1 : 0;
    // r = y - P x; s = P^T r; p = s; gamma = ||s||^2
    TRY(launch_project(G, x, sx, sy, sz, y, w.R, PM_RESID, w.partials, 0.0f, st, storage, w.sc, traces));
    TRY(finalize(w.partials, nbp, w.sc, FIN_RR, st));
    TRY(launch_row_prefix(G, w.R, w.PS, prescale, st, storage));
    TRY(launch_backproject(G, w.PS, w.S, sx, sy, sz, w.P, w.partials, st));
    TRY(finalize(w.partials, nbb, w.sc, FIN_GAMMA, st, scale_q));
    for (int l = 0; l < n_iter; ++l) {
        // q = P p, alpha = gamma / ||q||^2
        TRY(launch_project(G, w.P, sx, sy, sz, nullptr, w.Q, PM_Q_SCALED, w.partials, 0.0f, st, storage, w.sc,
                           traces));
        TRY(finalize(w.partials, nbp, w.sc, FIN_ALPHA, st));
        if (l == n_iter - 1) { // last update: x only; s and p would not be used again
            CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_update_xp<<<vec_blocks(N), 256, 0, st>>>(x, w.P, w.S, w.sc, N, 0));
            TRY(check_cuda(cudaGetLastError(), "update launch"));
            break;
        }
        TRY(launch_update_r(w.R, w.Q, w.sc, M, storage, st));
        // s = P^T r, beta = ||s||^2 / gamma
        TRY(launch_row_prefix(G, w.R, w.PS, prescale, st, storage));
        TRY(launch_backproject(G, w.PS, w.S, sx, sy, sz, nullptr, w.partials, st));
        TRY(finalize(w.partials, nbb, w.sc, FIN_BETA, st, scale_q));
        // x += alpha p; p = s + beta p
        CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_update_xp<<<vec_blocks(N), 256, 0, st>>>(x, w.P, w.S, w.sc, N, 1));
        TRY(check_cuda(cudaGetLastError(), "update launch"));
    }
    return CBCT_OK;
}

static cbct_status read_flags(const Work &w, cudaStream_t st)
{
    unsigned int flags = 0;
    cudaError_t e = cudaMemcpyAsync(&flags, &w.sc->flags, sizeof(flags), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return check_cuda(e, "status read-back");
    if (flags & 2u) return set_error(CBCT_ERR_TIMEOUT, "a projector block timed out waiting for its trace record");
    if (flags & 1u) return set_error(CBCT_ERR_NONFINITE, "an inner product of the iteration was not finite");
    return CBCT_OK;
}

static cbct_status reset_scalars(const Work &w, cudaStream_t st)
{
    return check_cuda(cudaMemsetAsync(w.sc, 0, sizeof(Scalars), st), "scalar reset");
}

// ------------------------------------------------------------------------------------
// Algorithm A2 on one level and the multigrid driver
// ------------------------------------------------------------------------------------

// One iteration k of Algorithm A2 on one level: CGLS from the momentum point X, then
// f^(k+1) = H(D^T T_mu D x) fused with the next momentum point
// v^(k+1) = f^(k+1) + (t^(k) - 1) / t^(k+1) (f^(k+1) - f^(k)) into X2 (skipped on the
// level's last iteration); t is advanced to t^(k+1). Internal layout: axis 0 = z,
// axis 1 = x, axis 2 = y.
static cbct_status run_a2_iteration(const GeomDev &G, const float *y, float mu, bool last, const cbct_recon_opts &o,
                                    Work &w, const void *traces, double &t, float **f_cur, float **f_other,
                                    cudaStream_t st)
{
    TRY(run_cgls(G, y, w.X, o.n_cgls, w, o.storage, traces, st));
    const double t_next = 0.5 * (1.0 + std::sqrt(1.0 + 4.0 * t * t));
    const float c = o.momentum ? (float)((t - 1.0) / t_next) : 0.0f;
    TRY(launch_tf_shrink_fused(G.nz, G.nx, G.ny, w.X, mu, o.positivity, *f_other, *f_cur, c, last ? nullptr : w.X2,
                               st));
    std::swap(*f_cur, *f_other);
    std::swap(w.X, w.X2);
    t = t_next;
    return CBCT_OK;
}

// A reconstruction as a sequence of steps, each one A2 iteration of one level; a level's
// set-up (the zero start on the coarsest grid, the prolongation onto the next) rides on
// its first step and the change back to the public layout on the last. Enqueued step by
// step, on one stream or handed from stream to stream, it issues exactly the launches of
// the whole-run enqueue below (which is this loop), so the results are bit-identical.
struct ReconCursor {
    const float *y = nullptr;
    cbct_geometry *g = nullptr;
    float mu = 0.0f;
    int levels = 1;
    std::vector<int> iters;
    cbct_recon_opts o{};
    float *f_out = nullptr;
    Work w{};
    bool started = false, finished = false, need_setup = true;
    int lev = 0, k = 0;  // current level (levels - 1 = coarsest) and its next A2 iteration
    double t = 1.0;      // t^(k) of Algorithm A2 on the current level
    float *f_cur = nullptr, *f_other = nullptr;
    GeomDev Gprev{};
};

cbct_status reconstruct_cursor_create(const float *y, cbct_geometry *g, float mu, int levels, const int *iters,
                                      const cbct_recon_opts &o, void *ws, size_t ws_bytes, float *f_out,
                                      ReconCursor **out)
{
    std::unique_ptr<ReconCursor> c(new ReconCursor());
    TRY(get_work(g, ws, ws_bytes, &c->w));
    c->y = y;
    c->g = g;
    c->mu = mu;
    c->levels = levels;
    c->iters.assign(iters, iters + levels);
    c->o = o;
    c->f_out = f_out;
    *out = c.release();
    return CBCT_OK;
}

void reconstruct_cursor_destroy(ReconCursor *c) { delete c; }

bool reconstruct_cursor_finished(const ReconCursor *c) { return c->finished; }

cbct_status reconstruct_cursor_step(ReconCursor *c, cudaStream_t st)
{
    if (c->finished) return CBCT_OK;
    Work &w = c->w;
    if (!c->started) {
        TRY(reset_scalars(w, st));
        // the projector's trace table of every level, once per reconstruction (the iteration's
        // volumes are z-contiguous: strides nz and nx nz)
        for (int lev = 0; lev < c->levels; ++lev) {
            const GeomDev G = level_geom(c->g, lev);
            TRY(launch_trace_table(G, G.nz, (long long)G.nx * G.nz, w.TR[lev], st));
        }
        c->f_cur = w.Fa;
        c->f_other = w.Fb;
        c->lev = c->levels - 1;
        c->k = 0;
        c->need_setup = true;
        c->started = true;
    }
    for (;;) {
        if (c->lev < 0) { // every level done: the volume back to the public layout
            const GeomDev G0 = level_geom(c->g, 0);
            TRY(transpose(c->f_cur, c->f_out, G0.nx, G0.ny, G0.nz, false, st));
            c->finished = true;
            return CBCT_OK;
        }
        const GeomDev G = level_geom(c->g, c->lev);
        const size_t N = (size_t)G.nx * G.ny * G.nz;
        const int iters = c->iters[c->levels - 1 - c->lev];
        if (c->need_setup) {
            if (c->lev == c->levels - 1) {
                TRY(check_cuda(cudaMemsetAsync(c->f_cur, 0, sizeof(float) * N, st), "memset"));
            } else {
                const GeomDev &P = c->Gprev;
                TRY(launch_prolong(grid3(P.nx, P.ny, P.nz, P.dx, P.dy, P.dz), c->f_cur,
                                   grid3(G.nx, G.ny, G.nz, G.dx, G.dy, G.dz), c->f_other, 1, st));
                std::swap(c->f_cur, c->f_other);
            }
            // v^(0) = f^(0): the first momentum coefficient is 0
            TRY(check_cuda(cudaMemcpyAsync(w.X, c->f_cur, sizeof(float) * N, cudaMemcpyDeviceToDevice, st), "copy"));
            c->t = 1.0;
            c->need_setup = false;
        }
        const bool had_iteration = c->k < iters;
        if (had_iteration) {
            TRY(run_a2_iteration(G, c->y, c->mu, c->k + 1 == iters, c->o, w, w.TR[c->lev], c->t, &c->f_cur,
                                 &c->f_other, st));
            c->k++;
        }
        if (c->k >= iters) { // level done: the next one starts with the prolongation
            c->Gprev = G;
            c->lev--;
            c->k = 0;
            c->need_setup = true;
            if (c->lev < 0) continue; // the final layout change belongs to this step
        }
        if (had_iteration) return CBCT_OK;
    }
}

cbct_status reconstruct_enqueue(const float *y, cbct_geometry *g, float mu, int levels, const int *iters,
                                const cbct_recon_opts &o, void *ws, size_t ws_bytes, float *f_out, cudaStream_t st)
{
    ReconCursor *c = nullptr;
    TRY(reconstruct_cursor_create(y, g, mu, levels, iters, o, ws, ws_bytes, f_out, &c));
    std::unique_ptr<ReconCursor> hold(c);
    while (!c->finished) TRY(reconstruct_cursor_step(c, st));
    return CBCT_OK;
}

size_t reconstruct_ws_bytes(const cbct_geometry *g) { return work_layout(g, nullptr, nullptr); }

const unsigned int *reconstruct_flags_address(const cbct_geometry *g, void *ws)
{
    Work w;
    work_layout(g, (char *)ws, &w);
    return &w.sc->flags;
}

static cbct_status reconstruct_impl(const float *y, cbct_geometry *g, float mu, int levels, const int *iters,
                                    const cbct_recon_opts &o, void *ws, size_t ws_bytes, float *f_out,
                                    cudaStream_t st)
{
    TRY(reconstruct_enqueue(y, g, mu, levels, iters, o, ws, ws_bytes, f_out, st));
    Work w;
    TRY(get_work(g, ws, ws_bytes, &w));
    return read_flags(w, st);
}

} // namespace cbct

using namespace cbct;

static cbct_status check_geom(const cbct_geometry *g, const char *what)
{
    if (!g) return set_error(CBCT_ERR_INVALID_ARG, "%s: null geometry", what);
    int dev = -1;
    cudaGetDevice(&dev);
    if (dev != g->device) return set_error(CBCT_ERR_INVALID_ARG, "%s: geometry belongs to device %d, current is %d", what, g->device, dev);
    return CBCT_OK;
}

static bool valid_dtype(int t) { return t == CBCT_F32 || t == CBCT_BF16 || t == CBCT_F16; }

extern "C" cbct_status cbct_project_ex(const cbct_geometry *gc, const float *f, void *g_out, cbct_dtype g_type,
                                       cbct_stream_t stream)
{
    TRY(check_geom(gc, "project"));
    if (!f || !g_out) return set_error(CBCT_ERR_INVALID_ARG, "project: null pointer");
    if (!valid_dtype(g_type)) return set_error(CBCT_ERR_INVALID_ARG, "project: unknown storage type %d", (int)g_type);
    cbct_geometry *g = const_cast<cbct_geometry *>(gc);
    const GeomDev G = level_geom(g, 0);
    const size_t N = (size_t)G.nx * G.ny * G.nz;
    const size_t vol_bytes = align256(sizeof(float) * N + PROJECT_VOLUME_SLACK);
    TRY(ensure_scratch(g, vol_bytes + trace_table_bytes(G)));
    cudaStream_t st = (cudaStream_t)stream;
    float *fz = g->d_scratch;
    void *traces = reinterpret_cast<char *>(g->d_scratch) + vol_bytes;
    TRY(transpose(f, fz, G.nx, G.ny, G.nz, true, st));
    TRY(launch_trace_table(G, G.nz, (long long)G.nx * G.nz, traces, st));
    return launch_project(G, fz, G.nz, (long long)G.nx * G.nz, 1, nullptr, g_out, PM_PLAIN, nullptr, 0.0f, st,
                          (int)g_type, nullptr, traces);
}

extern "C" cbct_status cbct_project(const cbct_geometry *gc, const float *f, float *g_out, cbct_stream_t stream)
{
    return cbct_project_ex(gc, f, g_out, CBCT_F32, stream);
}

extern "C" cbct_status cbct_backproject_ex(const cbct_geometry *gc, const void *gin, cbct_dtype g_type, float *f,
                                           cbct_stream_t stream)
{
    TRY(check_geom(gc, "backproject"));
    if (!gin || !f) return set_error(CBCT_ERR_INVALID_ARG, "backproject: null pointer");
    if (!valid_dtype(g_type)) return set_error(CBCT_ERR_INVALID_ARG, "backproject: unknown storage type %d", (int)g_type);
    cbct_geometry *g = const_cast<cbct_geometry *>(gc);
    const GeomDev G = level_geom(g, 0);
    TRY(ensure_scratch(g, sizeof(float2) * prefix_elems(g->desc)));
    cudaStream_t st = (cudaStream_t)stream;
    float2 *ps = reinterpret_cast<float2 *>(g->d_scratch);
    TRY(launch_row_prefix(G, gin, ps, 1, st, (int)g_type));
    return launch_backproject(G, ps, f, 1, G.nx, (long long)G.nx * G.ny, nullptr, nullptr, st);
}

extern "C" cbct_status cbct_backproject(const cbct_geometry *gc, const float *gin, float *f, cbct_stream_t stream)
{
    return cbct_backproject_ex(gc, gin, CBCT_F32, f, stream);
}

extern "C" cbct_status cbct_tf_analyze_ex(int nx, int ny, int nz, const float *f, void *alpha27, cbct_dtype a_type,
                                          cbct_stream_t stream)
{
    if (nx < 1 || ny < 1 || nz < 1) return set_error(CBCT_ERR_INVALID_ARG, "tf_analyze: sizes must be >= 1");
    if (ny > 65535 * 8) return set_error(CBCT_ERR_INVALID_ARG, "tf_analyze: ny too large");
    if (!f || !alpha27) return set_error(CBCT_ERR_INVALID_ARG, "tf_analyze: null pointer");
    if ((double)nx * ny * nz * 27.0 > 9.2e18) return set_error(CBCT_ERR_INVALID_ARG, "tf_analyze: too large");
    if (!valid_dtype(a_type)) return set_error(CBCT_ERR_INVALID_ARG, "tf_analyze: unknown storage type %d", (int)a_type);
    return launch_tf_analyze(nx, ny, nz, f, alpha27, (cudaStream_t)stream, (int)a_type);
}

extern "C" cbct_status cbct_tf_analyze(int nx, int ny, int nz, const float *f, float *alpha27, cbct_stream_t stream)
{
    return cbct_tf_analyze_ex(nx, ny, nz, f, alpha27, CBCT_F32, stream);
}

extern "C" cbct_status cbct_tf_synthesize_shrink_ex(int nx, int ny, int nz, const void *alpha27, cbct_dtype a_type,
                                                    float mu, int positivity, float *f, cbct_stream_t stream)
{
    if (nx < 1 || ny < 1 || nz < 1) return set_error(CBCT_ERR_INVALID_ARG, "tf_synthesize_shrink: sizes must be >= 1");
    if (ny > 65535 * 8) return set_error(CBCT_ERR_INVALID_ARG, "tf_synthesize_shrink: ny too large");
    if (!f || !alpha27) return set_error(CBCT_ERR_INVALID_ARG, "tf_synthesize_shrink: null pointer");
    if (!(mu >= 0.0f) || !std::isfinite(mu)) return set_error(CBCT_ERR_INVALID_ARG, "tf_synthesize_shrink: mu must be finite and >= 0");
    if (!valid_dtype(a_type))
        return set_error(CBCT_ERR_INVALID_ARG, "tf_synthesize_shrink: unknown storage type %d", (int)a_type);
    return launch_tf_synth_shrink(nx, ny, nz, alpha27, mu, positivity, f, (cudaStream_t)stream, (int)a_type);
}

extern "C" cbct_status cbct_tf_synthesize_shrink(int nx, int ny, int nz, const float *alpha27, float mu,
                                                 int positivity, float *f, cbct_stream_t stream)
{
    return cbct_tf_synthesize_shrink_ex(nx, ny, nz, alpha27, CBCT_F32, mu, positivity, f, stream);
}

extern "C" cbct_status cbct_reconstruct_workspace_size(const cbct_geometry *g, size_t *bytes)
{
    if (!g || !bytes) return set_error(CBCT_ERR_INVALID_ARG, "workspace_size: null argument");
    *bytes = work_layout(g, nullptr, nullptr);
    return CBCT_OK;
}

namespace cbct {
cbct_status validate_recon_args(float mu, float lambda, int levels, const int *iters, const cbct_recon_opts &o)
{
    if (!iters) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: null pointer");
    if (!(mu >= 0.0f) || !std::isfinite(mu)) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: mu must be finite and >= 0");
    if (!std::isfinite(lambda)) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: lambda must be finite");
    if (lambda != 0.0f)
        return set_error(CBCT_ERR_UNSUPPORTED, "reconstruct: lambda must be 0 (the method's only parameter is mu)");
    if (levels < 1 || levels > MAX_LEVELS)
        return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: levels must be in 1..%d", MAX_LEVELS);
    for (int i = 0; i < levels; ++i)
        if (iters[i] < 0 || iters[i] > 100000) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: bad iteration count");
    if (o.n_cgls < 1 || o.n_cgls > 1000) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: n_cgls must be in 1..1000");
    if (o.storage != CBCT_F32 && o.storage != CBCT_BF16 && o.storage != CBCT_F16)
        return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: storage must be CBCT_F32, CBCT_BF16 or CBCT_F16");
    return CBCT_OK;
}
} // namespace cbct

static cbct_status validate_recon(const float *y, const cbct_geometry *g, float mu, float lambda, int levels,
                                  const int *iters, float *f_out, const cbct_recon_opts &o)
{
    TRY(check_geom(g, "reconstruct"));
    if (!y || !f_out || !iters) return set_error(CBCT_ERR_INVALID_ARG, "reconstruct: null pointer");
    return validate_recon_args(mu, lambda, levels, iters, o);
}

extern "C" cbct_status cbct_reconstruct_ex(const float *y, const cbct_geometry *g, float mu, float lambda,
                                           int levels, const int *iters, const cbct_recon_opts *opts,
                                           void *workspace, size_t workspace_bytes, float *f_out,
                                           cbct_stream_t stream)
{
    cbct_recon_opts o{3, 1, 1, CBCT_F32};
    if (opts) o = *opts;
    TRY(validate_recon(y, g, mu, lambda, levels, iters, f_out, o));
    return reconstruct_impl(y, const_cast<cbct_geometry *>(g), mu, levels, iters, o, workspace, workspace_bytes,
                            f_out, (cudaStream_t)stream);
}

extern "C" cbct_status cbct_reconstruct(const float *y, const cbct_geometry *g, float mu, float lambda, int levels,
                                        const int *iters, float *f_out, cbct_stream_t stream)
{
    return cbct_reconstruct_ex(y, g, mu, lambda, levels, iters, nullptr, nullptr, 0, f_out, stream);
}

extern "C" cbct_status cbct_cgls(const cbct_geometry *gc, const float *y, float *x, int n_iter, cbct_stream_t stream)
{
    TRY(check_geom(gc, "cgls"));
    if (!y || !x) return set_error(CBCT_ERR_INVALID_ARG, "cgls: null pointer");
    if (n_iter < 0) return set_error(CBCT_ERR_INVALID_ARG, "cgls: n_iter must be >= 0");
    cbct_geometry *g = const_cast<cbct_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    Work w;
    TRY(get_work(g, nullptr, 0, &w));
    TRY(reset_scalars(w, st));
    const GeomDev G = level_geom(g, 0);
    TRY(transpose(x, w.Fa, G.nx, G.ny, G.nz, true, st));
    TRY(launch_trace_table(G, G.nz, (long long)G.nx * G.nz, w.TR[0], st));
    if (n_iter > 0) TRY(run_cgls(G, y, w.Fa, n_iter, w, ST_F32, w.TR[0], st));
    TRY(transpose(w.Fa, x, G.nx, G.ny, G.nz, false, st));
    return read_flags(w, st);
}

extern "C" cbct_status cbct_prolong(int cnx, int cny, int cnz, double cdx, double cdy, double cdz, const float *fc,
                                    int nx, int ny, int nz, double dx, double dy, double dz, float *ff,
                                    cbct_stream_t stream)
{
    if (cnx < 1 || cny < 1 || cnz < 1 || nx < 1 || ny < 1 || nz < 1)
        return set_error(CBCT_ERR_INVALID_ARG, "prolong: sizes must be >= 1");
    if (!(cdx > 0 && cdy > 0 && cdz > 0 && dx > 0 && dy > 0 && dz > 0))
        return set_error(CBCT_ERR_INVALID_ARG, "prolong: spacings must be > 0");
    if (!fc || !ff) return set_error(CBCT_ERR_INVALID_ARG, "prolong: null pointer");
    return launch_prolong(grid3(cnx, cny, cnz, cdx, cdy, cdz), fc, grid3(nx, ny, nz, dx, dy, dz), ff, 0,
                          (cudaStream_t)stream);
}

extern "C" cbct_status cbct_restrict(int nx, int ny, int nz, double dx, double dy, double dz, const float *ff,
                                     int cnx, int cny, int cnz, double cdx, double cdy, double cdz, float *fc,
                                     cbct_stream_t stream)
{
    if (cnx < 1 || cny < 1 || cnz < 1 || nx < 1 || ny < 1 || nz < 1)
        return set_error(CBCT_ERR_INVALID_ARG, "restrict: sizes must be >= 1");
    if (!(cdx > 0 && cdy > 0 && cdz > 0 && dx > 0 && dy > 0 && dz > 0))
        return set_error(CBCT_ERR_INVALID_ARG, "restrict: spacings must be > 0");
    if (!fc || !ff) return set_error(CBCT_ERR_INVALID_ARG, "restrict: null pointer");
    const size_t N = (size_t)cnx * cny * cnz;
    cudaStream_t st = (cudaStream_t)stream;
    CBCT_TIMED(CBCT_KERNEL_OTHER, st, k_restrict<<<vec_blocks(N), 256, 0, st>>>(grid3(nx, ny, nz, dx, dy, dz), ff,
                                                                grid3(cnx, cny, cnz, cdx, cdy, cdz), fc, dx, dy, dz,
                                                                cdx, cdy, cdz, 0));
    return check_cuda(cudaGetLastError(), "restrict launch");
}

extern "C" cbct_status cbct_backproject_eq3(const cbct_geometry *gc, const float *gin, float *f, cbct_stream_t stream)
{
    TRY(check_geom(gc, "backproject_eq3"));
    if (!gin || !f) return set_error(CBCT_ERR_INVALID_ARG, "backproject_eq3: null pointer");
    const GeomDev G = level_geom(gc, 0);
    const cbct_geometry_desc &d = gc->desc;
    const float pref = (float)(d.dx * d.dy * d.dz / (d.du * d.dv));
    return launch_backproject_eq3(G, gin, f, pref, (cudaStream_t)stream);
}

extern "C" cbct_status cbct_project_batch(const cbct_geometry *gc, int batch, const float *f, float *g,
                                          cbct_stream_t stream)
{
    TRY(check_geom(gc, "project_batch"));
    if (batch < 0 || (batch > 0 && (!f || !g))) return set_error(CBCT_ERR_INVALID_ARG, "project_batch: bad arguments");
    const cbct_geometry_desc &d = gc->desc;
    const size_t N = (size_t)d.nx * d.ny * d.nz, M = (size_t)d.n_views * d.nv * d.nu;
    for (int b = 0; b < batch; ++b) TRY(cbct_project(gc, f + b * N, g + b * M, stream));
    return CBCT_OK;
}

extern "C" cbct_status cbct_backproject_batch(const cbct_geometry *gc, int batch, const float *g, float *f,
                                              cbct_stream_t stream)
{
    TRY(check_geom(gc, "backproject_batch"));
    if (batch < 0 || (batch > 0 && (!f || !g))) return set_error(CBCT_ERR_INVALID_ARG, "backproject_batch: bad arguments");
    const cbct_geometry_desc &d = gc->desc;
    const size_t N = (size_t)d.nx * d.ny * d.nz, M = (size_t)d.n_views * d.nv * d.nu;
    for (int b = 0; b < batch; ++b) TRY(cbct_backproject(gc, g + b * M, f + b * N, stream));
    return CBCT_OK;
}

extern "C" cbct_status cbct_tf_shrink(int nx, int ny, int nz, const float *f, float mu, int positivity, float *out,
                                      cbct_stream_t stream)
{
    if (nx < 1 || ny < 1 || nz < 1) return set_error(CBCT_ERR_INVALID_ARG, "tf_shrink: sizes must be >= 1");
    if (ny > 65535 * 8) return set_error(CBCT_ERR_INVALID_ARG, "tf_shrink: ny too large");
    if (!f || !out) return set_error(CBCT_ERR_INVALID_ARG, "tf_shrink: null pointer");
    if (f == out) return set_error(CBCT_ERR_INVALID_ARG, "tf_shrink: input and output must differ");
    if (!(mu >= 0.0f) || !std::isfinite(mu)) return set_error(CBCT_ERR_INVALID_ARG, "tf_shrink: mu must be finite and >= 0");
    return launch_tf_shrink_fused(nx, ny, nz, f, mu, positivity, out, nullptr, 0.0f, nullptr, (cudaStream_t)stream);
}
