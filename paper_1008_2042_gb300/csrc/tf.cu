// Piecewise-linear tight frame (Section 2.1): analysis W, and vector shrinkage T_mu
// (Eq. (2)) + synthesis W^T + positivity H.
//
// The 3-D filters are tensor products of h0 = [1,2,1]/4, h1 = sqrt(2)/4 [1,0,-1],
// h2 = [-1,2,-1]/4, so both transforms run as three 3-tap passes. Arrays are addressed as
// (i2 * n1 + i1) * n0 + i0 with i0 the contiguous axis; channel i = l + 3m + 9n applies
// h_l along axis 0, h_m along axis 1 and h_n along axis 2. The boundary is periodic.
//
// GB300 mapping. Every kernel marches along axis 2 so that each input value is read from
// DRAM once and each output written once, with warps reading and writing rows along the
// contiguous axis. The analysis W owns a 32 x 8 tile of the (axis 0, axis 1) plane and
// keeps three planes of it in shared memory (with a one-voxel halo). The shrink +
// synthesis and the fused step give each lane whole positions and pass neighbour values by
// warp shuffles (axis 0), a shared exchange (axis 1) and registers (axis 2); they are
// described at their kernels. The public transforms are bandwidth bound: 4 B in + 108 B
// out per voxel for W, 108 B in + 4 B out for the shrink/synthesis (FP32 coefficients).
#include "cbct_internal.cuh"

namespace cbct {

constexpr int TA = 32, TB = 8, TF_THREADS = TA * TB;
constexpr float R2_4 = 0.35355339059327373f; // sqrt(2) / 4

__device__ __forceinline__ int wrapi(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// Analysis along one axis for the window (f(x-1), f(x), f(x+1)) = (p, c, n):
// alpha_l(x) = h_l[-1] f(x+1) + h_l[0] f(x) + h_l[1] f(x-1).
__device__ __forceinline__ void ana3(float p, float c, float n, float &o0, float &o1, float &o2)
{
    const float s = n + p;
    o0 = fmaf(0.25f, s, 0.5f * c);
    o1 = R2_4 * (n - p);
    o2 = fmaf(-0.25f, s, 0.5f * c);
}

// Synthesis along one axis: sum_l sum_k h_l[k] a_l(x + k) from the three channels at
// x-1 (P*), x (C*), x+1 (N*).
__device__ __forceinline__ float syn3(float P0, float C0, float N0, float P1, float N1, float P2,
                                      float C2, float N2)
{
    return fmaf(0.25f, (P0 + N0) - (P2 + N2), fmaf(0.5f, C0 + C2, R2_4 * (P1 - N1)));
}


template <typename TA_T>
__global__ void __launch_bounds__(TF_THREADS)
k_tf_analyze(int n0, int n1, int n2, int chunk, const float *__restrict__ f, TA_T *__restrict__ alpha)
{
    __shared__ float s[3][TB + 2][TA + 2];
    const int a0 = blockIdx.x * TA, b0 = blockIdx.y * TB;
    const int c_begin = blockIdx.z * chunk;
    const int c_end = min(n2, c_begin + chunk);
    if (c_begin >= c_end) return;
    const int tid = threadIdx.y * TA + threadIdx.x;
    const size_t N = (size_t)n0 * n1 * n2;

    int off[2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int pos = tid + k * TF_THREADS;
        if (pos < (TA + 2) * (TB + 2)) {
            const int r = pos / (TA + 2), q = pos - r * (TA + 2);
            off[k] = wrapi(b0 + r - 1, n1) * n0 + wrapi(a0 + q - 1, n0);
        } else {
            off[k] = -1;
        }
    }
    // the haloed tile of plane c: this thread's (at most two) values
    float nxt[2] = {0.0f, 0.0f};
    auto fetch = [&](int c) {
        const float *src = f + (size_t)wrapi(c, n2) * n1 * n0;
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (off[k] >= 0) nxt[k] = __ldg(src + off[k]);
    };
    auto put = [&](int slot) {
        float *d = &s[slot][0][0];
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (off[k] >= 0) d[tid + k * TF_THREADS] = nxt[k];
    };
    fetch(c_begin - 1);
    put(0);
    fetch(c_begin);
    put(1);
    fetch(c_begin + 1);
    const int ta = threadIdx.x, tb = threadIdx.y;
    const bool inside = a0 + ta < n0 && b0 + tb < n1;
    for (int c = c_begin; c < c_end; ++c) {
        const int j = c - c_begin;
        put((j + 2) % 3); // plane c + 1, loaded during the previous plane
        __syncthreads();
        if (c + 1 < c_end) fetch(c + 2); // lands while this plane is computed and stored
        if (inside) {
            const int sl[3] = {j % 3, (j + 1) % 3, (j + 2) % 3}; // planes c-1, c, c+1
            // axis 0 then axis 1: u[cc][m][l]
            float u[3][3][3];
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                float t[3][3]; // [bb][l]
#pragma unroll
                for (int bb = 0; bb < 3; ++bb)
                    ana3(s[sl[cc]][tb + bb][ta], s[sl[cc]][tb + bb][ta + 1], s[sl[cc]][tb + bb][ta + 2],
                         t[bb][0], t[bb][1], t[bb][2]);
#pragma unroll
                for (int l = 0; l < 3; ++l) ana3(t[0][l], t[1][l], t[2][l], u[cc][0][l], u[cc][1][l], u[cc][2][l]);
            }
            const size_t o = ((size_t)c * n1 + (b0 + tb)) * n0 + (a0 + ta);
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int l = 0; l < 3; ++l) {
                    float w0, w1, w2;
                    ana3(u[0][m][l], u[1][m][l], u[2][m][l], w0, w1, w2);
                    store_stream(alpha + (size_t)(l + 3 * m) * N + o, w0);
                    store_stream(alpha + (size_t)(l + 3 * m + 9) * N + o, w1);
                    store_stream(alpha + (size_t)(l + 3 * m + 18) * N + o, w2);
                }
        }
        __syncthreads();
    }
}

// Planes per block along axis 2 (shrink + synthesis and the fused step): the split whose blocks fill whole
// waves of the resident slots best, counting the two extra planes each block recomputes
// at its start (a block's cost grows with chunk + 2).
static int fused_chunk(long long tiles, int n2, int slots)
{
    int best = n2;
    double best_eff = -1.0;
    for (int nch = 1; nch <= n2; ++nch) {
        const int chunk = (n2 + nch - 1) / nch;
        if (nch > 1 && chunk == (n2 + nch - 2) / (nch - 1)) continue; // same split as nch - 1
        const long long nb = tiles * ((n2 + chunk - 1) / chunk);
        const long long waves = (nb + slots - 1) / slots;
        const double eff = (double)n2 / ((double)((n2 + chunk - 1) / chunk) * (chunk + 2)) * (double)nb /
                           ((double)waves * slots);
        if (eff > best_eff + 1e-9) {
            best_eff = eff;
            best = chunk;
        }
    }
    return best;
}

// ------------------------------------------------------------------------------------
// Shrink + synthesis f = H(W^T T_mu alpha) of the public entry point.
//
// A warp covers 32 consecutive positions of one row along axis 0 (the 30 positions of the
// tile plus one halo position on either side); a block stacks SY_ROWS + 2 such warps along
// axis 1 (its SY_ROWS rows plus one halo row on either side) and marches along axis 2.
// Every lane reads the 27 coefficients of its own position (coalesced 128-byte rows per
// channel), the next plane's while the current one is computed, and shrinks them in
// registers (Eq. (2)). The separable synthesis then splits each 3-tap sum into what a
// position gives its neighbours: along axis 1 of the filter triple (a_0, a_1, a_2) at
// position p, p + 1 receives a_0/4 + (sqrt(2)/4) a_1 - a_2/4, p itself (a_0 + a_2)/2 and
// p - 1 a_0/4 - (sqrt(2)/4) a_1 - a_2/4. Axis 0 passes those shares between lanes with
// two shuffles per channel group, axis 1 between warps through shared memory (one
// barrier per plane, double buffered), and axis 2 between planes in registers.
// HBM traffic: 27 coefficients read and one value written per voxel; the halo positions
// (32/30 along axis 0, (SY_ROWS + 2)/SY_ROWS along axis 1) are re-read from L2.
// ------------------------------------------------------------------------------------
#ifndef CBCT_SY_ROWS
#define CBCT_SY_ROWS 8
#endif
constexpr int SY_ROWS = CBCT_SY_ROWS;
constexpr int SY_OUT = 30;                       // output positions per warp along axis 0
constexpr int SY_WARPS = SY_ROWS + 2;
constexpr int SY_THREADS = 32 * SY_WARPS;

__device__ __forceinline__ float raw_to_float(float v) { return v; }
__device__ __forceinline__ float raw_to_float(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float raw_to_float(__half v) { return __half2float(v); }

// shares of a filter triple (a0, a1, a2): to p + 1, to p, to p - 1
__device__ __forceinline__ void syn_shares(float a0, float a1, float a2, float &up, float &mid, float &dn)
{
    const float q = 0.25f * (a0 - a2);
    up = fmaf(R2_4, a1, q);
    dn = fmaf(-R2_4, a1, q);
    mid = 0.5f * (a0 + a2);
}

template <typename TA_T>
__global__ void __launch_bounds__(SY_THREADS, SY_THREADS <= 320 ? 2 : 1)
k_tf_synth_shrink(int n0, int n1, int n2, int chunk, const TA_T *__restrict__ alpha, float mu,
                  int positivity, float *__restrict__ f)
{
    __shared__ float s_up[2][SY_WARPS][3][32], s_dn[2][SY_WARPS][3][32];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int a_out = blockIdx.x * SY_OUT;           // first output position along axis 0
    const int b_out = blockIdx.y * SY_ROWS;          // first output row along axis 1
    const int c_begin = blockIdx.z * chunk;
    const int c_end = min(n2, c_begin + chunk);
    if (c_begin >= c_end) return;
    const size_t N = (size_t)n0 * n1 * n2;
    const size_t plane = (size_t)n0 * n1;
    const int pa = a_out + lane - 1, pb = b_out + w - 1; // this lane's position (unwrapped)
    const size_t inplane = (size_t)wrapi(pb, n1) * n0 + wrapi(pa, n0);
    const bool out_lane = lane >= 1 && lane <= SY_OUT && pa < n0;
    const bool out_row = w >= 1 && w <= SY_ROWS && pb < n1;

    TA_T nxt[27];
    auto fetch = [&](int c) {
        const TA_T *src = alpha + (size_t)wrapi(c, n2) * plane + inplane;
#pragma unroll
        for (int ch = 0; ch < 27; ++ch) nxt[ch] = src[(size_t)ch * N];
    };
    fetch(c_begin - 1);
    float w_m2[3] = {0.f, 0.f, 0.f}, w_m1[3] = {0.f, 0.f, 0.f}; // axis-2 inputs at planes cp-2, cp-1
    int buf = 0;
    for (int cp = c_begin - 1; cp <= c_end; ++cp, buf ^= 1) {
        float a[27];
#pragma unroll
        for (int ch = 0; ch < 27; ++ch) a[ch] = raw_to_float(nxt[ch]);
        if (cp < c_end) fetch(cp + 1);
        // vector shrinkage, Eq. (2)
        float s2 = 0.0f;
#pragma unroll
        for (int ch = 1; ch < 27; ++ch) s2 = fmaf(a[ch], a[ch], s2);
        const float nrm = sqrtf(s2);
        const float scale = nrm > mu ? 1.0f - mu / nrm : 0.0f;
#pragma unroll
        for (int ch = 1; ch < 27; ++ch) a[ch] *= scale;
        // axis 0 (lanes): u[m + 3n] = sum over l and the lane's neighbours
        float u[9];
#pragma unroll
        for (int mn = 0; mn < 9; ++mn) {
            float up, mid, dn;
            syn_shares(a[3 * mn], a[3 * mn + 1], a[3 * mn + 2], up, mid, dn);
            u[mn] = __shfl_up_sync(0xffffffffu, up, 1) + mid + __shfl_down_sync(0xffffffffu, dn, 1);
        }
        // axis 1 (warps): shares of rows to the rows above and below through shared memory
        float midn[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            float up, dn;
            syn_shares(u[3 * n], u[3 * n + 1], u[3 * n + 2], up, midn[n], dn);
            s_up[buf][w][n][lane] = up;
            s_dn[buf][w][n][lane] = dn;
        }
        __syncthreads();
        if (out_row) {
            float wv[3];
#pragma unroll
            for (int n = 0; n < 3; ++n) wv[n] = s_up[buf][w - 1][n][lane] + midn[n] + s_dn[buf][w + 1][n][lane];
            // axis 2 (planes): plane cp - 1 from planes cp - 2, cp - 1, cp
            if (cp >= c_begin + 1 && out_lane) {
                float o = syn3(w_m2[0], w_m1[0], wv[0], w_m2[1], wv[1], w_m2[2], w_m1[2], wv[2]);
                if (positivity && o < 0.0f) o = 0.0f;
                f[(size_t)(cp - 1) * plane + (size_t)pb * n0 + pa] = o;
            }
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                w_m2[n] = w_m1[n];
                w_m1[n] = wv[n];
            }
        }
    }
}

template <typename TA_T>
static cbct_status launch_tf_analyze_t(int n0, int n1, int n2, const float *f, TA_T *alpha, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tf_analyze<TA_T>, TF_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(e, "tf_analyze occupancy");
    const long long tiles = (long long)((n0 + TA - 1) / TA) * ((n1 + TB - 1) / TB);
    const int chunk = fused_chunk(tiles, n2, (per_sm > 0 ? per_sm : 1) * device_sm_count());
    dim3 grid((n0 + TA - 1) / TA, (n1 + TB - 1) / TB, (n2 + chunk - 1) / chunk);
    CBCT_TIMED(CBCT_KERNEL_TF_ANALYZE, st, k_tf_analyze<<<grid, dim3(TA, TB), 0, st>>>(n0, n1, n2, chunk, f, alpha));
    return check_cuda(cudaGetLastError(), "tf_analyze launch");
}

cbct_status launch_tf_analyze(int n0, int n1, int n2, const float *f, void *alpha, cudaStream_t st, int storage)
{
    if (storage == ST_BF16) return launch_tf_analyze_t(n0, n1, n2, f, static_cast<__nv_bfloat16 *>(alpha), st);
    if (storage == ST_F16) return launch_tf_analyze_t(n0, n1, n2, f, static_cast<__half *>(alpha), st);
    return launch_tf_analyze_t(n0, n1, n2, f, static_cast<float *>(alpha), st);
}

// The same step for 16-bit coefficients with two adjacent positions per lane: each
// channel is one 4-byte load of the pair, and one pair of shuffles per channel group
// serves both positions (the pair's inner shares stay in the lane). A warp covers 64
// positions: 60 outputs, the halo position on either side and one unused position at each
// end, so that every pair starts on an even position (4-byte aligned when the contiguous
// extent n0 is even, which the launcher requires; an even n0 also keeps a pair from
// straddling the periodic wrap).
constexpr int SP_OUT = 60;
// output rows per block: one block of 16 warps per SM (128 registers, 48 KB of shared
// memory) measured 0.338 ms at 512x512x70 BF16 against 0.352 ms for two blocks of 6 rows
#ifndef CBCT_SP_ROWS
#define CBCT_SP_ROWS 14
#endif
constexpr int SP_ROWS = CBCT_SP_ROWS;
constexpr int SP_WARPS = SP_ROWS + 2;
constexpr int SP_THREADS = 32 * SP_WARPS;

template <typename T16> struct Pair16;
template <> struct Pair16<__nv_bfloat16> {
    using T2 = __nv_bfloat162;
    static __device__ __forceinline__ float2 f2(T2 v) { return __bfloat1622float2(v); }
};
template <> struct Pair16<__half> {
    using T2 = __half2;
    static __device__ __forceinline__ float2 f2(T2 v) { return __half22float2(v); }
};

template <typename T16>
__global__ void __launch_bounds__(SP_THREADS, SP_THREADS <= 256 ? 2 : 1)
k_tf_synth_shrink_pair(int n0, int n1, int n2, int chunk, const T16 *__restrict__ alpha, float mu, int positivity,
                       float *__restrict__ f)
{
    using P = Pair16<T16>;
    using T2 = typename P::T2;
    __shared__ float2 s_up[2][SP_WARPS][3][32], s_dn[2][SP_WARPS][3][32];
    const int lane = threadIdx.x, w = threadIdx.y;
    const int a_out = blockIdx.x * SP_OUT, b_out = blockIdx.y * SP_ROWS;
    const int c_begin = blockIdx.z * chunk;
    const int c_end = min(n2, c_begin + chunk);
    if (c_begin >= c_end) return;
    const size_t N = (size_t)n0 * n1 * n2;
    const size_t plane = (size_t)n0 * n1;
    const int pa = a_out - 2 + 2 * lane, pb = b_out + w - 1; // the pair (pa, pa + 1), unwrapped
    const size_t inplane = (size_t)wrapi(pb, n1) * n0 + wrapi(pa, n0);
    const bool out_lane = lane >= 1 && lane <= SP_OUT / 2 && pa < n0; // n0 even: pa + 1 < n0 too
    const bool out_row = w >= 1 && w <= SP_ROWS && pb < n1;

    T2 nxt[27];
    auto fetch = [&](int c) {
        const T2 *src = reinterpret_cast<const T2 *>(alpha + (size_t)wrapi(c, n2) * plane + inplane);
        const size_t stride = N / 2; // channels in pairs (N is even)
#pragma unroll
        for (int ch = 0; ch < 27; ++ch) nxt[ch] = src[(size_t)ch * stride];
    };
    fetch(c_begin - 1);
    float2 w_m2[3], w_m1[3];
#pragma unroll
    for (int n = 0; n < 3; ++n) w_m2[n] = w_m1[n] = make_float2(0.f, 0.f);
    int buf = 0;
    for (int cp = c_begin - 1; cp <= c_end; ++cp, buf ^= 1) {
        T2 cur[27];
#pragma unroll
        for (int ch = 0; ch < 27; ++ch) cur[ch] = nxt[ch];
        if (cp < c_end) fetch(cp + 1);
        // vector shrinkage, Eq. (2), for both positions
        float2 s2 = make_float2(0.f, 0.f);
#pragma unroll
        for (int ch = 1; ch < 27; ++ch) {
            const float2 a = P::f2(cur[ch]);
            s2.x = fmaf(a.x, a.x, s2.x);
            s2.y = fmaf(a.y, a.y, s2.y);
        }
        const float na = sqrtf(s2.x), nb = sqrtf(s2.y);
        const float sa = na > mu ? 1.0f - mu / na : 0.0f, sb = nb > mu ? 1.0f - mu / nb : 0.0f;
        // axis 0: position A (even) takes lane - 1's B and its own B; B takes its own A and
        // lane + 1's A
        float2 u[9];
#pragma unroll
        for (int mn = 0; mn < 9; ++mn) {
            float2 a0 = P::f2(cur[3 * mn]), a1 = P::f2(cur[3 * mn + 1]), a2 = P::f2(cur[3 * mn + 2]);
            if (mn) {
                a0.x *= sa;
                a0.y *= sb;
            }
            a1.x *= sa;
            a1.y *= sb;
            a2.x *= sa;
            a2.y *= sb;
            float upA, midA, dnA, upB, midB, dnB;
            syn_shares(a0.x, a1.x, a2.x, upA, midA, dnA);
            syn_shares(a0.y, a1.y, a2.y, upB, midB, dnB);
            u[mn].x = __shfl_up_sync(0xffffffffu, upB, 1) + midA + dnB;
            u[mn].y = upA + midB + __shfl_down_sync(0xffffffffu, dnA, 1);
        }
        // axis 1 (warps) through shared memory
        float2 midn[3];
#pragma unroll
        for (int n = 0; n < 3; ++n) {
            float2 up, dn;
            syn_shares(u[3 * n].x, u[3 * n + 1].x, u[3 * n + 2].x, up.x, midn[n].x, dn.x);
            syn_shares(u[3 * n].y, u[3 * n + 1].y, u[3 * n + 2].y, up.y, midn[n].y, dn.y);
            s_up[buf][w][n][lane] = up;
            s_dn[buf][w][n][lane] = dn;
        }
        __syncthreads();
        if (out_row) {
            float2 wv[3];
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                const float2 a = s_up[buf][w - 1][n][lane], b = s_dn[buf][w + 1][n][lane];
                wv[n] = make_float2(a.x + midn[n].x + b.x, a.y + midn[n].y + b.y);
            }
            if (cp >= c_begin + 1 && out_lane) {
                float2 o;
                o.x = syn3(w_m2[0].x, w_m1[0].x, wv[0].x, w_m2[1].x, wv[1].x, w_m2[2].x, w_m1[2].x, wv[2].x);
                o.y = syn3(w_m2[0].y, w_m1[0].y, wv[0].y, w_m2[1].y, wv[1].y, w_m2[2].y, w_m1[2].y, wv[2].y);
                if (positivity) {
                    o.x = o.x < 0.0f ? 0.0f : o.x;
                    o.y = o.y < 0.0f ? 0.0f : o.y;
                }
                *reinterpret_cast<float2 *>(f + (size_t)(cp - 1) * plane + (size_t)pb * n0 + pa) = o;
            }
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                w_m2[n] = w_m1[n];
                w_m1[n] = wv[n];
            }
        }
    }
}

template <typename T16>
static cbct_status launch_tf_synth_shrink_pair(int n0, int n1, int n2, const T16 *alpha, float mu, int positivity,
                                               float *f, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tf_synth_shrink_pair<T16>, SP_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(e, "tf_synth_shrink occupancy");
    const long long tiles = (long long)((n0 + SP_OUT - 1) / SP_OUT) * ((n1 + SP_ROWS - 1) / SP_ROWS);
    const int chunk = fused_chunk(tiles, n2, (per_sm > 0 ? per_sm : 1) * device_sm_count());
    dim3 grid((n0 + SP_OUT - 1) / SP_OUT, (n1 + SP_ROWS - 1) / SP_ROWS, (n2 + chunk - 1) / chunk);
    CBCT_TIMED(CBCT_KERNEL_TF_SYNTH, st,
               k_tf_synth_shrink_pair<T16><<<grid, dim3(32, SP_WARPS), 0, st>>>(n0, n1, n2, chunk, alpha, mu, positivity,
                                                                                f));
    return check_cuda(cudaGetLastError(), "tf_synth_shrink launch");
}

template <typename TA_T>
static cbct_status launch_tf_synth_shrink_t(int n0, int n1, int n2, const TA_T *alpha, float mu, int positivity,
                                            float *f, cudaStream_t st)
{
    // 16-bit coefficients of an even contiguous extent: two positions per lane (aligned pairs;
    // the array's base is at least 4-byte aligned, as for any 16-bit tensor the API accepts)
    if constexpr (sizeof(TA_T) == 2)
        if (n0 % 2 == 0 && (reinterpret_cast<uintptr_t>(alpha) & 3) == 0 && (reinterpret_cast<uintptr_t>(f) & 7) == 0)
            return launch_tf_synth_shrink_pair(n0, n1, n2, alpha, mu, positivity, f, st);
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tf_synth_shrink<TA_T>, SY_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(e, "tf_synth_shrink occupancy");
    const long long tiles = (long long)((n0 + SY_OUT - 1) / SY_OUT) * ((n1 + SY_ROWS - 1) / SY_ROWS);
    const int chunk = fused_chunk(tiles, n2, (per_sm > 0 ? per_sm : 1) * device_sm_count());
    dim3 grid((n0 + SY_OUT - 1) / SY_OUT, (n1 + SY_ROWS - 1) / SY_ROWS, (n2 + chunk - 1) / chunk);
    CBCT_TIMED(CBCT_KERNEL_TF_SYNTH, st,
               k_tf_synth_shrink<TA_T><<<grid, dim3(32, SY_WARPS), 0, st>>>(n0, n1, n2, chunk, alpha, mu, positivity, f));
    return check_cuda(cudaGetLastError(), "tf_synth_shrink launch");
}

cbct_status launch_tf_synth_shrink(int n0, int n1, int n2, const void *alpha, float mu,
                                   int positivity, float *f, cudaStream_t st, int storage)
{
    if (storage == ST_BF16)
        return launch_tf_synth_shrink_t(n0, n1, n2, static_cast<const __nv_bfloat16 *>(alpha), mu, positivity, f, st);
    if (storage == ST_F16)
        return launch_tf_synth_shrink_t(n0, n1, n2, static_cast<const __half *>(alpha), mu, positivity, f, st);
    return launch_tf_synth_shrink_t(n0, n1, n2, static_cast<const float *>(alpha), mu, positivity, f, st);
}

} // namespace cbct

namespace cbct {

// ------------------------------------------------------------------------------------
// Fused shrinkage step of Algorithm A2 (steps 3-4, then step 1 of the next iteration):
//   f_new = H(W^T T_mu W x)   and optionally   v = f_new + c (f_new - f_old).
// The 27 coefficients never leave the SM: HBM traffic is one read of x (halo re-reads hit
// L2) and the writes of f_new (and v, with one read of f_old).
//
// A warp covers 32 consecutive positions of one row along axis 0: the 28 output positions
// of its tile and two halo positions on either side (the coefficients of the outputs'
// neighbours need x one position further out). A block stacks FR_ROWS + 4 such warps along
// axis 1 (its output rows, the two rows of coefficients around them and the two rows of x
// those need) and marches along axis 2. Per plane every lane
//   1. analyses along axis 2 from the three x planes it holds in registers (the next plane
//      is loaded while this one is computed),
//   2. along axis 1 from its neighbour rows' values through shared memory,
//   3. along axis 0 from its neighbour lanes by shuffles, giving its position's 27
//      coefficients, which it shrinks in registers (Eq. (2)),
// and then synthesises back as the shrink + synthesis kernel does: shares of neighbouring
// lanes by shuffles, of neighbouring rows through shared memory, of neighbouring planes in
// registers, finishing the output plane one behind the analysed one.
// ------------------------------------------------------------------------------------
// Output rows per block along axis 1. Each block recomputes the coefficients of two halo
// rows, so taller blocks waste less; one block of 22 warps per SM (80 registers, 47.6 KB of
// shared memory) measured 0.418 ms on the iteration's 512x512x70 grid against 0.471 ms for two
// blocks of 6 rows (10 warps each).
#ifndef CBCT_FR_ROWS
#define CBCT_FR_ROWS 18
#endif
constexpr int FR_ROWS = CBCT_FR_ROWS;
constexpr int FR_OUT = 28;                       // output positions per warp along axis 0
constexpr int FR_WARPS = FR_ROWS + 4;
constexpr int FR_THREADS = 32 * FR_WARPS;

__global__ void __launch_bounds__(FR_THREADS, FR_THREADS <= 320 ? 2 : 1)
k_tf_shrink_fused(int n0, int n1, int n2, int chunk, const float *__restrict__ x, float mu, int positivity,
                  float *__restrict__ fnew, const float *__restrict__ fold, float coef, float *__restrict__ vout)
{
    __shared__ float s_t[2][FR_WARPS][3][32];              // axis-2 analysis of each row
    __shared__ float s_up[2][FR_ROWS + 2][3][32], s_dn[2][FR_ROWS + 2][3][32]; // axis-1 synthesis shares
    const int lane = threadIdx.x, w = threadIdx.y;
    const int a_out = blockIdx.x * FR_OUT, b_out = blockIdx.y * FR_ROWS;
    const int c_begin = blockIdx.z * chunk;
    const int c_end = min(n2, c_begin + chunk);
    if (c_begin >= c_end) return;
    const size_t plane = (size_t)n0 * n1;
    const int pa = a_out + lane - 2, pb = b_out + w - 2;  // this lane's position (unwrapped)
    const size_t inplane = (size_t)wrapi(pb, n1) * n0 + wrapi(pa, n0);
    const bool coef_row = w >= 1 && w <= FR_ROWS + 2;     // rows whose coefficients are formed
    const bool out_row = w >= 2 && w <= FR_ROWS + 1 && pb < n1;
    const bool out_lane = lane >= 2 && lane < 2 + FR_OUT && pa < n0;
    const float *src = x + inplane;

    // x of this position at planes cp - 1, cp, cp + 1 (cp: the analysed plane)
    float xm = __ldg(src + (size_t)wrapi(c_begin - 2, n2) * plane);
    float x0 = __ldg(src + (size_t)wrapi(c_begin - 1, n2) * plane);
    float xp = __ldg(src + (size_t)wrapi(c_begin, n2) * plane);
    float w_m2[3] = {0.f, 0.f, 0.f}, w_m1[3] = {0.f, 0.f, 0.f}; // axis-2 synthesis inputs at cp-2, cp-1
    int buf = 0;
    for (int cp = c_begin - 1; cp <= c_end; ++cp, buf ^= 1) {
        const float xn = cp < c_end ? __ldg(src + (size_t)wrapi(cp + 2, n2) * plane) : 0.0f;
        // 1. analysis along axis 2
        float t[3];
        ana3(xm, x0, xp, t[0], t[1], t[2]);
#pragma unroll
        for (int n = 0; n < 3; ++n) s_t[buf][w][n][lane] = t[n];
        __syncthreads();
        float midn[3] = {0.f, 0.f, 0.f};
        if (coef_row) { // warp-uniform
            // 2. along axis 1: u[m][n]
            float u[3][3];
#pragma unroll
            for (int n = 0; n < 3; ++n)
                ana3(s_t[buf][w - 1][n][lane], t[n], s_t[buf][w + 1][n][lane], u[0][n], u[1][n], u[2][n]);
            // 3. along axis 0: alpha[l + 3m + 9n]
            float al[27];
#pragma unroll
            for (int m = 0; m < 3; ++m)
#pragma unroll
                for (int n = 0; n < 3; ++n) {
                    const float pv = __shfl_up_sync(0xffffffffu, u[m][n], 1);
                    const float nv = __shfl_down_sync(0xffffffffu, u[m][n], 1);
                    ana3(pv, u[m][n], nv, al[3 * m + 9 * n], al[1 + 3 * m + 9 * n], al[2 + 3 * m + 9 * n]);
                }
            // vector shrinkage, Eq. (2)
            float s2 = 0.0f;
#pragma unroll
            for (int ch = 1; ch < 27; ++ch) s2 = fmaf(al[ch], al[ch], s2);
            const float nrm = sqrtf(s2);
            const float scale = nrm > mu ? 1.0f - mu / nrm : 0.0f;
#pragma unroll
            for (int ch = 1; ch < 27; ++ch) al[ch] *= scale;
            // synthesis along axis 0 (lanes), then the shares along axis 1
            float us[9];
#pragma unroll
            for (int mn = 0; mn < 9; ++mn) {
                float up, mid, dn;
                syn_shares(al[3 * mn], al[3 * mn + 1], al[3 * mn + 2], up, mid, dn);
                us[mn] = __shfl_up_sync(0xffffffffu, up, 1) + mid + __shfl_down_sync(0xffffffffu, dn, 1);
            }
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                float up, dn;
                syn_shares(us[3 * n], us[3 * n + 1], us[3 * n + 2], up, midn[n], dn);
                s_up[buf][w - 1][n][lane] = up;
                s_dn[buf][w - 1][n][lane] = dn;
            }
        }
        __syncthreads();
        if (out_row) {
            float wv[3];
#pragma unroll
            for (int n = 0; n < 3; ++n) wv[n] = s_up[buf][w - 2][n][lane] + midn[n] + s_dn[buf][w][n][lane];
            // synthesis along axis 2: plane cp - 1 from planes cp - 2, cp - 1, cp
            if (cp >= c_begin + 1 && out_lane) {
                float o = syn3(w_m2[0], w_m1[0], wv[0], w_m2[1], wv[1], w_m2[2], w_m1[2], wv[2]);
                if (positivity && o < 0.0f) o = 0.0f;
                const size_t idx = (size_t)(cp - 1) * plane + (size_t)pb * n0 + pa;
                fnew[idx] = o;
                if (vout) vout[idx] = fmaf(coef, o - __ldg(fold + idx), o);
            }
#pragma unroll
            for (int n = 0; n < 3; ++n) {
                w_m2[n] = w_m1[n];
                w_m1[n] = wv[n];
            }
        }
        xm = x0;
        x0 = xp;
        xp = xn;
    }
}

cbct_status tf_prepare() { return CBCT_OK; }

cbct_status launch_tf_shrink_fused(int n0, int n1, int n2, const float *x, float mu, int positivity, float *fnew,
                                   const float *fold, float coef, float *vout, cudaStream_t st)
{
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tf_shrink_fused, FR_THREADS, 0);
    if (e != cudaSuccess) return check_cuda(e, "tf_shrink_fused occupancy");
    const long long tiles = (long long)((n0 + FR_OUT - 1) / FR_OUT) * ((n1 + FR_ROWS - 1) / FR_ROWS);
    const int chunk = fused_chunk(tiles, n2, (per_sm > 0 ? per_sm : 1) * device_sm_count());
    dim3 grid((n0 + FR_OUT - 1) / FR_OUT, (n1 + FR_ROWS - 1) / FR_ROWS, (n2 + chunk - 1) / chunk);
    CBCT_TIMED(CBCT_KERNEL_TF_SYNTH, st,
               k_tf_shrink_fused<<<grid, dim3(32, FR_WARPS), 0, st>>>(n0, n1, n2, chunk, x, mu, positivity, fnew, fold,
                                                                      coef, vout));
    return check_cuda(cudaGetLastError(), "tf_shrink_fused launch");
}

} // namespace cbct
