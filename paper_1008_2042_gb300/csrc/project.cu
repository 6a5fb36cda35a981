// Forward projector P (Eq. (1), Section 2.2.1: one ray per imager pixel, Siddon's exact
// ray tracing, g_i = sum_j a_ij f_j with a_ij the length of ray i inside voxel j).
//
// GB300 mapping. All rays of one view that hit the same imager column u share their
// transverse path through the (x, y) voxel columns; the imager row v only tilts them in
// z. A block therefore owns one (view, column) pair and its threads own consecutive
// rows: the 2-D Siddon walk over (x, y) columns is identical in every lane (warp-uniform
// control flow, no divergence), and at each column a lane reads the voxel of its own
// z slab. With the iteration's z-fastest volume layout the 32 lanes of a warp read a few
// consecutive floats of one column — one or two 32-byte sectors per load. z-plane
// crossings (about one per 40 column steps at the paper's sizes) are handled by a short
// per-lane loop. Accumulation is FP32; the epilogue can scale by |D - S|, form the
// CGLS residual and reduce squared norms in FP64 into one partial per block.
#include <cfloat>

#include "cbct_internal.cuh"

namespace cbct {

constexpr int PROJ_ROWS = 128;
constexpr float P_INF = 3.0e38f;

static inline int proj_rows(const GeomDev &G)
{
    int r = ((G.nv + 31) / 32) * 32;
    return r < PROJ_ROWS ? r : PROJ_ROWS;
}

int project_num_blocks(const GeomDev &G)
{
    int rows = proj_rows(G);
    return G.nviews * G.nu * ((G.nv + rows - 1) / rows);
}

__device__ __forceinline__ double block_sum(double v, double *s_warp)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_warp[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int w = 0; w < nw; ++w) t += s_warp[w];
    }
    return t;
}

template <int MODE>
__global__ void __launch_bounds__(PROJ_ROWS)
k_project(GeomDev G, const float *__restrict__ f, long long sx, long long sy, long long sz,
          const float *__restrict__ y, float *__restrict__ out, double *__restrict__ partials,
          float count_thr)
{
    __shared__ double s_warp[PROJ_ROWS / 32];
    const int view = blockIdx.x / G.nu;
    const int iu = blockIdx.x - view * G.nu;
    const int iv = blockIdx.y * blockDim.x + threadIdx.x;
    const bool row_ok = iv < G.nv;

    // ---- transverse ray (uniform over the block) ----
    const float2 cs = G.cs[view];
    float dxr, dyr, qx, qy;
    ray_xy(G, cs.x, cs.y, imager_u(G, iu), dxr, dyr, qx, qy);
    const float inv_x = safe_rcp(dxr), inv_y = safe_rcp(dyr);
    const float xa = tau_plane(G.x0, qx, inv_x), xb = tau_plane(plane_at(G.nx, G.dx, G.x0), qx, inv_x);
    const float ya = tau_plane(G.y0, qy, inv_y), yb = tau_plane(plane_at(G.ny, G.dy, G.y0), qy, inv_y);
    const float tau_in = fmaxf(fmaxf(fminf(xa, xb), fminf(ya, yb)), -G.tc);
    const float tau_out = fminf(fminf(fmaxf(xa, xb), fmaxf(ya, yb)), 1.0f - G.tc);

    const int sxs = dxr > 0.0f ? 1 : -1, sys = dyr > 0.0f ? 1 : -1;
    int ix = (int)floorf((fmaf(tau_in, dxr, qx) - G.x0) / G.dx);
    int iy = (int)floorf((fmaf(tau_in, dyr, qy) - G.y0) / G.dy);
    ix = min(max(ix, 0), G.nx - 1);
    iy = min(max(iy, 0), G.ny - 1);
    float txn = dxr != 0.0f ? tau_plane(plane_at(ix + (sxs > 0), G.dx, G.x0), qx, inv_x) : P_INF;
    float tyn = dyr != 0.0f ? tau_plane(plane_at(iy + (sys > 0), G.dy, G.y0), qy, inv_y) : P_INF;
    // a crossing computed at or before the entry point has already been passed
    for (int r = 0; r < 2 && txn <= tau_in; ++r) {
        ix += sxs;
        txn = tau_plane(plane_at(ix + (sxs > 0), G.dx, G.x0), qx, inv_x);
    }
    for (int r = 0; r < 2 && tyn <= tau_in; ++r) {
        iy += sys;
        tyn = tau_plane(plane_at(iy + (sys > 0), G.dy, G.y0), qy, inv_y);
    }
    const bool hit = tau_in < tau_out && (unsigned)ix < (unsigned)G.nx && (unsigned)iy < (unsigned)G.ny;

    // ---- per-lane z state ----
    const float v = imager_v(G, iv);
    const float inv_v = v != 0.0f ? __frcp_rn(v) : 1e30f;
    const int skz = v >= 0.0f ? 1 : -1;
    int kz = (int)floorf((v * (G.tc + tau_in) - G.z0) / G.dz);
    bool active = hit && row_ok && kz >= 0 && kz < G.nz;
    float tzn = active ? tau_zplane(plane_at(kz + (skz > 0), G.dz, G.z0), inv_v, G.tc) : P_INF;
    if (active && tzn <= tau_in) {
        kz += skz;
        if ((unsigned)kz >= (unsigned)G.nz) {
            active = false;
            tzn = P_INF;
        } else {
            tzn = tau_zplane(plane_at(kz + (skz > 0), G.dz, G.z0), inv_v, G.tc);
        }
    }
    const float L = ray_length(dxr, dyr, v);
    const float thr_tau = MODE == PM_COUNT ? count_thr / L : 0.0f;

    float acc = 0.0f;
    int cnt = 0;
    if (hit) {
        float tau = tau_in;
        const int max_steps = G.nx + G.ny + 2;
        for (int step = 0; step < max_steps; ++step) {
            const float tnext = fminf(fminf(txn, tyn), tau_out);
            const long long col = (long long)ix * sx + (long long)iy * sy;
            float tl = tau;
            while (tzn < tnext) { // z-plane crossing inside this column (lane-divergent, rare)
                if (MODE == PM_COUNT) cnt += (tzn - tl) > thr_tau;
                else acc = fmaf(__ldg(f + col + kz * sz), tzn - tl, acc);
                tl = tzn;
                kz += skz;
                if ((unsigned)kz >= (unsigned)G.nz) {
                    active = false;
                    tzn = P_INF;
                } else {
                    tzn = tau_zplane(plane_at(kz + (skz > 0), G.dz, G.z0), inv_v, G.tc);
                }
            }
            if (active) {
                if (MODE == PM_COUNT) cnt += (tnext - tl) > thr_tau;
                else acc = fmaf(__ldg(f + col + kz * sz), tnext - tl, acc);
            }
            if (tnext >= tau_out) break;
            tau = tnext;
            if (txn <= tyn) {
                ix += sxs;
                if ((unsigned)ix >= (unsigned)G.nx) break;
                txn = tau_plane(plane_at(ix + (sxs > 0), G.dx, G.x0), qx, inv_x);
            } else {
                iy += sys;
                if ((unsigned)iy >= (unsigned)G.ny) break;
                tyn = tau_plane(plane_at(iy + (sys > 0), G.dy, G.y0), qy, inv_y);
            }
        }
    }

    // ---- epilogue ----
    double red = 0.0;
    if (row_ok) {
        const size_t idx = ((size_t)view * G.nv + iv) * G.nu + iu;
        const float q = acc * L;
        if (MODE == PM_PLAIN) {
            out[idx] = q;
        } else if (MODE == PM_Q_PRESCALED) {
            out[idx] = q * L;
            red = (double)q * (double)q;
        } else if (MODE == PM_R_PRESCALED) {
            const float r = y[idx] - q;
            out[idx] = r * L;
            red = (double)r * (double)r;
        } else {
            red = (double)cnt;
        }
    }
    if (MODE != PM_PLAIN) {
        const double t = block_sum(red, s_warp);
        if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
    }
}

cbct_status launch_project(const GeomDev &G, const float *f, long long sx, long long sy,
                           long long sz, const float *y, float *out, int mode,
                           double *partials, float count_thr, cudaStream_t st)
{
    const int rows = proj_rows(G);
    dim3 grid((unsigned)(G.nviews * G.nu), (unsigned)((G.nv + rows - 1) / rows));
    ProfToken tok = prof_start(CBCT_KERNEL_PROJECT, st);
    switch (mode) {
    case PM_PLAIN:
        k_project<PM_PLAIN><<<grid, rows, 0, st>>>(G, f, sx, sy, sz, y, out, partials, count_thr);
        break;
    case PM_Q_PRESCALED:
        k_project<PM_Q_PRESCALED><<<grid, rows, 0, st>>>(G, f, sx, sy, sz, y, out, partials, count_thr);
        break;
    case PM_R_PRESCALED:
        k_project<PM_R_PRESCALED><<<grid, rows, 0, st>>>(G, f, sx, sy, sz, y, out, partials, count_thr);
        break;
    default:
        k_project<PM_COUNT><<<grid, rows, 0, st>>>(G, f, sx, sy, sz, y, out, partials, count_thr);
        break;
    }
    prof_stop(tok, st);
    note_launch();
    return check_cuda(cudaGetLastError(), "project launch");
}

} // namespace cbct
