// Forward projector P (Eq. (1), Section 2.2.1: one ray per imager pixel, Siddon's exact
// ray tracing, g_i = sum_j a_ij f_j with a_ij the length of ray i inside voxel j).
//
// GB300 mapping. All rays of one view that hit the same imager column u share their
// transverse path through the (x, y) voxel columns; the imager row v only tilts them in
// z. A block owns one (view, column) pair and its threads own the imager rows. The
// block first computes the shared transverse Siddon trace once, cooperatively, into
// shared memory (a parallel merge of the x-plane and y-plane crossing lists). Along that
// trace a ray of row v stays in one z slab for long runs of columns (the cone is narrow),
// and the block holds more rows than the volume has slabs. So, group by group of
// columns, the block stages the columns' z-lines (contiguous in the iteration's
// z-fastest layout) and forms per slab the running sum of voxel value x segment length;
// a row's line integral over a run of columns in one slab is then the difference of two
// table entries, and only the columns where it crosses a z plane are split explicitly.
// Accumulation is FP32; the epilogue can
// scale by |D - S|, form the CGLS residual and reduce squared norms in FP64 into one
// partial per block; the output is stored as FP32, BF16 or FP16.
//
// This header holds the kernel template; it is instantiated for each group size in the
// project_groups_*.cu units (compiled in parallel) and launched from project.cu.
#pragma once
#include <cfloat>

#include "project.cuh"

namespace cbct {

// 16-byte asynchronous global -> shared copy (L2 only); both addresses 16-byte aligned
__device__ __forceinline__ void cp_async16(float *smem_dst, const float *gsrc)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// One-shot bulk (TMA) copy of a block's trace record into shared memory, completed on an
// mbarrier that one thread initialises, arms, feeds and waits on (the others wait at the
// block barrier that follows, so no warp spins).
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// global -> shared bulk copy of `bytes` (a multiple of 16) between 16-byte-aligned addresses,
// marked evict-first in L2: each record is read once per projection, and the volume lines
// and the stack the projector and the next kernels reuse should stay
__device__ __forceinline__ void bulk_copy_g2s(void *smem_dst, const void *gsrc, unsigned bytes, unsigned long long *bar)
{
    unsigned long long policy;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(policy));
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::"r"(
            smem_u32(smem_dst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
        : "memory");
}
// tries of the record wait before a block gives up (each try may suspend the thread for a
// while; together well over a second): a copy that never lands ends the block with NaN
// results and bit 1 of the iteration's status word instead of a hang
constexpr int PROJ_WAIT_TRIES = 1 << 22;

// The transverse ray shared by every row of imager column iu in a view, and the tau
// interval in which it crosses the volume's (x, y) footprint.
struct ColumnRay {
    float dxr, dyr, qx, qy, inv_x, inv_y, tau_in, tau_out;
    int sxs, sys;
    bool hit;
};
__device__ __forceinline__ ColumnRay column_ray(const GeomDev &G, int view, int iu)
{
    ColumnRay c;
    const float2 cs = G.cs[view];
    ray_xy(G, cs.x, cs.y, imager_u(G, iu), c.dxr, c.dyr, c.qx, c.qy);
    c.inv_x = safe_rcp(c.dxr);
    c.inv_y = safe_rcp(c.dyr);
    const float xa = tau_plane(G.x0, c.qx, c.inv_x), xb = tau_plane(plane_at(G.nx, G.dx, G.x0), c.qx, c.inv_x);
    const float ya = tau_plane(G.y0, c.qy, c.inv_y), yb = tau_plane(plane_at(G.ny, G.dy, G.y0), c.qy, c.inv_y);
    c.tau_in = fmaxf(fmaxf(fminf(xa, xb), fminf(ya, yb)), -G.tc);
    c.tau_out = fminf(fminf(fmaxf(xa, xb), fmaxf(ya, yb)), 1.0f - G.tc);
    c.hit = c.tau_in < c.tau_out;
    c.sxs = c.dxr > 0.0f ? 1 : -1;
    c.sys = c.dyr > 0.0f ? 1 : -1;
    return c;
}

// Phase 1 of a column (whole block, one barrier inside): the crossings of the ray with
// each plane family are increasing in tau, so every crossing's position in the merged order
// is its own index plus the number of crossings of the other family before it. Writes, for
// the nseg = nA + nB + 1 segments the ray spends in (x, y) voxel columns, sEnd[j] (the tau at
// which segment j ends) and sCol[j] (its column's offset ix * sx + iy * sy); sA (nx + 1
// floats), sB (ny + 1) and s_cnt (4 per warp) are scratch. Returns (nA, nB, ix_e, iy_e): the
// x- and y-plane crossings inside the volume and the column entered first.
__device__ __forceinline__ int4 trace_column(const GeomDev &G, const ColumnRay &ray, int sx, int sy, float *sA,
                                             float *sB, unsigned *s_cnt, float *sEnd, int *sCol, int tid, int nthr)
{
    const float dxr = ray.dxr, dyr = ray.dyr, qx = ray.qx, qy = ray.qy, inv_x = ray.inv_x, inv_y = ray.inv_y;
    const float tau_in = ray.tau_in, tau_out = ray.tau_out;
    const bool hit = ray.hit;
    const int sxs = ray.sxs, sys = ray.sys;
    // counts of the crossings before the entry point and inside the volume: per thread, then
    // one block-wide sum (the lists are written before the barrier of that sum)
    unsigned cnt4[4] = {0u, 0u, 0u, 0u}; // a_le, a_in, b_le, b_in
    for (int a = tid; a <= G.nx; a += nthr) {
        if (hit && dxr != 0.0f) {
            const float t = tau_plane(plane_at(dxr > 0.0f ? a : G.nx - a, G.dx, G.x0), qx, inv_x);
            sA[a] = t;
            cnt4[0] += t <= tau_in;
            cnt4[1] += t > tau_in && t < tau_out;
        }
    }
    for (int b = tid; b <= G.ny; b += nthr) {
        if (hit && dyr != 0.0f) {
            const float t = tau_plane(plane_at(dyr > 0.0f ? b : G.ny - b, G.dy, G.y0), qy, inv_y);
            sB[b] = t;
            cnt4[2] += t <= tau_in;
            cnt4[3] += t > tau_in && t < tau_out;
        }
    }
    // per-warp sums
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const unsigned v = __reduce_add_sync(0xffffffffu, cnt4[q]);
        if ((tid & 31) == 0) s_cnt[4 * (tid >> 5) + q] = v;
    }
    __syncthreads();
    int a_le = 0, a_in = 0, b_le = 0, b_in = 0;
    for (int wq = 0; wq < (nthr + 31) / 32; ++wq) {
        a_le += (int)s_cnt[4 * wq + 0];
        a_in += (int)s_cnt[4 * wq + 1];
        b_le += (int)s_cnt[4 * wq + 2];
        b_in += (int)s_cnt[4 * wq + 3];
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
    // The rank of a crossing in the other family's list: the planes of that family the ray has
    // passed at t, estimated from its transverse position and then moved to the exact count
    // (# LB[j] < t for an x crossing, # LA[i] <= t for a y crossing), which the lists decide.
    auto passed = [&](float pos, float o, float inv_h, int n, int sgn, int le) {
        const int k = (int)floorf((pos - o) * inv_h); // the plane at or below pos
        return sgn > 0 ? k + 1 - le : n - k - le;
    };
    const float inv_dx = 1.0f / G.dx, inv_dy = 1.0f / G.dy;
    for (int i = tid; i < nA; i += nthr) {
        const float t = LA[i];
        int nb = 0;
        if (nB) {
            nb = min(max(passed(fmaf(t, dyr, qy), G.y0, inv_dy, G.ny, sys, b_le), 0), nB);
            while (nb > 0 && !(LB[nb - 1] < t)) --nb;
            while (nb < nB && LB[nb] < t) ++nb;
        }
        const int r = i + nb;
        const int cx = min(max(ix_e + sxs * (i + 1), 0), G.nx - 1), cy = min(max(iy_e + sys * nb, 0), G.ny - 1);
        sEnd[r] = t;
        sCol[r + 1] = cx * sx + cy * sy;
    }
    for (int j = tid; j < nB; j += nthr) {
        const float t = LB[j];
        int na = 0;
        if (nA) {
            na = min(max(passed(fmaf(t, dxr, qx), G.x0, inv_dx, G.nx, sxs, a_le), 0), nA);
            while (na > 0 && LA[na - 1] > t) --na;
            while (na < nA && LA[na] <= t) ++na;
        }
        const int r = j + na;
        const int cx = min(max(ix_e + sxs * na, 0), G.nx - 1), cy = min(max(iy_e + sys * (j + 1), 0), G.ny - 1);
        sEnd[r] = t;
        sCol[r + 1] = cx * sx + cy * sy;
    }
    if (tid == 0) {
        sCol[0] = ix_e * sx + iy_e * sy;
        sEnd[nseg - 1] = tau_out;
    }
    return make_int4(nA, nB, ix_e, iy_e);
}


// One block per (view, imager column, chunk of rows), volume z-contiguous (sz = 1).
// Phase 1 (whole block): the transverse Siddon trace of the column's rays — the
// crossings with the x planes and with the y planes are each increasing in tau, so every
// crossing's position in the merged order is its own index plus the number of crossings
// of the other family before it (binary search); this yields the list of (x, y) voxel
// columns the rays visit and the tau at which each is left. For every segment the block
// also stores its length and where its column's z-line will sit in shared memory.
// Phase 2, per group of SG segments: the block stages the group's z-lines and builds
// the per-slab prefix table T[k][u] over the group's columns; then each thread (two
// imager rows) adds, for each run of whole columns a row spends in one z slab, the
// table difference, and splits exactly each column in which the row crosses a z plane.
template <int MODE, typename TP, int SG>
__global__ void __launch_bounds__(PROJ_THREADS, CBCT_PROJ_MIN_BLOCKS)
k_project(GeomDev G, const float *__restrict__ f, int sx, int sy, const float *__restrict__ y,
          TP *__restrict__ out, double *__restrict__ partials, float count_thr, Scalars *__restrict__ sc,
          const int4 *__restrict__ traces, int trace_cap)
{
    extern __shared__ __align__(16) float smem[];
    __shared__ double s_warp[PROJ_THREADS / 32];
    __shared__ __align__(8) unsigned long long s_bar; // completion of the trace record's copy
    const int cap = ((G.nx + G.ny + 2 + SG - 1) / SG) * SG;
    float *sEnd = smem;                                    // tau at which segment j ends
    int *sCol = reinterpret_cast<int *>(sEnd + cap);      // voxel-column offset of segment j
    float2 *sSeg = reinterpret_cast<float2 *>(sCol + cap); // (line offset bits, length) of segment j
    const int pitch = ((G.nz + 6 + 3) / 4) * 4;            // floats per staged line
    const int quads = pitch / 4;                           // 16-byte pieces per line slot
    float *sLine = reinterpret_cast<float *>(sSeg + cap);  // the staged z-lines of one group
    float *sA = sLine;                                     // phase 1: x-plane crossings, in ray order
    float *sB = sA + (G.nx + 1);                           // phase 1: y-plane crossings
    const int lregion = max(SG * pitch, ((G.nx + G.ny + 2 + 3) / 4) * 4);
    constexpr int TPITCH = SG + 1;                         // odd: the build's threads (slabs) hit distinct banks
    float *sTab = sLine + lregion;                         // [nz][SG + 1] per-slab prefix table
    float *sBase = sTab + G.nz * TPITCH;                   // [2][nz] running per-slab totals

    const int tid = threadIdx.x, nthr = blockDim.x;
    const int view = blockIdx.x / G.nu;
    const int iu = blockIdx.x - view * G.nu;

    // ---- transverse ray, shared by every row ----
    const ColumnRay ray = column_ray(G, view, iu);
    const float dxr = ray.dxr, dyr = ray.dyr, qx = ray.qx, qy = ray.qy;
    const float tau_in = ray.tau_in, tau_out = ray.tau_out;
    const bool hit = ray.hit;
    const int sxs = ray.sxs, sys = ray.sys;

    // ---- phase 1: crossings of each plane family, then their merged order ----
    int4 tr;
    bool timed_out = false;
    if (traces && hit) {
        // phase 1 from the grid's trace table: the record's segment lists by one bulk copy
        const int4 *rec = traces + (size_t)blockIdx.x * (1 + trace_cap / 2);
        tr = __ldg(rec);
        int bad = 0;
        if (tid == 0) {
            const unsigned bytes = 4u * (unsigned)((tr.x + tr.y + 1 + 3) & ~3);
            mbar_init(&s_bar, 1u);
            mbar_arrive_expect_tx(&s_bar, 2u * bytes);
            bulk_copy_g2s(sEnd, rec + 1, bytes, &s_bar);
            bulk_copy_g2s(sCol, reinterpret_cast<const float *>(rec + 1) + trace_cap, bytes, &s_bar);
            bool landed = false;
            for (int it = 0; it < PROJ_WAIT_TRIES && !(landed = mbar_try_wait(&s_bar, 0u)); ++it) {
            }
            bad = !landed;
        }
        timed_out = __syncthreads_or(bad) != 0;
        if (timed_out && sc && tid == 0) atomicOr(&sc->flags, 2u);
    } else {
        // per-warp sums of phase 1 are parked in the segment records (written after it)
        tr = trace_column(G, ray, sx, sy, sA, sB, reinterpret_cast<unsigned *>(sSeg), sEnd, sCol, tid, nthr);
    }
    const int nA = tr.x, nB = tr.y, ix_e = tr.z, iy_e = tr.w, nseg = nA + nB + 1;
    const int col0 = ix_e * sx + iy_e * sy;
    const float inv_dx = 1.0f / G.dx, inv_dy = 1.0f / G.dy;
    for (int q = nseg + tid; q < cap; q += nthr) { // zero-length padding up to whole groups
        sEnd[q] = tau_out;
        sCol[q] = col0;
    }
    __syncthreads();
    for (int q = tid; q < cap; q += nthr) {
        const float st = q ? sEnd[q - 1] : tau_in;
        // where the column's first voxel lands in its staged line
        const int loff = (q % SG) * pitch + (sCol[q] & 3);
        sSeg[q] = make_float2(__int_as_float(loff), sEnd[q] - st);
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
        active[r] = hit && !timed_out && ok[r] && kz[r] >= 0 && kz[r] < G.nz;
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
    } else if (hit && !timed_out) {
        // Per group of SG segments: stage the z-lines of its columns (16-byte cp.async into
        // one buffer: a second buffer to copy the next group ahead would cost a resident
        // block, which hides more latency than the early copy), build once for the block the
        // per-slab prefix table over the group's columns,
        //     T[k][u] = sum_{u' < u} f(column u', slab k) * length(u'),   u = 0..SG,
        // and let every row add T[k][u1] - T[k][u0] for each run of whole columns it
        // spends in slab k. Only the columns in which a row crosses a z plane are split,
        // exactly, at the crossing. A block has far more rows than slabs, so the table
        // does the per-column work once per slab instead of once per row.
        const int nchunk = (nseg + SG - 1) / SG;
        // 16-byte pieces of a group's lines: slot c = (line u, piece i), c = u * quads + i;
        // thread tid takes c = tid, tid + nthr, ... (the same slots for every group)
        const int u_0 = tid / quads, i_0 = tid - u_0 * quads;
        const int du = nthr / quads, di = nthr - du * quads;
        auto fill = [&](int chunk) {
            float *dst = sLine;
            const int *col = sCol + chunk * SG;
            for (int u = u_0, i = i_0; u < SG;) {
                const int c0 = col[u];
                const int first = c0 & ~3, last = (c0 + G.nz + 3) & ~3; // 16-byte rounded line
                if (first + 4 * i < last) cp_async16(dst + u * pitch + 4 * i, f + first + 4 * i);
                u += du;
                i += di;
                if (i >= quads) {
                    i -= quads;
                    ++u;
                }
            }
            cp_async_commit();
        };
        const bool split = nthr >= 2 * G.nz;
        // T[k][u]: the table entry, plus the first half's total for a second-half entry
        auto tab = [&](int k, int u) {
            const float *trow = sTab + k * TPITCH;
            return split && u > SG / 2 ? trow[u] + trow[SG / 2] : trow[u];
        };
        float E[R] = {0.0f, 0.0f}; // running total where each row's current run starts
        for (int k = tid; k < G.nz; k += nthr) sBase[k] = 0.0f; // published by the first barrier
        float g0 = tau_in;
        for (int ch = 0; ch < nchunk; ++ch) {
            const int j = ch * SG;
            if (ch) __syncthreads(); // every thread is done with the previous group's lines
            fill(ch);
            cp_async_wait<0>();
            __syncthreads();
            const float *lines = sLine;
            // The group's prefix table. With threads to spare each slab's running sum is
            // split into two chains of SG / 2 columns computed side by side; the second
            // half's entries then hold sums from column SG / 2 on, and tab() adds the
            // first half's total.
            if (split) {
                for (int task = tid; task < 2 * G.nz; task += nthr) {
                    const int k = task >> 1, h = (task & 1) * (SG / 2);
                    float *trow = sTab + k * TPITCH + h;
                    float sum = 0.0f;
                    if (!h) trow[0] = 0.0f;
#pragma unroll 8
                    for (int u = 0; u < SG / 2; ++u) {
                        const float2 seg = sSeg[j + h + u]; // (line offset, length)
                        sum = fmaf(lines[__float_as_int(seg.x) + k], seg.y, sum);
                        trow[u + 1] = sum;
                    }
                }
            } else {
                for (int k = tid; k < G.nz; k += nthr) {
                    float *trow = sTab + k * TPITCH;
                    float sum = 0.0f;
                    trow[0] = 0.0f;
#pragma unroll 8
                    for (int u = 0; u < SG; ++u) {
                        const float2 seg = sSeg[j + u];
                        sum = fmaf(lines[__float_as_int(seg.x) + k], seg.y, sum);
                        trow[u + 1] = sum;
                    }
                }
            }
            __syncthreads();
            const float gend = sEnd[j + SG - 1];
            // running per-slab totals: C[k][j + u] = base[k] + T[k][u] is the sum over all
            // columns of the trace before column j + u; one thread per slab carries it on
            const float *bcur = sBase + (ch & 1) * G.nz;
            float *bnext = sBase + ((ch + 1) & 1) * G.nz;
            for (int k = tid; k < G.nz; k += nthr) bnext[k] = bcur[k] + tab(k, SG);
            // A row does nothing in a group it crosses no z plane in. At a crossing it adds
            // its run in the slab it leaves (a difference of running totals, plus the part
            // of the crossing column before the plane) and books the rest of that column to
            // the slab it enters; E remembers the running total where that slab's run of
            // whole columns starts.
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float a = acc[r];
                int cpend = -1; // column of this row's previous crossing in this group
                while (tzn[r] < gend) { // a z crossing inside this group (the row is active)
                    const float t = tzn[r];
                    // The segment holding the crossing: the x and y planes the ray has passed
                    // at t, from its transverse position (no search). At a near tie this may
                    // name the neighbouring segment, which only moves a rounding-sized piece
                    // of length between two adjacent columns; it is kept monotone.
                    int na = (int)floorf((fmaf(t, dxr, qx) - G.x0) * inv_dx) - ix_e;
                    int nb = (int)floorf((fmaf(t, dyr, qy) - G.y0) * inv_dy) - iy_e;
                    na = min(max(sxs > 0 ? na : -na, 0), nA);
                    nb = min(max(sys > 0 ? nb : -nb, 0), nB);
                    const int c = min(max(na + nb - j, max(cpend, 0)), SG - 1);
                    const int lo = __float_as_int(sSeg[j + c].x);
                    const float en = sEnd[j + c];
                    const float fcur = lines[lo + kz[r]];
                    if (c == cpend) // entered this slab in this same column: trim the booked rest
                        a = fmaf(-fcur, en - t, a);
                    else
                        a += (bcur[kz[r]] + tab(kz[r], c)) - E[r] +
                             fcur * fmaxf(t - (c ? sEnd[j + c - 1] : g0), 0.0f);
                    cpend = c;
                    kz[r] += skz[r];
                    active[r] = (unsigned)kz[r] < (unsigned)G.nz;
                    if (active[r]) {
                        a = fmaf(lines[lo + kz[r]], en - t, a);
                        E[r] = bcur[kz[r]] + tab(kz[r], c + 1);
                    }
                    tzn[r] = active[r] ? tau_zplane(plane_at(kz[r] + (skz[r] > 0), G.dz, G.z0), inv_v[r], G.tc) : P_INF;
                }
                acc[r] = a;
            }
            g0 = gend;
        }
        __syncthreads();
        // the run each still-active row ends in: up to the end of the trace
        const float *bend = sBase + (nchunk & 1) * G.nz;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (active[r]) acc[r] += bend[kz[r]] - E[r];
    }

    // ---- epilogue ----
    if (timed_out) { // the trace record never arrived: NaN rows, reported through sc
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = __int_as_float(0x7fc00000);
    }
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

template <int MODE, typename TP, int SG> static const void *kernel_ptr()
{
    return reinterpret_cast<const void *>(&k_project<MODE, TP, SG>);
}

template <int SG> const void *project_kernel(int mode, int storage)
{
    if (mode == PM_COUNT) {
        if constexpr (SG == PROJECT_GROUP_SIZES[0]) return kernel_ptr<PM_COUNT, float, SG>();
        else return nullptr;
    }
    const int s = storage == ST_BF16 ? 1 : storage == ST_F16 ? 2 : 0;
    switch (mode * 3 + s) {
    case PM_PLAIN * 3 + 0: return kernel_ptr<PM_PLAIN, float, SG>();
    case PM_PLAIN * 3 + 1: return kernel_ptr<PM_PLAIN, __nv_bfloat16, SG>();
    case PM_PLAIN * 3 + 2: return kernel_ptr<PM_PLAIN, __half, SG>();
    case PM_Q_SCALED * 3 + 0: return kernel_ptr<PM_Q_SCALED, float, SG>();
    case PM_Q_SCALED * 3 + 1: return kernel_ptr<PM_Q_SCALED, __nv_bfloat16, SG>();
    case PM_Q_SCALED * 3 + 2: return kernel_ptr<PM_Q_SCALED, __half, SG>();
    case PM_RESID * 3 + 0: return kernel_ptr<PM_RESID, float, SG>();
    case PM_RESID * 3 + 1: return kernel_ptr<PM_RESID, __nv_bfloat16, SG>();
    case PM_RESID * 3 + 2: return kernel_ptr<PM_RESID, __half, SG>();
    default: return nullptr;
    }
}

} // namespace cbct
