// The projector's trace table: phase 1 of every (view, imager column), stored so that the
// projections of a reconstruction read it instead of recomputing it (Section 2.2.1: the
// transverse part of every ray of an imager column is the same Siddon trace).
#include "project_kernel.cuh"

namespace cbct {

// The grid's trace table: one record per (view, imager column), written by phase 1 of that
// column (the same code as the projector's): an int4 header (nA, nB, ix_e, iy_e), then
// End[trace_cap] floats and Col[trace_cap] ints, of which the first nseg rounded up to 4 are
// written (the rounding tail with the padding values, tau_out and the first column).
// trace_cap = nx + ny + 2 rounded up to 4; the column offsets use the strides sx, sy that the
// projector will be given. The trace depends on the geometry only, so a reconstruction
// builds it once per level and every projection of that level reads it.
__global__ void __launch_bounds__(PROJ_THREADS) k_trace_table(GeomDev G, int sx, int sy, int4 *__restrict__ traces,
                                                              int trace_cap)
{
    extern __shared__ __align__(16) float smem[];
    float *sEnd = smem;
    int *sCol = reinterpret_cast<int *>(sEnd + trace_cap);
    unsigned *s_cnt = reinterpret_cast<unsigned *>(sCol + trace_cap); // 4 per warp
    float *sA = reinterpret_cast<float *>(s_cnt + 4 * (PROJ_THREADS / 32));
    float *sB = sA + (G.nx + 1);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int view = blockIdx.x / G.nu, iu = blockIdx.x - view * G.nu;
    const ColumnRay ray = column_ray(G, view, iu);
    const int4 tr = trace_column(G, ray, sx, sy, sA, sB, s_cnt, sEnd, sCol, tid, nthr);
    __syncthreads();
    const int nseg = tr.x + tr.y + 1, n4 = (nseg + 3) & ~3, col0 = tr.z * sx + tr.w * sy;
    int4 *rec = traces + (size_t)blockIdx.x * (1 + trace_cap / 2);
    float *E = reinterpret_cast<float *>(rec + 1);
    int *C = reinterpret_cast<int *>(E + trace_cap);
    // streaming stores: the table is read back once per projection, not kept in L2
    for (int q = tid; q < n4; q += nthr) {
        __stcs(E + q, q < nseg ? sEnd[q] : ray.tau_out);
        __stcs(C + q, q < nseg ? sCol[q] : col0);
    }
    if (tid == 0) __stcs(rec, tr);
}

size_t trace_table_bytes(const GeomDev &G)
{
    return (size_t)G.nviews * G.nu * (16 + 8 * (size_t)trace_cap(G));
}

static std::atomic<unsigned long long> g_trace_optin{0};

cbct_status trace_table_prepare()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "trace table device");
    const unsigned long long bit = 1ull << (dev & 63);
    if (g_trace_optin.load() & bit) return CBCT_OK;
    e = cudaFuncSetAttribute(k_trace_table, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PROJECT_SMEM_LIMIT);
    if (e != cudaSuccess) return check_cuda(e, "trace table attribute");
    g_trace_optin.fetch_or(bit);
    return CBCT_OK;
}

cbct_status launch_trace_table(const GeomDev &G, long long sx, long long sy, void *tab, cudaStream_t st)
{
    const size_t smem = trace_smem(G);
    if (smem > PROJECT_SMEM_LIMIT) return set_error(CBCT_ERR_UNSUPPORTED, "trace table: grid too large (nx + ny)");
    cbct_status r = trace_table_prepare();
    if (r != CBCT_OK) return r;
    k_trace_table<<<(unsigned)(G.nviews * G.nu), PROJ_THREADS, smem, st>>>(G, (int)sx, (int)sy,
                                                                         reinterpret_cast<int4 *>(tab), trace_cap(G));
    note_launch();
    return check_cuda(cudaGetLastError(), "trace table launch");
}

} // namespace cbct
