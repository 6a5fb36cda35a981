// Forward projector P (Eq. (1), Section 2.2.1): host dispatcher. Chooses the column-group
// size of each launch, opts the kernel into its shared memory and launches it. The kernel
// itself is in project_kernel.cuh.
#include <atomic>
#include <cmath>
#include <map>
#include <mutex>
#include <tuple>

#include "project.cuh"

namespace cbct {

int project_num_blocks(const GeomDev &G)
{
    const int rows = 2 * proj_threads(G);
    return G.nviews * G.nu * ((G.nv + rows - 1) / rows);
}

// the smallest group needs the least shared memory: a grid is accepted when it fits
size_t project_smem_bytes(const GeomDev &G) { return project_smem(G, PROJECT_GROUP_SIZES[0]); }

static const void *kernel_for(int sg, int mode, int storage)
{
    switch (sg) {
    case 16: return project_kernel<16>(mode, storage);
    case 24: return project_kernel<24>(mode, storage);
    case 32: return project_kernel<32>(mode, storage);
    case 40: return project_kernel<40>(mode, storage);
    case 48: return project_kernel<48>(mode, storage);
    case 56: return project_kernel<56>(mode, storage);
    case 64: return project_kernel<64>(mode, storage);
    case 80: return project_kernel<80>(mode, storage);
    case 96: return project_kernel<96>(mode, storage);
    default: return nullptr;
    }
}

static int group_index(int sg)
{
    for (int i = 0; i < PROJECT_N_GROUP_SIZES; ++i)
        if (PROJECT_GROUP_SIZES[i] == sg) return i;
    return -1;
}

// per-device record of the shared-memory opt-in, one per (group size, mode, storage)
static std::atomic<unsigned long long> g_optin[PROJECT_N_GROUP_SIZES][4][3];

static cbct_status optin(int sg, int mode, int storage, const void **fn)
{
    *fn = kernel_for(sg, mode, storage);
    if (!*fn) return set_error(CBCT_ERR_UNSUPPORTED, "project: no kernel for group %d, mode %d", sg, mode);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "project device");
    std::atomic<unsigned long long> &done = g_optin[group_index(sg)][mode][storage == ST_BF16 ? 1 : storage == ST_F16 ? 2 : 0];
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return CBCT_OK;
    e = cudaFuncSetAttribute(*fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PROJECT_SMEM_LIMIT);
    if (e != cudaSuccess) return check_cuda(e, "project attribute");
    done.fetch_or(bit);
    return CBCT_OK;
}

static std::atomic<int> g_forced_group{0}; // 0: automatic

// The group size of a launch. Two effects compete (measured on GB300 over group sizes,
// register budgets and seven grids): a group pays a fixed cost (barriers, the copy loop,
// the running totals) that a larger group spreads over more columns, and a larger group
// needs more shared memory, so fewer blocks stay resident to hide each other's latency.
// Where each slab's prefix chain is split in two (threads >= 2 nz) the estimate
//     (1 + GROUP_COST / sg) * (REF_WARPS / resident warps)^OCC_EXP
// with GROUP_COST = 17 columns, REF_WARPS = 24 and OCC_EXP = 0.6 ranks the sizes as the
// measurements do; without the split the chain's latency grows with the group and the
// most resident blocks win. Resident blocks come from the occupancy query (registers,
// threads and shared memory of that instantiation). Ties go to the larger group. Cached
// per device, mode, storage, block size and the grid extents the shared memory depends on.
constexpr double GROUP_COST = 17.0, REF_WARPS = 24.0, OCC_EXP = 0.6;

static cbct_status choose_group(const GeomDev &G, int threads, int mode, int storage, int *sg_out)
{
    const int forced = g_forced_group.load();
    if (mode == PM_COUNT) {
        *sg_out = PROJECT_GROUP_SIZES[0];
        return CBCT_OK;
    }
    if (forced && project_smem(G, forced) <= PROJECT_SMEM_LIMIT) {
        *sg_out = forced;
        return CBCT_OK;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return check_cuda(e, "project device");
    using Key = std::tuple<int, int, int, int, int, int>;
    static std::mutex mu;
    static std::map<Key, int> cache;
    const Key key{dev, mode, storage, threads, G.nz, G.nx + G.ny};
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *sg_out = it->second;
            return CBCT_OK;
        }
    }
    const bool split = threads >= 2 * G.nz;
    int best = PROJECT_GROUP_SIZES[0];
    double best_cost = 1e300;
    for (int i = 0; i < PROJECT_N_GROUP_SIZES; ++i) {
        const int sg = PROJECT_GROUP_SIZES[i];
        const size_t smem = project_smem(G, sg);
        if (smem > PROJECT_SMEM_LIMIT) break; // grows with sg
        const void *fn = nullptr;
        cbct_status r = optin(sg, mode, storage, &fn);
        if (r != CBCT_OK) return r;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem);
        if (e != cudaSuccess) return check_cuda(e, "project occupancy");
        if (nb < 1) continue;
        const double warps = (double)nb * (threads / 32);
        const double cost = split ? (1.0 + GROUP_COST / sg) * std::pow(REF_WARPS / warps, OCC_EXP) : 1.0 / warps;
        if (cost <= best_cost) {
            best_cost = cost;
            best = sg;
        }
    }
    std::lock_guard<std::mutex> lk(mu);
    cache[key] = best;
    *sg_out = best;
    return CBCT_OK;
}

cbct_status project_set_group(int sg)
{
    if (sg != 0 && group_index(sg) < 0)
        return set_error(CBCT_ERR_INVALID_ARG, "set_project_group: %d is not one of the compiled group sizes", sg);
    g_forced_group.store(sg);
    return CBCT_OK;
}

cbct_status project_group_of(const GeomDev &G, int *sg) { return choose_group(G, proj_threads(G), PM_PLAIN, ST_F32, sg); }

cbct_status project_prepare()
{
    cbct_status t = trace_table_prepare();
    if (t != CBCT_OK) return t;
    for (int i = 0; i < PROJECT_N_GROUP_SIZES; ++i)
        for (int mode = PM_PLAIN; mode <= PM_COUNT; ++mode)
            for (int storage = ST_F32; storage <= ST_F16; ++storage) {
                if (mode == PM_COUNT && (i > 0 || storage != ST_F32)) continue;
                const void *fn = nullptr;
                cbct_status r = optin(PROJECT_GROUP_SIZES[i], mode, storage, &fn);
                if (r != CBCT_OK) return r;
            }
    return CBCT_OK;
}

cbct_status launch_project(const GeomDev &G, const float *f, long long sx, long long sy,
                           long long sz, const float *y, void *out, int mode,
                           double *partials, float count_thr, cudaStream_t st, int storage, Scalars *sc,
                           const void *traces)
{
    const int threads = proj_threads(G); // 2 rows each
    dim3 grid((unsigned)(G.nviews * G.nu), (unsigned)((G.nv + 2 * threads - 1) / (2 * threads)));
    if (project_smem_bytes(G) > PROJECT_SMEM_LIMIT)
        return set_error(CBCT_ERR_UNSUPPORTED, "project: grid too large for the projector's shared memory (nx + ny and nz)");
    if (sz != 1) return set_error(CBCT_ERR_INVALID_ARG, "project: the volume must be z-contiguous");
    if (mode == PM_COUNT) storage = ST_F32;
    int sg = 0;
    cbct_status r = choose_group(G, threads, mode, storage, &sg);
    if (r != CBCT_OK) return r;
    const void *fn = nullptr;
    r = optin(sg, mode, storage, &fn);
    if (r != CBCT_OK) return r;
    const size_t smem = project_smem(G, sg);
    GeomDev g = G;
    int isx = (int)sx, isy = (int)sy;
    const int4 *tr = mode == PM_COUNT ? nullptr : reinterpret_cast<const int4 *>(traces);
    int tcap = trace_cap(G);
    void *args[] = {&g, &f, &isx, &isy, &y, &out, &partials, &count_thr, &sc, &tr, &tcap};
    ProfToken tok = prof_start(CBCT_KERNEL_PROJECT, st);
    cudaError_t e = cudaLaunchKernel(fn, grid, dim3((unsigned)threads), args, smem, st);
    prof_stop(tok, st);
    note_launch();
    if (e != cudaSuccess) cudaGetLastError(); // the error is returned, not left pending
    return check_cuda(e, "project launch");
}

} // namespace cbct
