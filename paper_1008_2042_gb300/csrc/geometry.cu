// Geometry handle, error reporting and the non-zero count of P.
#include <atomic>
#include <mutex>
#include <vector>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "cbct_internal.cuh"

namespace cbct {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

cbct_status set_error(cbct_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return st;
}

cbct_status check_cuda(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return CBCT_OK;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return set_error(CBCT_ERR_OUT_OF_MEMORY, "%s: %s", what, cudaGetErrorString(e));
    }
    return set_error(CBCT_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void note_launch(unsigned n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// ---- per-launch timing -----------------------------------------------------------------
struct PendingTiming {
    int kind;
    cudaEvent_t a, b;
};
static std::mutex g_prof_mu;
static std::atomic<unsigned> g_prof_mask{0}; // bit k: time launches of kernel kind k
static std::vector<PendingTiming> g_prof_pending;
static std::vector<cudaEvent_t> g_prof_pool; // events reused across launches
static double g_prof_ms[CBCT_KERNEL_KINDS];
static unsigned long long g_prof_n[CBCT_KERNEL_KINDS];

static cudaEvent_t prof_event()
{
    {
        std::lock_guard<std::mutex> lk(g_prof_mu);
        if (!g_prof_pool.empty()) {
            cudaEvent_t e = g_prof_pool.back();
            g_prof_pool.pop_back();
            return e;
        }
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

ProfToken prof_start(int kind, cudaStream_t st)
{
    ProfToken t{nullptr, kind};
    if (!(g_prof_mask.load(std::memory_order_relaxed) & (1u << kind))) return t;
    // work captured into a CUDA graph is not timed launch by launch
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return t;
    t.start = prof_event();
    if (t.start) cudaEventRecord(t.start, st);
    return t;
}

void prof_stop(const ProfToken &t, cudaStream_t st)
{
    if (!t.start) return;
    cudaEvent_t b = prof_event();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!b) {
        g_prof_pool.push_back(t.start);
        return;
    }
    cudaEventRecord(b, st);
    g_prof_pending.push_back(PendingTiming{t.kind, t.start, b});
}

static cbct_status prof_resolve()
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaError_t err = cudaSuccess;
    for (auto &p : g_prof_pending) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(p.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, p.a, p.b);
        if (e == cudaSuccess) {
            g_prof_ms[p.kind] += ms;
            g_prof_n[p.kind] += 1;
        } else if (err == cudaSuccess) {
            err = e;
        }
        g_prof_pool.push_back(p.a);
        g_prof_pool.push_back(p.b);
    }
    g_prof_pending.clear();
    return check_cuda(err, "kernel timing");
}

int device_sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

GeomDev level_geom(const cbct_geometry *g, int level)
{
    const cbct_geometry_desc &d = g->desc;
    int s = 1 << level;
    GeomDev G;
    G.nx = (d.nx + s - 1) / s;
    G.ny = (d.ny + s - 1) / s;
    G.nz = (d.nz + s - 1) / s;
    double dx = d.dx * s, dy = d.dy * s, dz = d.dz * s;
    G.dx = (float)dx;
    G.dy = (float)dy;
    G.dz = (float)dz;
    G.x0 = (float)(-0.5 * G.nx * dx);
    G.y0 = (float)(-0.5 * G.ny * dy);
    G.z0 = (float)(-0.5 * G.nz * dz);
    G.nu = d.nu;
    G.nv = d.nv;
    G.nviews = d.n_views;
    G.du = (float)d.du;
    G.dv = (float)d.dv;
    G.u_first = (float)(d.u_off - 0.5 * (d.nu - 1) * d.du);
    G.v_first = (float)(d.v_off - 0.5 * (d.nv - 1) * d.dv);
    G.inv_du = (float)(1.0 / d.du);
    G.inv_dv = (float)(1.0 / d.dv);
    G.sad = (float)d.sad;
    G.sdd = (float)d.sdd;
    G.tc = (float)(d.sad / d.sdd);
    G.cs = g->d_cs;
    G.ray4 = g->d_ray4;
    G.ray2 = g->d_ray2;
    return G;
}

// Transverse ray of every (view, imager column), computed once per geometry with the
// same expressions the projector evaluates per block (so the values are identical).
__global__ void k_ray_table(GeomDev G, float4 *ray4, float2 *ray2)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= G.nviews * G.nu) return;
    const int k = t / G.nu, iu = t - k * G.nu;
    const float2 cs = G.cs[k];
    float dxr, dyr, qx, qy;
    ray_xy(G, cs.x, cs.y, imager_u(G, iu), dxr, dyr, qx, qy);
    ray4[t] = make_float4(dxr, dyr, qx, qy);
    ray2[t] = make_float2(safe_rcp(dxr), safe_rcp(dyr));
}

cbct_status ensure_scratch(cbct_geometry *g, size_t bytes)
{
    if (g->scratch_bytes >= bytes) return CBCT_OK;
    if (g->d_scratch) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return check_cuda(e, "scratch reallocation");
        cudaFree(g->d_scratch);
        g->d_scratch = nullptr;
        g->scratch_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&g->d_scratch, bytes);
    if (e != cudaSuccess) return check_cuda(e, "scratch allocation");
    g->scratch_bytes = bytes;
    return CBCT_OK;
}

} // namespace cbct

using namespace cbct;

extern "C" const char *cbct_last_error(void) { return g_last_error; }

extern "C" unsigned long long cbct_launch_count(void) { return g_launches.load(); }

extern "C" const char *cbct_version(void) { return "cbcttf 0.1 (sm_103a)"; }

extern "C" cbct_status cbct_profiling_enable(int enable)
{
    return cbct_profiling_select(enable ? (1u << CBCT_KERNEL_KINDS) - 1u : 0u);
}

extern "C" cbct_status cbct_profiling_select(unsigned int kinds)
{
    if (kinds >> CBCT_KERNEL_KINDS) return set_error(CBCT_ERR_INVALID_ARG, "profiling_select: unknown kernel kind bit");
    if (!kinds) {
        cbct_status st = prof_resolve();
        g_prof_mask.store(0u);
        return st;
    }
    g_prof_mask.store(kinds);
    return CBCT_OK;
}

extern "C" cbct_status cbct_profiling_reset(void)
{
    cbct_status st = prof_resolve();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (int k = 0; k < CBCT_KERNEL_KINDS; ++k) {
        g_prof_ms[k] = 0.0;
        g_prof_n[k] = 0;
    }
    return st;
}

extern "C" cbct_status cbct_kernel_time(int kind, double *total_ms, unsigned long long *launches)
{
    if (kind < 0 || kind >= CBCT_KERNEL_KINDS || !total_ms || !launches)
        return set_error(CBCT_ERR_INVALID_ARG, "kernel_time: bad argument");
    cbct_status st = prof_resolve();
    std::lock_guard<std::mutex> lk(g_prof_mu);
    *total_ms = g_prof_ms[kind];
    *launches = g_prof_n[kind];
    return st;
}

namespace cbct {

cbct_status validate_geometry_desc(const cbct_geometry_desc &d)
{
    if (d.nx < 1 || d.ny < 1 || d.nz < 1 || d.nu < 1 || d.nv < 1 || d.n_views < 1)
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: sizes must be >= 1");
    if (d.nv > 8192) return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: nv > 8192");
    if (d.n_views > 65535) return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: n_views > 65535");
    if (d.nx > 65535 || d.ny > 65535 || d.nz > 65535 || d.nx + d.ny > 4096 || d.nz > 1024)
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: need nx + ny <= 4096 and nz <= 1024");
    if (!(d.dx > 0 && d.dy > 0 && d.dz > 0 && d.du > 0 && d.dv > 0))
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: spacings must be > 0");
    if (!(d.sad > 0 && d.sdd > d.sad) || !std::isfinite(d.sad) || !std::isfinite(d.sdd))
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: need 0 < sad < sdd");
    if (!std::isfinite(d.u_off) || !std::isfinite(d.v_off))
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: offsets must be finite");
    double N = (double)d.nx * d.ny * d.nz, M = (double)d.n_views * d.nv * d.nu;
    if (N >= 2147483647.0 || M >= 2147483647.0)
        return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: volume or projection stack too large");
    double r = 0.5 * std::sqrt((d.nx * d.dx) * (d.nx * d.dx) + (d.ny * d.dy) * (d.ny * d.dy));
    if (!(r < d.sad) || !(r < d.sdd - d.sad))
        return set_error(CBCT_ERR_INVALID_ARG,
                         "geometry_create: the volume must lie strictly between source and imager");
    if (d.angles)
        for (int k = 0; k < d.n_views; k++)
            if (!std::isfinite(d.angles[k]))
                return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: non-finite angle");

    return CBCT_OK;
}

cbct_status check_projector_fits(const cbct_geometry_desc &d)
{
    cbct_geometry tmp{};
    tmp.desc = d;
    const size_t need = project_smem_bytes(level_geom(&tmp, 0));
    if (need > PROJECT_SMEM_LIMIT)
        return set_error(CBCT_ERR_UNSUPPORTED,
                         "geometry: the projector needs %zu bytes of shared memory per block for this grid "
                         "(limit %zu): reduce nz or nx + ny",
                         need, PROJECT_SMEM_LIMIT);
    return CBCT_OK;
}

void view_table(const cbct_geometry_desc &d, double *angles, float2 *cs)
{
    for (int k = 0; k < d.n_views; k++) {
        double t = d.angles ? d.angles[k] : 2.0 * M_PI * k / d.n_views;
        angles[k] = t;
        cs[k] = make_float2((float)std::cos(t), (float)std::sin(t));
    }
}

cbct_status launch_ray_table(const cbct_geometry *g, cudaStream_t st)
{
    const size_t nrays = (size_t)g->desc.n_views * g->desc.nu;
    const GeomDev G = level_geom(g, 0);
    k_ray_table<<<(unsigned)((nrays + 127) / 128), 128, 0, st>>>(G, g->d_ray4, g->d_ray2);
    note_launch();
    return check_cuda(cudaGetLastError(), "ray table launch");
}

} // namespace cbct

extern "C" cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, cbct_geometry **out)
{
    g_last_error[0] = '\0';
    if (!desc || !out) return set_error(CBCT_ERR_INVALID_ARG, "geometry_create: null argument");
    *out = nullptr;
    const cbct_geometry_desc &d = *desc;
    {
        cbct_status v = validate_geometry_desc(d);
        if (v != CBCT_OK) return v;
        v = check_projector_fits(d);
        if (v != CBCT_OK) return v;
    }

    cbct_geometry *g = (cbct_geometry *)calloc(1, sizeof(cbct_geometry));
    if (!g) return set_error(CBCT_ERR_OUT_OF_MEMORY, "geometry_create: host allocation");
    g->desc = d;
    g->angles = (double *)malloc(sizeof(double) * d.n_views);
    float2 *h_cs = (float2 *)malloc(sizeof(float2) * d.n_views);
    if (!g->angles || !h_cs) {
        free(g->angles);
        free(h_cs);
        free(g);
        return set_error(CBCT_ERR_OUT_OF_MEMORY, "geometry_create: host allocation");
    }
    view_table(d, g->angles, h_cs);
    g->desc.angles = g->angles;
    cudaGetDevice(&g->device);
    const size_t nrays = (size_t)d.n_views * d.nu;
    cudaError_t e = cudaMalloc(&g->d_cs, sizeof(float2) * d.n_views);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_ray4, sizeof(float4) * nrays);
    if (e == cudaSuccess) e = cudaMalloc(&g->d_ray2, sizeof(float2) * nrays);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_cs, h_cs, sizeof(float2) * d.n_views, cudaMemcpyHostToDevice);
    free(h_cs);
    if (e == cudaSuccess) {
        const GeomDev G = level_geom(g, 0);
        k_ray_table<<<(unsigned)((nrays + 127) / 128), 128>>>(G, g->d_ray4, g->d_ray2);
        note_launch();
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        cbct_status st = check_cuda(e, "geometry_create");
        cudaFree(g->d_cs);
        cudaFree(g->d_ray4);
        cudaFree(g->d_ray2);
        free(g->angles);
        free(g);
        return st;
    }
    *out = g;
    return CBCT_OK;
}

extern "C" cbct_status cbct_geometry_destroy(cbct_geometry *g)
{
    if (!g) return CBCT_OK;
    cudaError_t e = cudaDeviceSynchronize();
    cudaFree(g->d_cs);
    cudaFree(g->d_ray4);
    cudaFree(g->d_ray2);
    cudaFree(g->d_scratch);
    cudaFree(g->d_ws);
    free(g->angles);
    free(g);
    return check_cuda(e, "geometry_destroy");
}

extern "C" cbct_status cbct_set_project_group(int segments)
{
    g_last_error[0] = '\0';
    return project_set_group(segments);
}

extern "C" cbct_status cbct_project_group(const cbct_geometry *gc, int level, int *segments)
{
    g_last_error[0] = '\0';
    if (!gc || !segments) return set_error(CBCT_ERR_INVALID_ARG, "project_group: null argument");
    if (level < 0 || level > 16) return set_error(CBCT_ERR_INVALID_ARG, "project_group: bad level");
    return project_group_of(level_geom(const_cast<cbct_geometry *>(gc), level), segments);
}

// Non-zeros of P: the projector run in counting mode, one partial per block, summed on
// the host in block order.
extern "C" cbct_status cbct_count_nnz(const cbct_geometry *gc, int level, unsigned long long *nnz,
                                      cbct_stream_t stream)
{
    g_last_error[0] = '\0';
    if (!gc || !nnz) return set_error(CBCT_ERR_INVALID_ARG, "count_nnz: null argument");
    if (level < 0 || level > 16) return set_error(CBCT_ERR_INVALID_ARG, "count_nnz: bad level");
    cbct_geometry *g = const_cast<cbct_geometry *>(gc);
    GeomDev G = level_geom(g, level);
    int nb = project_num_blocks(G);
    cbct_status st = ensure_scratch(g, sizeof(double) * nb);
    if (st != CBCT_OK) return st;
    double *partials = (double *)g->d_scratch;
    float thr = 1e-3f * fminf(G.dx, fminf(G.dy, G.dz));
    long long sz = 1, sx = G.nz, sy = (long long)G.nx * G.nz;
    // counting mode reads no volume
    st = launch_project(G, nullptr, sx, sy, sz, nullptr, nullptr, PM_COUNT, partials, thr,
                        (cudaStream_t)stream);
    if (st != CBCT_OK) return st;
    double *h = (double *)malloc(sizeof(double) * nb);
    if (!h) return set_error(CBCT_ERR_OUT_OF_MEMORY, "count_nnz: host allocation");
    cudaError_t e = cudaMemcpyAsync(h, partials, sizeof(double) * nb, cudaMemcpyDeviceToHost,
                                    (cudaStream_t)stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) {
        free(h);
        return check_cuda(e, "count_nnz");
    }
    double total = 0.0;
    for (int b = 0; b < nb; b++) total += h[b];
    free(h);
    *nnz = (unsigned long long)(total + 0.5);
    return CBCT_OK;
}
