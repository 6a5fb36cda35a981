// Internal declarations of the cbcttf CUDA library (not part of the C ABI).
//
// Internal data layouts (the public ABI converts at its boundary):
//   volumes inside the iteration are z-fastest, [ny][nx][nz], so that the projector's
//   warps, whose lanes are adjacent imager rows, read adjacent z voxels of one (x, y)
//   column; public volumes are x-fastest [nz][ny][nx]. Kernels that touch volumes take
//   the element strides (sx, sy, sz) so they serve both layouts.
//   projection stacks are always [n_views][nv][nu].
#pragma once

#include <atomic>

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "../../include/cbcttf.h"

namespace cbct {

// Geometry of one multigrid level as the kernels see it (FP32, derived from the FP64
// description on the host). All rays of view k at imager column u share their
// transverse (x, y) path; the v coordinate only tilts the ray in z (Section 2.1 geometry:
// the source orbit lies in the plane z = 0 and the imager's v axis is z).
struct GeomDev {
    int nx, ny, nz;
    float dx, dy, dz;
    float x0, y0, z0;       // volume corner, -n * d / 2
    int nu, nv, nviews;
    float du, dv;
    float u_first, v_first; // coordinates of pixel 0
    float inv_du, inv_dv;
    float sad, sdd;
    float tc;               // sad / sdd: ray parameter of the isocentre plane
    const float2 *cs;       // (cos t_k, sin t_k) per view, device memory
    const float4 *ray4;     // per (view, imager column): (dxr, dyr, qx, qy) of ray_xy
    const float2 *ray2;     // per (view, imager column): (1/dxr, 1/dyr) of safe_rcp
};

// Rays are parametrised as X(tau) = Q + tau * d, d = D - S (source to pixel centre) and
// Q = S + tc * d, the point where the ray crosses the plane through the rotation axis
// parallel to the imager. For the circular orbit Q = tc * (u e_u + v e_z), so Q and the
// plane offsets stay small numbers and FP32 keeps ~1e-5 mm resolution along the ray.
// tau runs from -tc (source) to 1 - tc (pixel); the volume lies strictly inside.

// Coordinate of plane i of an axis with origin o and spacing h. P and P^T both use this
// exact expression so that both compute bit-identical crossing parameters.
__device__ __forceinline__ float plane_at(int i, float h, float o) { return fmaf((float)i, h, o); }

// Transverse part of ray (view with cos/sin c, s; imager coordinate u).
__device__ __forceinline__ void ray_xy(const GeomDev &G, float c, float s, float u, float &dxr,
                                       float &dyr, float &qx, float &qy)
{
    dxr = fmaf(-u, s, -G.sdd * c);
    dyr = fmaf(u, c, -G.sdd * s);
    float tu = G.tc * u;
    qx = -tu * s;
    qy = tu * c;
}

// 1 / d with a finite stand-in for d == 0 (such a ray never crosses that plane family).
__device__ __forceinline__ float safe_rcp(float d) { return d != 0.0f ? __frcp_rn(d) : 1e30f; }

// tau at which a ray with transverse offset q and reciprocal direction inv crosses plane p.
__device__ __forceinline__ float tau_plane(float p, float q, float inv) { return (p - q) * inv; }

// tau at which the ray through imager row v (1/v = inv_v) crosses the plane z = p:
// z(tau) = v (tc + tau) for every ray of the orbit, hence tau = p / v - tc.
__device__ __forceinline__ float tau_zplane(float p, float inv_v, float tc) { return fmaf(p, inv_v, -tc); }

__device__ __forceinline__ float imager_u(const GeomDev &G, int iu) { return fmaf((float)iu, G.du, G.u_first); }
__device__ __forceinline__ float imager_v(const GeomDev &G, int iv) { return fmaf((float)iv, G.dv, G.v_first); }

// Exact ceil / floor of |x| < 2^22 through the FP adder (no conversion instruction):
// adding 1.5 * 2^23 with rounding up / down leaves the integer in the low mantissa bits.
__device__ __forceinline__ int ceil_small(float x) { return __float_as_int(__fadd_ru(x, 12582912.0f)) - 0x4B400000; }
__device__ __forceinline__ int floor_small(float x) { return __float_as_int(__fadd_rd(x, 12582912.0f)) - 0x4B400000; }

// Length of ray (d) per unit tau: |D - S|.
__device__ __forceinline__ float ray_length(float dxr, float dyr, float v)
{
    return sqrtf(fmaf(dxr, dxr, fmaf(dyr, dyr, v * v)));
}

// Storage type of the projection-domain working vectors (y, r, q) and of stored frame
// coefficients: FP32, BF16 or FP16. Arithmetic is always FP32 (FP64 for inner products).
enum StorageType { ST_F32 = 0, ST_BF16 = 1, ST_F16 = 2 };

template <typename T> __device__ __forceinline__ float load_as_float(const T *p);
template <> __device__ __forceinline__ float load_as_float<float>(const float *p) { return __ldg(p); }
template <> __device__ __forceinline__ float load_as_float<__nv_bfloat16>(const __nv_bfloat16 *p)
{
    return __bfloat162float(__ldg(p));
}
template <> __device__ __forceinline__ float load_as_float<__half>(const __half *p) { return __half2float(__ldg(p)); }
template <typename T> __device__ __forceinline__ void store_from_float(T *p, float v);
template <> __device__ __forceinline__ void store_from_float<float>(float *p, float v) { *p = v; }
template <> __device__ __forceinline__ void store_from_float<__nv_bfloat16>(__nv_bfloat16 *p, float v)
{
    *p = __float2bfloat16_rn(v);
}
template <> __device__ __forceinline__ void store_from_float<__half>(__half *p, float v) { *p = __float2half_rn(v); }

// streaming (evict-first) store of a value that is not read again by this kernel
template <typename T> __device__ __forceinline__ void store_stream(T *p, float v);
template <> __device__ __forceinline__ void store_stream<float>(float *p, float v) { __stcs(p, v); }
template <> __device__ __forceinline__ void store_stream<__nv_bfloat16>(__nv_bfloat16 *p, float v)
{
    __stcs(p, __float2bfloat16_rn(v));
}
template <> __device__ __forceinline__ void store_stream<__half>(__half *p, float v) { __stcs(p, __float2half_rn(v)); }

static inline size_t storage_bytes(int storage) { return storage == ST_F32 ? 4 : 2; }

// Opts a kernel into more than 48 KB of dynamic shared memory. The attribute belongs to
// the function on one device, so it is set once per device (`done` holds one bit each).
template <typename Kernel>
inline cudaError_t smem_optin_once(Kernel *fn, int bytes, std::atomic<unsigned long long> &done)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

// Device-resident scalars of CGLS (Appendix 1), FP64.
struct Scalars {
    double gamma;    // ||s||^2
    double delta;    // ||q||^2
    double alpha;    // gamma / delta
    double beta;     // gamma' / gamma
    double rr;       // ||r||^2 (monitoring)
    double kappa;    // q is stored as kappa * q, kappa = 1 / sqrt(gamma): keeps FP16 in range
    unsigned int flags; // bit 0: a reduction was not finite; bit 1: a projector block's wait timed out
    unsigned int pad;
};

enum FinalizeOp { FIN_GAMMA = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_RR = 3 };

// Projector epilogues (q = |D - S| * sum of f * dtau is the projection of the ray).
enum ProjectMode {
    PM_PLAIN = 0,      // out = q                                     (public P)
    PM_Q_SCALED = 1,   // out = kappa * q (stored type), partial sums of q^2
    PM_RESID = 2,      // out = y - q (stored type), partial sums of (y - q)^2
    PM_COUNT = 3       // count segments longer than a threshold
};

// ---- host side ----------------------------------------------------------------------

// Optional per-launch timing (cbct_profiling_enable): events around each launch.
struct ProfToken {
    cudaEvent_t start;
    int kind;
};
ProfToken prof_start(int kind, cudaStream_t st);
void prof_stop(const ProfToken &t, cudaStream_t st);

// Launch a kernel with optional timing and the launch counter:
//   CBCT_TIMED(kind, stream, kernel<<<grid, block, smem, stream>>>(args...));
#define CBCT_TIMED(kind, st, ...)                                                                  \
    do {                                                                                           \
        ::cbct::ProfToken _cbct_tok = ::cbct::prof_start((kind), (st));                            \
        __VA_ARGS__;                                                                               \
        ::cbct::prof_stop(_cbct_tok, (st));                                                        \
        ::cbct::note_launch();                                                                     \
    } while (0)

cbct_status set_error(cbct_status st, const char *fmt, ...);
cbct_status check_cuda(cudaError_t e, const char *what);
void note_launch(unsigned n = 1);
int device_sm_count();

// Launchers (all asynchronous on `st`; return CBCT_ERR_CUDA on launch failure).
// Volume element (ix, iy, iz) lives at ix*sx + iy*sy + iz*sz.
int project_num_blocks(const GeomDev &G);
// Bytes past the end of a volume that the projector may read (its 16-byte staging copies
// round the last z-line up): every volume buffer passed to launch_project is allocated with
// at least this much slack, and its base is 16-byte aligned.
constexpr size_t PROJECT_VOLUME_SLACK = 64;

// Dynamic shared memory a projector block may use (opted in per kernel).
constexpr size_t PROJECT_SMEM_LIMIT = 200 * 1024;

// out holds `storage`-typed values (PM_COUNT: none); y is FP32; sc supplies kappa in
// PM_Q_SCALED and, when given, receives bit 1 of its flags if a block's wait for its trace
// record timed out (that block's rows are NaN). With FP32 storage the CGLS modes store
// |D - S| r and |D - S| q. traces: the grid's trace table from launch_trace_table built with
// the same sx, sy (the projector then copies each column's phase 1 instead of computing
// it), or nullptr.
cbct_status launch_project(const GeomDev &G, const float *f, long long sx, long long sy,
                           long long sz, const float *y, void *out, int mode,
                           double *partials, float count_thr, cudaStream_t st,
                           int storage = ST_F32, Scalars *sc = nullptr, const void *traces = nullptr);
// The projector's trace table of a grid (trace_table_bytes(G) bytes, 16-byte aligned):
// phase 1 of every (view, imager column), column offsets for the strides sx, sy.
size_t trace_table_bytes(const GeomDev &G);
cbct_status launch_trace_table(const GeomDev &G, long long sx, long long sy, void *tab, cudaStream_t st);
cbct_status trace_table_prepare();
int backproject_num_blocks(const GeomDev &G);
// Upper bound of backproject_num_blocks over every grid no larger than G's (any z chunk).
int backproject_max_blocks(const GeomDev &G);
// ps: per-(view, imager column) prefix sums over rows of the |D - S|-weighted stack,
// [n_views][nv + 1][nu] float2 (prefix of the rows below m, value of row m), built by
// launch_row_prefix.
cbct_status launch_backproject(const GeomDev &G, const float2 *ps, float *out, long long sx,
                               long long sy, long long sz, float *out2, double *partials,
                               cudaStream_t st);
cbct_status launch_row_prefix(const GeomDev &G, const void *g, float2 *ps, int prescale,
                              cudaStream_t st, int storage = ST_F32);
cbct_status launch_backproject_eq3(const GeomDev &G, const float *g, float *f, float pref,
                                   cudaStream_t st);

// alpha holds `storage`-typed coefficients (FP32, BF16 or FP16); arithmetic is FP32
cbct_status launch_tf_analyze(int n0, int n1, int n2, const float *f, void *alpha,
                              cudaStream_t st, int storage = ST_F32);
cbct_status launch_tf_synth_shrink(int n0, int n1, int n2, const void *alpha, float mu,
                                   int positivity, float *f, cudaStream_t st, int storage = ST_F32);
// Fused f_new = H(W^T T_mu W x) and, if vout != nullptr, v = f_new + coef (f_new - f_old).
cbct_status launch_tf_shrink_fused(int n0, int n1, int n2, const float *x, float mu, int positivity,
                                   float *fnew, const float *fold, float coef, float *vout,
                                   cudaStream_t st);
// Public x-fastest [nz][ny][nx] <-> internal z-fastest [ny][nx][nz] volume layout.
cbct_status transpose(const float *in, float *out, int nx, int ny, int nz, bool to_internal,
                      cudaStream_t st);

} // namespace cbct

// Library-owned geometry handle.
struct cbct_geometry {
    cbct_geometry_desc desc; // angles points into `angles`
    double *angles;          // host copy
    int device;
    float2 *d_cs;            // per-view (cos, sin)
    float4 *d_ray4;          // per (view, imager column) transverse ray (ray_xy)
    float2 *d_ray2;          // per (view, imager column) reciprocal directions
    float *d_scratch;        // public project/backproject scratch (lazily allocated)
    size_t scratch_bytes;
    void *d_ws;              // reconstruction workspace (lazily allocated)
    size_t ws_bytes;
};

namespace cbct {
constexpr int MAX_LEVELS = 8; // multigrid levels a reconstruction may use
GeomDev level_geom(const cbct_geometry *g, int level);
cbct_status ensure_scratch(cbct_geometry *g, size_t bytes);

// Geometry pieces for callers that build a cbct_geometry in memory they own (the request
// server): argument checks, the host view table (angles and FP32 cos/sin), and the
// stream-ordered ray-table kernel.
cbct_status validate_geometry_desc(const cbct_geometry_desc &d);
// Shared memory one projector block needs on the finest grid (the largest level).
size_t project_smem_bytes(const GeomDev &G);
// Force the projector's column-group size (0: choose per launch); the size a PM_PLAIN FP32
// launch on G uses.
cbct_status project_set_group(int sg);
cbct_status project_group_of(const GeomDev &G, int *sg);
// UNSUPPORTED when the projector's per-block shared memory for this geometry exceeds what
// it may use (its staged z-lines and tables grow with nz, its segment lists with nx + ny).
cbct_status check_projector_fits(const cbct_geometry_desc &d);
void view_table(const cbct_geometry_desc &d, double *angles, float2 *cs);
cbct_status launch_ray_table(const cbct_geometry *g, cudaStream_t st);

// The reconstruction as pure stream work: no allocation, no synchronisation, nothing read
// back (capturable into a CUDA graph). ws must hold reconstruct_ws_bytes(g) bytes, 256-byte
// aligned; the iteration's status word (bit 0: a non-finite inner product) is at
// reconstruct_flags_address(g, ws) once the work has run.
cbct_status validate_recon_args(float mu, float lambda, int levels, const int *iters, const cbct_recon_opts &o);
size_t reconstruct_ws_bytes(const cbct_geometry *g);
cbct_status reconstruct_enqueue(const float *y, cbct_geometry *g, float mu, int levels, const int *iters,
                                const cbct_recon_opts &o, void *ws, size_t ws_bytes, float *f_out, cudaStream_t st);
const unsigned int *reconstruct_flags_address(const cbct_geometry *g, void *ws);

// The same reconstruction enqueued one step at a time (one A2 iteration per step; the
// set-up of a level rides on its first step, the change back to the public layout on the
// last). Consecutive steps may go to different streams if the caller orders them (an
// event recorded after one step, waited on by the stream of the next). The cursor keeps
// iters; the buffers must outlive the last step.
struct ReconCursor;
cbct_status reconstruct_cursor_create(const float *y, cbct_geometry *g, float mu, int levels, const int *iters,
                                      const cbct_recon_opts &o, void *ws, size_t ws_bytes, float *f_out,
                                      ReconCursor **out);
cbct_status reconstruct_cursor_step(ReconCursor *c, cudaStream_t st);
bool reconstruct_cursor_finished(const ReconCursor *c);
void reconstruct_cursor_destroy(ReconCursor *c);

// Sets every kernel attribute the launchers would otherwise set on first use (shared
// memory opt-ins) on the current device, so that later launches can be graph-captured.
cbct_status project_prepare();
cbct_status tf_prepare();
}
