/*
 * cbcttf — tight-frame regularised cone-beam CT reconstruction on one GPU (sm_103a).
 *
 * C ABI of the CUDA library. It implements the hot path of Jia, Dong, Lou and Jiang,
 * "GPU-based iterative cone beam CT reconstruction using tight frame regularization":
 * the Siddon forward projector P, its exact adjoint P^T, the piecewise-linear tight-frame
 * analysis W (the paper's D) and synthesis W^T with vector soft-thresholding T_mu and the
 * positivity correction H, CGLS, Algorithm A2 and the coarse-to-fine multigrid.
 *
 * Conventions shared by every call
 *   - Volumes are float32, layout [nz][ny][nx] (x fastest). Voxel (ix, iy, iz) is the
 *     half-open box [x0 + ix dx, x0 + (ix+1) dx) x ..., with x0 = -nx dx / 2 (the volume
 *     is centred on the rotation axis z); the same for y and z.
 *   - Projection stacks are float32, layout [n_views][nv][nu] (u fastest).
 *   - Tight-frame coefficients are float32, layout [27][nz][ny][nx]; channel
 *     i = l + 3 m + 9 n holds the filter h_l along x, h_m along y and h_n along z.
 *   - Geometry (Section 2.1, Fig. 1): view k at angle t_k puts the source at
 *     sad (cos t, sin t, 0) and the imager centre at -(sdd - sad)(cos t, sin t, 0); the
 *     imager u axis is (-sin t, cos t, 0), its v axis is z. Pixel (iu, iv) is centred at
 *     u = u_off + (iu - (nu-1)/2) du, v = v_off + (iv - (nv-1)/2) dv. One ray per pixel
 *     centre. Lengths in mm, attenuation in 1/mm, angles in radians.
 *   - Data pointers are DEVICE pointers on the device that was current when the geometry
 *     was created, owned by the caller, never retained after the call returns. Outputs
 *     are overwritten (not accumulated). Input and output buffers must not overlap.
 *   - Every call is enqueued on `stream` (NULL = the legacy default stream) and returns
 *     without waiting, except where stated. Arguments are validated before anything is
 *     launched; an invalid call launches nothing and returns CBCT_ERR_INVALID_ARG.
 *   - Errors are returned as cbct_status; cbct_last_error() gives a message for the
 *     calling thread. No C++ exception crosses this interface.
 *   - A geometry handle is not thread-safe: calls sharing one handle must not run
 *     concurrently from several host threads (they share the handle's device scratch).
 */
#ifndef CBCTTF_H
#define CBCTTF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *cbct_stream_t;

typedef enum {
    CBCT_OK = 0,
    CBCT_ERR_INVALID_ARG = 1,   /* null pointer, non-positive size, inconsistent geometry */
    CBCT_ERR_OUT_OF_MEMORY = 2, /* device allocation failed, or the workspace is too small */
    CBCT_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed */
    CBCT_ERR_NONFINITE = 4,     /* an inner product of the iteration was NaN or Inf */
    CBCT_ERR_UNSUPPORTED = 5,   /* a parameter the method does not define (e.g. lambda != 0) */
    CBCT_ERR_TIMEOUT = 6        /* a wait ended before the awaited work finished */
} cbct_status;

/* Scan geometry (Section 2.1, Fig. 1; Section 3 gives sad = 1000 mm, sdd = 1500 mm). */
typedef struct {
    int nx, ny, nz;          /* voxels per axis, >= 1 */
    double dx, dy, dz;       /* voxel size (mm), > 0 */
    int nu, nv;              /* imager pixels, >= 1, nv <= 8192 */
    double du, dv;           /* pixel pitch (mm), > 0 */
    double u_off, v_off;     /* imager offset from the central ray (mm) */
    double sad, sdd;         /* source-to-axis and source-to-imager distance (mm) */
    int n_views;             /* number of views, 1 .. 65535 */
    const double *angles;    /* host array of n_views angles (rad); NULL = 2 pi k / n_views */
} cbct_geometry_desc;

/*
 * Storage type of projections and frame coefficients in the typed (_ex) entry points and
 * of the projection-domain vectors inside CGLS. Arithmetic is FP32 whatever the storage
 * (line integrals, stencils, updates), inner products and norms FP64. The paper computes
 * in FP32 throughout; the 16-bit storage types have no counterpart there.
 * BF16 and FP16 values are IEEE-style binary16 / bfloat16, round-to-nearest-even.
 */
typedef enum {
    CBCT_F32 = 0,  /* float */
    CBCT_BF16 = 1, /* bfloat16: 8 significand bits, FP32's exponent range */
    CBCT_F16 = 2   /* IEEE binary16: 11 significand bits, |x| < 65504 */
} cbct_dtype;

/* Opaque, library-owned geometry: per-view tables and device scratch. */
typedef struct cbct_geometry cbct_geometry;

/* Options of the outer iteration. */
typedef struct {
    int n_cgls;     /* CGLS updates per outer iteration (Appendix 1: "M = 2~3"); default 3 */
    int momentum;   /* 1 = Algorithm A2 (default), 0 = Algorithm A1 */
    int positivity; /* 1 = apply H after the shrinkage (default), 0 = skip H */
    int storage;    /* cbct_dtype of the CGLS residual r and projected direction q (default
                       CBCT_F32). With CBCT_F16, q is stored as q / ||P^T r|| so that it stays
                       in range; y, x, p, s and f stay FP32. */
} cbct_recon_opts;

/*
 * Creates a geometry on the current CUDA device and copies the view table to it.
 * The whole volume must lie strictly between the source and the imager for every view
 * (its transverse half-diagonal below both sad and sdd - sad). Sizes are limited to
 * nx + ny <= 4096, nz <= 1024, nx*ny*nz < 2^31 voxels and n_views*nv*nu < 2^31 pixels,
 * and jointly by the projector's shared memory per block, about
 * 16 (nx + ny) + 140 nz bytes <= 200 KiB (it binds above nx + ny = 3806 for nz = 1024;
 * nz <= 990 at nx + ny = 4096); a larger grid gives UNSUPPORTED.
 * Synchronous. Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA.
 */
cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, cbct_geometry **out);

/* Frees the geometry and its device scratch (waits for the device). NULL is a no-op. */
cbct_status cbct_geometry_destroy(cbct_geometry *geom);

/*
 * Forward projection g = P f (Eq. (1); Section 2.2.1: one ray per pixel, Siddon's exact
 * ray tracing): g_i = sum_j a_ij f_j, a_ij = length (mm) of ray i inside voxel j.
 * f: device [nz][ny][nx]; g: device [n_views][nv][nu]. FP32 arithmetic.
 * Uses the geometry's scratch (allocated on first use, grown when too small): the volume in
 * the projector's z-fastest layout and the grid's ray-trace table, 16 + 8 (nx + ny + 2)
 * bytes per (view, imager column). Every projection block copies its trace record with a
 * bounded wait; should that wait ever run out, the block's rows are written as NaN (the
 * call itself cannot see it; cbct_reconstruct reports it as TIMEOUT).
 */
cbct_status cbct_project(const cbct_geometry *geom, const float *f, float *g,
                         cbct_stream_t stream);

/*
 * cbct_project with the projections stored as g_type (FP32 arithmetic, one rounding of
 * every line integral to the storage type). g: device [n_views][nv][nu] of g_type.
 * Errors: as cbct_project; INVALID_ARG for an unknown g_type.
 */
cbct_status cbct_project_ex(const cbct_geometry *geom, const float *f, void *g,
                            cbct_dtype g_type, cbct_stream_t stream);

/*
 * Exact adjoint f = P^T g: f_j = sum_i a_ij g_i with the same a_ij as cbct_project, so
 * <P f, g> = <f, P^T g> (Eq. (A1)). Computed by gathering per voxel (no atomics; the
 * result does not depend on scheduling). The paper's own backprojector (Eq. (3)) is an
 * approximation of this operator and is not what this call computes.
 * g: device [n_views][nv][nu]; f: device [nz][ny][nx]. FP32 arithmetic.
 * Uses the geometry's scratch (allocated on first use: per-column row prefix sums,
 * n_views * nu * (nv + 1) float pairs).
 */
cbct_status cbct_backproject(const cbct_geometry *geom, const float *g, float *f,
                             cbct_stream_t stream);

/* cbct_backproject reading projections stored as g_type (widened to FP32 on load). */
cbct_status cbct_backproject_ex(const cbct_geometry *geom, const void *g, cbct_dtype g_type,
                                float *f, cbct_stream_t stream);

/*
 * The paper's own backprojector, Eq. (3) (Section 2.2.2, derived in Appendix 2): for every
 * voxel centre x and view, the imager value at the point u* where the ray from the source
 * through x meets the imager (bilinear interpolation, zero outside the imager), weighted
 * by (dx dy dz / (du dv)) L^3(u*) / (L0 l^2(x)), summed over views. It approximates the
 * exact adjoint (the paper reports the dot identity within about 1%); cbct_backproject
 * computes the exact transpose instead. Same arguments and layouts as cbct_backproject.
 */
cbct_status cbct_backproject_eq3(const cbct_geometry *geom, const float *g, float *f,
                                 cbct_stream_t stream);

/*
 * Batched P and exact P^T: `batch` volumes [batch][nz][ny][nx] and stacks
 * [batch][n_views][nv][nu], contiguous, same geometry; item b is processed exactly as by
 * cbct_project / cbct_backproject. batch = 0 does nothing.
 */
cbct_status cbct_project_batch(const cbct_geometry *geom, int batch, const float *f, float *g,
                               cbct_stream_t stream);
cbct_status cbct_backproject_batch(const cbct_geometry *geom, int batch, const float *g,
                                   float *f, cbct_stream_t stream);

/*
 * Tight-frame analysis alpha = W f (Section 2.1): alpha_i(x) = sum_k psi_i(k) f(x - k),
 * psi_i(k) = h_l(k_x) h_m(k_y) h_n(k_z) with h_0 = [1,2,1]/4, h_1 = sqrt(2)/4 [1,0,-1],
 * h_2 = [-1,2,-1]/4 (taps at offsets -1, 0, +1). The volume is periodic along every
 * axis, which makes W^T W = I exact.
 * f: device [nz][ny][nx]; alpha27: device [27][nz][ny][nx].
 */
cbct_status cbct_tf_analyze(int nx, int ny, int nz, const float *f, float *alpha27,
                            cbct_stream_t stream);

/* cbct_tf_analyze storing the 27 channels as a_type (FP32 stencils, one rounding each). */
cbct_status cbct_tf_analyze_ex(int nx, int ny, int nz, const float *f, void *alpha27,
                               cbct_dtype a_type, cbct_stream_t stream);

/*
 * Shrinkage and synthesis f = H(W^T T_mu alpha) (Eq. (2) and Section 2.1): at every
 * voxel the 26 high-pass coefficients are scaled by max(1 - mu / ||alpha_h||, 0) (0 when
 * the norm is 0), alpha_0 is kept, then f(x) = sum_i sum_k psi_i(k) alpha_i(x + k)
 * (periodic); negative voxels are set to 0 if positivity != 0. mu >= 0.
 * alpha27: device [27][nz][ny][nx] (not modified); f: device [nz][ny][nx].
 */
cbct_status cbct_tf_synthesize_shrink(int nx, int ny, int nz, const float *alpha27,
                                      float mu, int positivity, float *f,
                                      cbct_stream_t stream);

/* cbct_tf_synthesize_shrink reading coefficients stored as a_type (widened to FP32). */
cbct_status cbct_tf_synthesize_shrink_ex(int nx, int ny, int nz, const void *alpha27,
                                         cbct_dtype a_type, float mu, int positivity,
                                         float *f, cbct_stream_t stream);

/*
 * The regularisation step of Algorithms A1/A2 in one pass: f_out = H(W^T T_mu W f)
 * (Section 2.1, Eq. (2)), equal to cbct_tf_analyze followed by cbct_tf_synthesize_shrink
 * but without materialising the 27 coefficient channels (they stay on chip). Periodic
 * boundary, layouts as above. f and f_out must not overlap.
 */
cbct_status cbct_tf_shrink(int nx, int ny, int nz, const float *f, float mu, int positivity,
                           float *f_out, cbct_stream_t stream);

/*
 * CGLS (Appendix 1): n_iter updates of x for min ||P x - y||^2 starting from x.
 * Inner products are accumulated in FP64 on the device; if ||P^T r||^2 or ||P p||^2
 * becomes zero the remaining updates leave x unchanged.
 * y: device [n_views][nv][nu]; x: device [nz][ny][nx], read and overwritten.
 * Uses the geometry's reconstruction workspace (allocated on first use).
 * Synchronises the stream to check for non-finite inner products (NONFINITE).
 */
cbct_status cbct_cgls(const cbct_geometry *geom, const float *y, float *x, int n_iter,
                      cbct_stream_t stream);

/*
 * Reconstruction (Section 2.2.3 multigrid around Algorithm A2 of Section 2.1):
 * `levels` grids, level l having ceil(n / 2^l) voxels per axis at 2^l times the voxel
 * size with the same centre; the imager and y are used unchanged on every level.
 * Starts from f = 0 on the coarsest grid, runs iters[levels-1-l] A2 iterations on
 * level l (iters is listed coarsest first), and prolongs each level's result by
 * trilinear interpolation as the next finer level's initial guess. Each A2 iteration
 * does n_cgls CGLS updates from the momentum point v, then f = H(W^T T_mu W x).
 * mu >= 0 is the threshold of Eq. (2), the method's only tuning parameter (Section 2.1);
 * lambda must be 0 (UNSUPPORTED otherwise: the method has no second parameter).
 * y: device [n_views][nv][nu]; f_out: device [nz][ny][nx] (finest grid).
 * Uses the geometry's reconstruction workspace (allocated on first use; its size is
 * cbct_reconstruct_workspace_size). Synchronises the stream at the end.
 * Errors: INVALID_ARG, UNSUPPORTED, OUT_OF_MEMORY, CUDA, NONFINITE; TIMEOUT if a
 * projector block's bounded wait for its precomputed ray trace ran out (its rows are then
 * NaN).
 */
cbct_status cbct_reconstruct(const float *y, const cbct_geometry *geom, float mu,
                             float lambda, int levels, const int *iters, float *f_out,
                             cbct_stream_t stream);

/*
 * As cbct_reconstruct with options (NULL = defaults) and a caller-provided device
 * workspace of at least cbct_reconstruct_workspace_size bytes (NULL = the geometry's
 * own workspace). The workspace must not be used by anything else while the call's
 * work is on the device.
 */
cbct_status cbct_reconstruct_ex(const float *y, const cbct_geometry *geom, float mu,
                                float lambda, int levels, const int *iters,
                                const cbct_recon_opts *opts, void *workspace,
                                size_t workspace_bytes, float *f_out, cbct_stream_t stream);

/* Bytes of device workspace cbct_reconstruct_ex needs for this geometry (any levels). */
cbct_status cbct_reconstruct_workspace_size(const cbct_geometry *geom, size_t *bytes);

/*
 * Trilinear prolongation between multigrid levels (Section 2.2.3, "linear
 * interpolation"): every fine voxel centre is interpolated from the coarse grid, both
 * grids centred on the origin, coarse coordinates clamped to the hull of coarse voxel
 * centres. fc: device [cnz][cny][cnx]; ff: device [nz][ny][nx].
 */
cbct_status cbct_prolong(int cnx, int cny, int cnz, double cdx, double cdy, double cdz,
                         const float *fc, int nx, int ny, int nz, double dx, double dy,
                         double dz, float *ff, cbct_stream_t stream);

/*
 * Restriction, the counterpart of cbct_prolong (not used by the coarse-to-fine scheme
 * of Section 2.2.3): each coarse voxel is the mean of the fine voxels whose centres lie
 * inside it (0 if there are none). ff: device [nz][ny][nx]; fc: device [cnz][cny][cnx].
 */
cbct_status cbct_restrict(int nx, int ny, int nz, double dx, double dy, double dz,
                          const float *ff, int cnx, int cny, int cnz, double cdx,
                          double cdy, double cdz, float *fc, cbct_stream_t stream);

/*
 * Number of non-zeros of P on multigrid level `level` (0 = the geometry's own grid):
 * the (ray, voxel) pairs whose segment is longer than 1e-3 of the smallest voxel side,
 * counted by the projector's own traversal. This is the work unit of the ray-voxel
 * update rate (Section 2.2.2 quotes about 4e9 for a clinical case). Synchronous.
 */
cbct_status cbct_count_nnz(const cbct_geometry *geom, int level, unsigned long long *nnz,
                           cbct_stream_t stream);

/*
 * Forward projection without device allocation. Same operation and result (bit for bit)
 * as cbct_project, for callers that cannot allocate device memory while they run: a
 * service that fixes its device memory footprint at start-up and treats any later
 * allocation as a failure, or a latency-critical loop that cannot afford the device-wide
 * synchronisation an allocation may cause. The paper has no counterpart: this is an
 * interface variant, not a step of the method. Instead of the geometry's lazily
 * allocated scratch it uses one fixed scratch array of CBCT_PROJECT_STATIC_MAX_VOXELS
 * floats that the library places on every GPU that loads it, held until the process
 * exits. Volumes larger than that are rejected with CBCT_ERR_INVALID_ARG. The geometry
 * must have been created beforehand. The first call on a device looks up the array's
 * device address (cudaGetSymbolAddress) and keeps it for the life of the process; make
 * that first call before any stream capture. A device reset (cudaDeviceReset) after the
 * first call is not supported: the kept address would no longer be valid. All calls
 * share the one array, so calls whose work overlaps on the GPU (different streams, or
 * several host threads) race and must be serialised by the caller. Each call overwrites
 * the part of the array it uses before reading it, so no clearing is needed.
 */
#define CBCT_PROJECT_STATIC_MAX_VOXELS 4194304
cbct_status cbct_project_static(const cbct_geometry *geom, const float *f, float *g,
                                cbct_stream_t stream);

/*
 * Request server: reconstructions of different geometries, view counts, noise levels and
 * storage types served concurrently on one GPU (continuous batching). The paper
 * reconstructs one scan at a time; this is an execution interface around the same
 * reconstruction, not a step of the method.
 *
 * Each submitted request is a full cbct_reconstruct_ex call described by its geometry,
 * host projections and options. A worker thread owned by the server admits queued
 * requests whenever a stream slot is free and the device bytes of all admitted requests
 * stay within the budget (granted in submission order); requests submitted while others
 * run are admitted as soon as slots and memory free up, and their kernels overlap on the
 * device. Two rules keep overlap from costing throughput: the summed volumes of the
 * admitted requests stay within an L2 bound (a request that would break it waits, and
 * smaller requests behind it may start first for a bounded time), and stream priorities
 * order the admitted requests' thread blocks (by size, smallest first, or by age, oldest
 * first).
 * An admitted request holds one device block (its geometry tables, y, the reconstruction
 * workspace and the output volume) taken from a stream-ordered memory pool; it runs on
 * its slot's stream as: copy y in, the whole multigrid iteration (captured once into a
 * CUDA graph and launched, when use_graphs != 0), copy the volume out. The block returns
 * to the pool when the request completes. The result of a request does not depend on
 * what else runs: every kernel of the iteration is deterministic and requests share no
 * device state.
 */
typedef struct cbct_server cbct_server;

#define CBCT_PRIORITY_NONE 0
#define CBCT_PRIORITY_SIZE 1
#define CBCT_PRIORITY_AGE 2

typedef struct {
    size_t hbm_budget_bytes; /* device bytes admitted requests may hold together; 0 = 150 GB,
                                capped at 90% of the device memory free at creation */
    int max_active;          /* requests on the device at once (one stream each), 1..64 */
    int use_graphs;          /* 1 = capture each request's iteration into a CUDA graph */
    size_t l2_budget_bytes;  /* bound on the summed finest-volume bytes of the admitted
                                requests, so that the volumes the projectors re-read stay in
                                L2 together (an idle device always admits); 0 = the device's
                                L2 size */
    int size_priority;       /* stream priorities (a request's thread blocks are scheduled
                                ahead of those of lower-priority requests):
                                CBCT_PRIORITY_NONE (0) = all equal;
                                CBCT_PRIORITY_SIZE (1) = by volume size, smallest first;
                                CBCT_PRIORITY_AGE (2) = by admission order, oldest first:
                                the oldest request runs as if alone and the others fill
                                what it leaves idle; a request moves up as older ones
                                finish (its iteration is enqueued one A2 iteration at a
                                time, each on the streams of its current rank; use_graphs
                                is ignored) */
    double max_bypass_s;     /* a queued request held back by the L2 bound is overtaken by
                                later requests only until it has waited this long; 0 = 2 s */
} cbct_server_opts;

/* Times are seconds on a steady clock since the server was created. */
typedef struct {
    int status;             /* cbct_status of the request (OK once complete) */
    int done;               /* 1 when the volume has been written to f_host */
    double t_submit;        /* cbct_server_submit returned */
    double t_admit;         /* the worker admitted the request (device block taken) */
    double t_done;          /* the worker saw the request's work complete */
    size_t device_bytes;    /* size of the request's device block */
} cbct_request_info;

typedef struct {
    long long submitted, completed, failed;
    int queued, active, max_active_seen;
    size_t bytes_in_use, max_bytes_seen, budget_bytes, l2_budget_bytes;
    long long bypassed;      /* admissions that overtook an earlier queued request */
} cbct_server_stats;

/*
 * Creates a server on the current CUDA device (opts NULL = defaults: 150 GB budget,
 * 16 slots, graphs on) and starts its worker thread. Errors: INVALID_ARG, CUDA.
 */
cbct_status cbct_server_create(const cbct_server_opts *opts, cbct_server **out);

/*
 * Queues a reconstruction (arguments and result as cbct_reconstruct_ex, with host
 * buffers): y_host [n_views][nv][nu] and f_host [nz][ny][nx] must be page-locked host
 * memory (cudaHostAlloc / cudaHostRegister) that stays valid and untouched until the
 * request is done. desc->angles is copied. Returns at once with the request's id.
 * Errors (nothing is queued): INVALID_ARG for bad arguments, pageable host buffers, or a
 * request whose device block exceeds the whole budget; UNSUPPORTED as cbct_reconstruct.
 */
cbct_status cbct_server_submit(cbct_server *srv, const cbct_geometry_desc *desc, const float *y_host,
                               float mu, float lambda, int levels, const int *iters,
                               const cbct_recon_opts *opts, float *f_host, long long *id);

/*
 * Waits up to timeout_s seconds (< 0: without limit) for request `id`; fills info (may be
 * NULL). Returns the request's own status once it is done (OUT_OF_MEMORY, CUDA or
 * NONFINITE for a failed request, with the message in cbct_last_error), TIMEOUT if it is
 * still queued or running, INVALID_ARG for an unknown id.
 */
cbct_status cbct_server_wait(cbct_server *srv, long long id, double timeout_s, cbct_request_info *info);

/* Counters of the server (a snapshot). */
cbct_status cbct_server_stats_get(cbct_server *srv, cbct_server_stats *stats);

/* Finishes every queued and admitted request, stops the worker and frees the server. */
cbct_status cbct_server_destroy(cbct_server *srv);

/*
 * Column groups of the projector (tuning and testing; not part of the paper's method).
 * Along each ray's transverse trace (Section 2.2.1's Siddon walk) the projector stages the
 * voxel columns in groups of 16, 24, 32, 40, 48, 56, 64, 80 or 96 and, by default, picks
 * the size per launch from an estimate of its per-group cost and of the blocks it keeps
 * resident per SM. Results of different group sizes agree to FP32 rounding (the sums are
 * associated differently).
 *
 * cbct_set_project_group: process-wide; 0 restores the automatic choice, one of the sizes
 * above forces it for every launch whose shared memory it fits (larger grids keep the
 * automatic choice). Any other value returns CBCT_ERR_INVALID_ARG and changes nothing.
 * cbct_project_group: the group size an FP32 projection of multigrid level `level` of `g`
 * uses on the current device, in *segments.
 */
cbct_status cbct_set_project_group(int segments);
cbct_status cbct_project_group(const cbct_geometry *g, int level, int *segments);

/* Kernel families reported by cbct_kernel_time. */
typedef enum {
    CBCT_KERNEL_PROJECT = 0,     /* the projector P */
    CBCT_KERNEL_BACKPROJECT = 1, /* the adjoint P^T */
    CBCT_KERNEL_TF_ANALYZE = 2,  /* W */
    CBCT_KERNEL_TF_SYNTH = 3,    /* T_mu, W^T, H */
    CBCT_KERNEL_OTHER = 4,       /* vector updates, reductions, transfers, layout changes */
    CBCT_KERNEL_KINDS = 5
} cbct_kernel_kind;

/*
 * Measurement support (not part of the paper's method). While enabled, every kernel the
 * library launches is bracketed by two CUDA events recorded on the launching stream;
 * cbct_kernel_time waits for the recorded events and returns, per family, the summed
 * device time and the number of launches since the last reset. Process-wide; enabling
 * adds two event records per launch.
 */
cbct_status cbct_profiling_enable(int enable);
/* As cbct_profiling_enable, timing only the kinds whose bit (1 << kind) is set in `kinds`
 * (0 stops timing); untimed launches pay nothing. Events are pooled and reused. */
cbct_status cbct_profiling_select(unsigned int kinds);
cbct_status cbct_profiling_reset(void);
cbct_status cbct_kernel_time(int kind, double *total_ms, unsigned long long *launches);

/* Message describing the last error on the calling thread ("" if none). */
const char *cbct_last_error(void);

/* Number of kernels this library has launched in this process (all threads). */
unsigned long long cbct_launch_count(void);

/* Library version string. */
const char *cbct_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CBCTTF_H */
