/*
 * FP64 CPU oracle for tight-frame regularised cone-beam CT reconstruction
 * (Jia, Dong, Lou, Jiang: "GPU-based iterative cone beam CT reconstruction using tight
 * frame regularization").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the CUDA
 * library is checked against. It shares no code, header, table or helper with the
 * CUDA library, and the library never calls it. Everything is double precision.
 *
 * Layouts: volume f[iz][iy][ix] (x fastest); projections g[k][iv][iu] (u fastest);
 * frame coefficients alpha[i][iz][iy][ix], channel i = l + 3m + 9n where filter l acts
 * along x, m along y, n along z.
 *
 * Geometry (Section 2.1, Fig. 1, and the set-up of Section 3): circular source orbit of
 * radius sad about the z axis, flat imager at distance sdd from the source.
 *   view k, angle t: source S = sad (cos t, sin t, 0); imager centre
 *   C = -(sdd - sad)(cos t, sin t, 0); imager axes e_u = (-sin t, cos t, 0), e_v = z.
 *   pixel (iu, iv) centre D = C + u e_u + v e_v, u = u_off + (iu - (nu-1)/2) du, same for v.
 *   voxel (ix, iy, iz) = half-open box [x0 + ix dx, x0 + (ix+1) dx) x ..., x0 = -nx dx / 2.
 * One ray per pixel centre; the projection of Eq. (1) along that ray is the sum over
 * voxels of (voxel value) x (length of the segment S->D inside the voxel).
 *
 * Parity status per function is stated in each header comment.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    int nx, ny, nz;
    double dx, dy, dz;
    int nu, nv;
    double du, dv, u_off, v_off;
    double sad, sdd;
    int n_views;
    const double *angles; /* n_views angles in radians */
} og_geom;

/* ------------------------------------------------------------------------------------ */
/* Geometry                                                                              */
/* ------------------------------------------------------------------------------------ */

/* Source position, imager centre and imager axes of view k (Section 2.1, Fig. 1). */
static void view_frame(const og_geom *g, int k, double S[3], double C[3], double eu[3],
                       double ev[3])
{
    double c = cos(g->angles[k]), s = sin(g->angles[k]);
    S[0] = g->sad * c;  S[1] = g->sad * s;  S[2] = 0.0;
    C[0] = -(g->sdd - g->sad) * c;  C[1] = -(g->sdd - g->sad) * s;  C[2] = 0.0;
    eu[0] = -s;  eu[1] = c;  eu[2] = 0.0;
    ev[0] = 0.0; ev[1] = 0.0; ev[2] = 1.0;
}

static double pixel_u(const og_geom *g, int iu) { return g->u_off + (iu - 0.5 * (g->nu - 1)) * g->du; }
static double pixel_v(const og_geom *g, int iv) { return g->v_off + (iv - 0.5 * (g->nv - 1)) * g->dv; }

/* Centre of pixel (iu, iv) of view k. */
static void pixel_centre(const og_geom *g, int k, int iu, int iv, double D[3])
{
    double S[3], C[3], eu[3], ev[3];
    view_frame(g, k, S, C, eu, ev);
    double u = pixel_u(g, iu), v = pixel_v(g, iv);
    for (int a = 0; a < 3; a++) D[a] = C[a] + u * eu[a] + v * ev[a];
}

static void grid_arrays(const og_geom *g, int n[3], double h[3], double o[3])
{
    n[0] = g->nx; n[1] = g->ny; n[2] = g->nz;
    h[0] = g->dx; h[1] = g->dy; h[2] = g->dz;
    for (int a = 0; a < 3; a++) o[a] = -0.5 * n[a] * h[a];
}

/* ------------------------------------------------------------------------------------ */
/* Siddon ray tracing (Section 2.2.1)                                                    */
/* ------------------------------------------------------------------------------------ */

/*
 * Siddon's exact ray tracing. The ray is S + a (D - S), a in [0, 1]. The crossings of
 * the ray with the three families of voxel planes, restricted to the part of the ray
 * inside the volume box, are merged into one increasing sequence; every gap between two
 * consecutive crossings is a segment lying in a single voxel, identified from the
 * gap's midpoint, and its length is (gap) x |D - S|.
 * Writes up to cap (voxel index, length) pairs; returns the number of segments with
 * positive length. scratch must hold nx + ny + nz + 3 doubles.
 * Pinned by: the brute-force slab-clipping system matrix, the chord of a uniform box,
 * the analytic chord of an ellipsoid (tests).
 */
static long trace_ray(const og_geom *g, const double S[3], const double D[3], long *vox,
                      double *len, long cap, double *scratch)
{
    int n[3];
    double h[3], o[3], d[3];
    grid_arrays(g, n, h, o);
    for (int a = 0; a < 3; a++) d[a] = D[a] - S[a];
    double L = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);

    /* part of the ray inside the volume box */
    double amin = 0.0, amax = 1.0;
    for (int a = 0; a < 3; a++) {
        if (d[a] != 0.0) {
            double a0 = (o[a] - S[a]) / d[a];
            double a1 = (o[a] + n[a] * h[a] - S[a]) / d[a];
            amin = fmax(amin, fmin(a0, a1));
            amax = fmin(amax, fmax(a0, a1));
        } else if (S[a] < o[a] || S[a] >= o[a] + n[a] * h[a]) {
            return 0;
        }
    }
    if (!(amax > amin)) return 0;

    /* crossings of each plane family strictly inside (amin, amax), in increasing order */
    double *list[3];
    int cnt[3];
    list[0] = scratch;
    list[1] = list[0] + (n[0] + 1);
    list[2] = list[1] + (n[1] + 1);
    for (int a = 0; a < 3; a++) {
        cnt[a] = 0;
        if (d[a] == 0.0) continue;
        for (int i = 0; i <= n[a]; i++) {
            int ii = d[a] > 0.0 ? i : n[a] - i; /* walk the planes in the ray's direction */
            double al = (o[a] + ii * h[a] - S[a]) / d[a];
            if (al > amin && al < amax) list[a][cnt[a]++] = al;
        }
    }

    /* three-way merge; each gap is one voxel segment */
    int head[3] = {0, 0, 0};
    double prev = amin;
    long m = 0;
    for (;;) {
        int best = -1;
        double next = amax;
        for (int a = 0; a < 3; a++)
            if (head[a] < cnt[a] && list[a][head[a]] < next) { next = list[a][head[a]]; best = a; }
        if (next > prev) {
            double mid = 0.5 * (prev + next);
            int idx[3];
            for (int a = 0; a < 3; a++) {
                double p = S[a] + mid * d[a];
                int i = (int)floor((p - o[a]) / h[a]);
                if (i < 0) i = 0;
                if (i > n[a] - 1) i = n[a] - 1;
                idx[a] = i;
            }
            if (m < cap) {
                vox[m] = ((long)idx[2] * n[1] + idx[1]) * n[0] + idx[0];
                len[m] = (next - prev) * L;
            }
            m++;
            prev = next;
        }
        if (best < 0) break;
        head[best]++;
    }
    return m;
}

static long trace_capacity(const og_geom *g) { return (long)g->nx + g->ny + g->nz + 4; }

/* Trace of one ray for inspection from Python: returns the segment count. */
long o_trace(const og_geom *g, int k, int iu, int iv, long *vox, double *len, long cap)
{
    double S[3], C[3], eu[3], ev[3], D[3];
    view_frame(g, k, S, C, eu, ev);
    pixel_centre(g, k, iu, iv, D);
    double *scratch = (double *)malloc(sizeof(double) * trace_capacity(g));
    long m = trace_ray(g, S, D, vox, len, cap, scratch);
    free(scratch);
    return m;
}

/*
 * Forward projection P (Eq. (1) discretised with Siddon's method, Section 2.2.1):
 * g_i = sum_j a_ij f_j, a_ij = length of ray i inside voxel j.
 */
void o_project(const og_geom *g, const double *f, double *out)
{
    long nrays = (long)g->n_views * g->nv * g->nu;
    long cap = trace_capacity(g);
#pragma omp parallel
    {
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *scratch = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; r++) {
            int k = (int)(r / ((long)g->nv * g->nu));
            int iv = (int)((r / g->nu) % g->nv);
            int iu = (int)(r % g->nu);
            double S[3], C[3], eu[3], ev[3], D[3];
            view_frame(g, k, S, C, eu, ev);
            pixel_centre(g, k, iu, iv, D);
            long m = trace_ray(g, S, D, vox, len, cap, scratch);
            double acc = 0.0;
            for (long s = 0; s < m; s++) acc += f[vox[s]] * len[s];
            out[r] = acc;
        }
        free(vox); free(len); free(scratch);
    }
}

/* Forward projection of selected rays only (ray index r = (k*nv + iv)*nu + iu). */
void o_project_rays(const og_geom *g, const double *f, long nsel, const long *rays, double *out)
{
    long cap = trace_capacity(g);
#pragma omp parallel
    {
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *scratch = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 16)
        for (long q = 0; q < nsel; q++) {
            long r = rays[q];
            int k = (int)(r / ((long)g->nv * g->nu));
            int iv = (int)((r / g->nu) % g->nv);
            int iu = (int)(r % g->nu);
            double S[3], C[3], eu[3], ev[3], D[3];
            view_frame(g, k, S, C, eu, ev);
            pixel_centre(g, k, iu, iv, D);
            long m = trace_ray(g, S, D, vox, len, cap, scratch);
            double acc = 0.0;
            for (long s = 0; s < m; s++) acc += f[vox[s]] * len[s];
            out[q] = acc;
        }
        free(vox); free(len); free(scratch);
    }
}

/*
 * Exact adjoint P^T: (P^T g)_j = sum_i a_ij g_i with the very same Siddon weights, so
 * <P f, g> = <f, P^T g> (Eq. (A1)) holds to rounding. Views are split over threads,
 * each scattering into a private volume; the private volumes are summed in thread order.
 */
void o_backproject(const og_geom *g, const double *gin, double *f)
{
    long N = (long)g->nx * g->ny * g->nz;
    long cap = trace_capacity(g);
    int T = 1;
#ifdef _OPENMP
    T = omp_get_max_threads();
#endif
    long maxT = (long)(2.0e9 / (8.0 * (double)N));
    if (maxT < 1) maxT = 1;
    if (T > maxT) T = (int)maxT;
    if (T > g->n_views) T = g->n_views > 0 ? g->n_views : 1;
    double **priv = (double **)malloc(sizeof(double *) * T);
    for (int t = 0; t < T; t++) priv[t] = (double *)calloc((size_t)N, sizeof(double));
#pragma omp parallel num_threads(T)
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double *acc = priv[tid];
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *scratch = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(static)
        for (int k = 0; k < g->n_views; k++) {
            double S[3], C[3], eu[3], ev[3], D[3];
            view_frame(g, k, S, C, eu, ev);
            for (int iv = 0; iv < g->nv; iv++)
                for (int iu = 0; iu < g->nu; iu++) {
                    double gi = gin[((long)k * g->nv + iv) * g->nu + iu];
                    pixel_centre(g, k, iu, iv, D);
                    long m = trace_ray(g, S, D, vox, len, cap, scratch);
                    for (long s = 0; s < m; s++) acc[vox[s]] += len[s] * gi;
                }
        }
        free(vox); free(len); free(scratch);
    }
    for (long j = 0; j < N; j++) {
        double s = 0.0;
        for (int t = 0; t < T; t++) s += priv[t][j];
        f[j] = s;
    }
    for (int t = 0; t < T; t++) free(priv[t]);
    free(priv);
}

/* Number of (ray, voxel) pairs whose segment is longer than 1e-9 of the smallest voxel
 * side: the non-zeros of P (rounding slivers where a ray passes a voxel edge exactly are
 * not counted). */
long long o_count_nnz(const og_geom *g)
{
    long nrays = (long)g->n_views * g->nv * g->nu;
    long cap = trace_capacity(g);
    long long total = 0;
    double eps = 1e-9 * fmin(g->dx, fmin(g->dy, g->dz));
#pragma omp parallel reduction(+ : total)
    {
        long *vox = (long *)malloc(sizeof(long) * cap);
        double *len = (double *)malloc(sizeof(double) * cap);
        double *scratch = (double *)malloc(sizeof(double) * cap);
#pragma omp for schedule(dynamic, 64)
        for (long r = 0; r < nrays; r++) {
            int k = (int)(r / ((long)g->nv * g->nu));
            int iv = (int)((r / g->nu) % g->nv);
            int iu = (int)(r % g->nu);
            double S[3], C[3], eu[3], ev[3], D[3];
            view_frame(g, k, S, C, eu, ev);
            pixel_centre(g, k, iu, iv, D);
            long m = trace_ray(g, S, D, vox, len, cap, scratch);
            for (long q = 0; q < m; q++) total += len[q] > eps;
        }
        free(vox); free(len); free(scratch);
    }
    return total;
}

/* ------------------------------------------------------------------------------------ */
/* Slab clipping: an independent definition of a_ij                                      */
/* ------------------------------------------------------------------------------------ */

/* Length of the segment S->D inside the half-open box [lo, hi) (slab method). */
static double ray_box_length(const double S[3], const double D[3], const double lo[3],
                             const double hi[3])
{
    double amin = 0.0, amax = 1.0, d[3];
    for (int a = 0; a < 3; a++) d[a] = D[a] - S[a];
    for (int a = 0; a < 3; a++) {
        if (d[a] != 0.0) {
            double a0 = (lo[a] - S[a]) / d[a], a1 = (hi[a] - S[a]) / d[a];
            amin = fmax(amin, fmin(a0, a1));
            amax = fmin(amax, fmax(a0, a1));
        } else if (S[a] < lo[a] || S[a] >= hi[a]) {
            return 0.0;
        }
    }
    if (!(amax > amin)) return 0.0;
    return (amax - amin) * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
}

/* Continuous pixel coordinates (iu, iv) where the ray from S through p meets the imager. */
static void project_point(const og_geom *g, int k, const double p[3], double *fu, double *fv)
{
    double S[3], C[3], eu[3], ev[3];
    view_frame(g, k, S, C, eu, ev);
    double nrm[3], w = 0.0;
    for (int a = 0; a < 3; a++) nrm[a] = (C[a] - S[a]) / g->sdd;
    for (int a = 0; a < 3; a++) w += (p[a] - S[a]) * nrm[a];
    double lam = g->sdd / w, u = 0.0, v = 0.0;
    for (int a = 0; a < 3; a++) {
        double hit = S[a] + lam * (p[a] - S[a]);
        u += (hit - C[a]) * eu[a];
        v += (hit - C[a]) * ev[a];
    }
    *fu = (u - g->u_off) / g->du + 0.5 * (g->nu - 1);
    *fv = (v - g->v_off) / g->dv + 0.5 * (g->nv - 1);
}

/*
 * P^T at selected voxels, by brute force: for each view, every pixel whose centre lies
 * in the bounding box (widened by one pixel) of the voxel's projected corners is a
 * candidate, and its weight is the slab-clipped length of its ray inside the voxel.
 * Independent of the Siddon trace; used for sampled checks at full size.
 */
void o_backproject_voxels(const og_geom *g, const double *gin, long nsel, const long *voxels,
                          double *out)
{
    int n[3];
    double h[3], o[3];
    grid_arrays(g, n, h, o);
#pragma omp parallel for schedule(dynamic, 4)
    for (long q = 0; q < nsel; q++) {
        long j = voxels[q];
        int ix = (int)(j % n[0]), iy = (int)((j / n[0]) % n[1]), iz = (int)(j / ((long)n[0] * n[1]));
        double lo[3] = {o[0] + ix * h[0], o[1] + iy * h[1], o[2] + iz * h[2]};
        double hi[3] = {lo[0] + h[0], lo[1] + h[1], lo[2] + h[2]};
        double acc = 0.0;
        for (int k = 0; k < g->n_views; k++) {
            double S[3], C[3], eu[3], ev[3], D[3];
            view_frame(g, k, S, C, eu, ev);
            double umin = 1e300, umax = -1e300, vmin = 1e300, vmax = -1e300;
            for (int c = 0; c < 8; c++) {
                double p[3] = {(c & 1) ? hi[0] : lo[0], (c & 2) ? hi[1] : lo[1], (c & 4) ? hi[2] : lo[2]};
                double fu, fv;
                project_point(g, k, p, &fu, &fv);
                umin = fmin(umin, fu); umax = fmax(umax, fu);
                vmin = fmin(vmin, fv); vmax = fmax(vmax, fv);
            }
            int u0 = (int)floor(umin) - 1, u1 = (int)ceil(umax) + 1;
            int v0 = (int)floor(vmin) - 1, v1 = (int)ceil(vmax) + 1;
            if (u0 < 0) u0 = 0;
            if (v0 < 0) v0 = 0;
            if (u1 > g->nu - 1) u1 = g->nu - 1;
            if (v1 > g->nv - 1) v1 = g->nv - 1;
            for (int iv = v0; iv <= v1; iv++)
                for (int iu = u0; iu <= u1; iu++) {
                    pixel_centre(g, k, iu, iv, D);
                    double a = ray_box_length(S, D, lo, hi);
                    if (a > 0.0) acc += a * gin[((long)k * g->nv + iv) * g->nu + iu];
                }
        }
        out[q] = acc;
    }
}

/* Slab-clipped length of ray (k, iu, iv) in the box [lo, hi) — exposed for tests. */
double o_ray_box_length(const og_geom *g, int k, int iu, int iv, const double lo[3],
                        const double hi[3])
{
    double S[3], C[3], eu[3], ev[3], D[3];
    view_frame(g, k, S, C, eu, ev);
    pixel_centre(g, k, iu, iv, D);
    return ray_box_length(S, D, lo, hi);
}

/*
 * The paper's own backprojector, Eq. (3): voxel-driven, for every view the imager value
 * at the point u* where the ray through the voxel centre x meets the imager is taken by
 * bilinear interpolation (zero outside the imager) and weighted by
 * (dx dy dz / (du dv)) L^3(u*) / (L0 l^2(x)), L0 = sdd, l = |x - S|, L = |u* - S|.
 * It approximates the exact adjoint (Appendix 2); pinned against the exact P^T in the
 * limit of many rays per voxel (tests).
 */
void o_backproject_eq3(const og_geom *g, const double *gin, double *f)
{
    int n[3];
    double h[3], o[3];
    grid_arrays(g, n, h, o);
    double pref = g->dx * g->dy * g->dz / (g->du * g->dv);
    long N = (long)n[0] * n[1] * n[2];
#pragma omp parallel for schedule(static)
    for (long j = 0; j < N; j++) {
        int ix = (int)(j % n[0]), iy = (int)((j / n[0]) % n[1]), iz = (int)(j / ((long)n[0] * n[1]));
        double x[3] = {o[0] + (ix + 0.5) * h[0], o[1] + (iy + 0.5) * h[1], o[2] + (iz + 0.5) * h[2]};
        double acc = 0.0;
        for (int k = 0; k < g->n_views; k++) {
            double S[3], C[3], eu[3], ev[3];
            view_frame(g, k, S, C, eu, ev);
            double fu, fv;
            project_point(g, k, x, &fu, &fv);
            double l2 = 0.0, w = 0.0;
            for (int a = 0; a < 3; a++) {
                l2 += (x[a] - S[a]) * (x[a] - S[a]);
                w += (x[a] - S[a]) * (C[a] - S[a]) / g->sdd;
            }
            double l = sqrt(l2);
            double L = l * g->sdd / w; /* distance from S to u* along the same ray */
            int i0 = (int)floor(fu), j0 = (int)floor(fv);
            double wu = fu - i0, wv = fv - j0, val = 0.0;
            for (int b = 0; b < 2; b++)
                for (int a = 0; a < 2; a++) {
                    int iu = i0 + a, iv = j0 + b;
                    if (iu < 0 || iu >= g->nu || iv < 0 || iv >= g->nv) continue;
                    double wt = (a ? wu : 1.0 - wu) * (b ? wv : 1.0 - wv);
                    val += wt * gin[((long)k * g->nv + iv) * g->nu + iu];
                }
            acc += pref * L * L * L / (g->sdd * l2) * val;
        }
        f[j] = acc;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Piecewise-linear tight frame (Section 2.1)                                            */
/* ------------------------------------------------------------------------------------ */

/* 1-D filters h0 = [1,2,1]/4, h1 = sqrt(2)/4 [1,0,-1], h2 = [-1,2,-1]/4; column t holds
 * the tap at offset t - 1, i.e. the printed order h[-1], h[0], h[1]. */
static void tf_taps(double H[3][3])
{
    double r = sqrt(2.0) / 4.0;
    H[0][0] = 0.25;  H[0][1] = 0.5; H[0][2] = 0.25;
    H[1][0] = r;     H[1][1] = 0.0; H[1][2] = -r;
    H[2][0] = -0.25; H[2][1] = 0.5; H[2][2] = -0.25;
}

static inline int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/*
 * Analysis W (the paper's D): alpha_i(x) = (psi_i conv f)(x) = sum_k psi_i(k) f(x - k),
 * psi_i(k) = h_l(k_x) h_m(k_y) h_n(k_z), i = l + 3m + 9n, k in {-1,0,1}^3. The paper does
 * not fix the boundary; the volume is taken as periodic, for which W^T W = I exactly.
 * Pinned by: W^T W = I, Parseval, constant and impulse responses against the printed
 * filter taps, the ramp slope of h1 (tests).
 */
void o_tf_analyze(int nx, int ny, int nz, const double *f, double *alpha)
{
    double H[3][3];
    tf_taps(H);
    long N = (long)nx * ny * nz;
#pragma omp parallel for collapse(2) schedule(static)
    for (int i = 0; i < 27; i++)
        for (int z = 0; z < nz; z++) {
            int l = i % 3, m = (i / 3) % 3, nn = i / 9;
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    double acc = 0.0;
                    for (int c = -1; c <= 1; c++)
                        for (int b = -1; b <= 1; b++)
                            for (int a = -1; a <= 1; a++) {
                                double w = H[l][a + 1] * H[m][b + 1] * H[nn][c + 1];
                                acc += w * f[((long)wrap(z - c, nz) * ny + wrap(y - b, ny)) * nx + wrap(x - a, nx)];
                            }
                    alpha[i * N + ((long)z * ny + y) * nx + x] = acc;
                }
        }
}

/*
 * Synthesis W^T (the paper's D^T): f(x) = sum_i (psi_i(-.) conv alpha_i)(x)
 *   = sum_i sum_k psi_i(k) alpha_i(x + k), periodic, the exact transpose of o_tf_analyze.
 */
void o_tf_synthesize(int nx, int ny, int nz, const double *alpha, double *f)
{
    double H[3][3];
    tf_taps(H);
    long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                double acc = 0.0;
                for (int i = 0; i < 27; i++) {
                    int l = i % 3, m = (i / 3) % 3, nn = i / 9;
                    for (int c = -1; c <= 1; c++)
                        for (int b = -1; b <= 1; b++)
                            for (int a = -1; a <= 1; a++) {
                                double w = H[l][a + 1] * H[m][b + 1] * H[nn][c + 1];
                                acc += w * alpha[i * N + ((long)wrap(z + c, nz) * ny + wrap(y + b, ny)) * nx + wrap(x + a, nx)];
                            }
                }
                f[((long)z * ny + y) * nx + x] = acc;
            }
}

/*
 * Vector shrinkage T_mu, Eq. (2), voxel-wise and in place: alpha_0 is kept; the 26
 * high-pass coefficients are multiplied by max(1 - mu / ||alpha_h||, 0), where
 * ||alpha_h|| is their l2 norm at that voxel (a zero norm gives factor 0).
 */
void o_tf_shrink(int nx, int ny, int nz, double *alpha, double mu)
{
    long N = (long)nx * ny * nz;
#pragma omp parallel for schedule(static)
    for (long j = 0; j < N; j++) {
        double s2 = 0.0;
        for (int i = 1; i < 27; i++) s2 += alpha[i * N + j] * alpha[i * N + j];
        double nrm = sqrt(s2);
        double scale = nrm > mu ? 1.0 - mu / nrm : 0.0;
        for (int i = 1; i < 27; i++) alpha[i * N + j] *= scale;
    }
}

/*
 * The regularisation step H(W^T T_mu W f) at selected voxels only (flat index
 * (z*ny + y)*nx + x), from the same three definitions as o_tf_analyze, o_tf_shrink and
 * o_tf_synthesize: the output at x needs the shrunk coefficients at x + k for k in
 * {-1,0,1}^3, each of which needs f on its own 3x3x3 neighbourhood (periodic). For sampled
 * checks at full size. Pinned by: equality with the three whole-volume steps (tests).
 */
void o_tf_shrink_voxels(int nx, int ny, int nz, const double *f, double mu, int positivity, long nsel,
                        const long *vox, double *out)
{
    double H[3][3];
    tf_taps(H);
#pragma omp parallel for schedule(dynamic, 16)
    for (long s = 0; s < nsel; s++) {
        const long j = vox[s];
        const int x = (int)(j % nx), y = (int)((j / nx) % ny), z = (int)(j / ((long)nx * ny));
        double acc = 0.0;
        for (int c = -1; c <= 1; c++)
            for (int b = -1; b <= 1; b++)
                for (int a = -1; a <= 1; a++) {
                    /* coefficients at p = x + (a, b, c) */
                    const int px = wrap(x + a, nx), py = wrap(y + b, ny), pz = wrap(z + c, nz);
                    double al[27];
                    for (int i = 0; i < 27; i++) {
                        int l = i % 3, m = (i / 3) % 3, nn = i / 9;
                        double t = 0.0;
                        for (int cc = -1; cc <= 1; cc++)
                            for (int bb = -1; bb <= 1; bb++)
                                for (int aa = -1; aa <= 1; aa++)
                                    t += H[l][aa + 1] * H[m][bb + 1] * H[nn][cc + 1] *
                                         f[((long)wrap(pz - cc, nz) * ny + wrap(py - bb, ny)) * nx + wrap(px - aa, nx)];
                        al[i] = t;
                    }
                    double s2 = 0.0;
                    for (int i = 1; i < 27; i++) s2 += al[i] * al[i];
                    const double nrm = sqrt(s2);
                    const double scale = nrm > mu ? 1.0 - mu / nrm : 0.0;
                    for (int i = 1; i < 27; i++) al[i] *= scale;
                    /* synthesis: psi_i(k) alpha_i(x + k) with k = (a, b, c) */
                    for (int i = 0; i < 27; i++) {
                        int l = i % 3, m = (i / 3) % 3, nn = i / 9;
                        acc += H[l][a + 1] * H[m][b + 1] * H[nn][c + 1] * al[i];
                    }
                }
        out[s] = (positivity && acc < 0.0) ? 0.0 : acc;
    }
}

/* Positivity correction H (Section 2.1): negative voxels set to zero (NaN passes). */
void o_positivity(long n, double *f)
{
    for (long j = 0; j < n; j++)
        if (f[j] < 0.0) f[j] = 0.0;
}

/* ------------------------------------------------------------------------------------ */
/* CGLS (Appendix 1), Algorithm A2 (Section 2.1), multigrid (Section 2.2.3)             */
/* ------------------------------------------------------------------------------------ */

static double dot(long n, const double *a, const double *b)
{
    double s = 0.0;
    for (long i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/*
 * Rounding to a 16-bit storage format, round to nearest with ties to even, written from
 * the formats' definitions. storage 1 = bfloat16 (8 significand bits, the exponent range
 * of binary32: smallest normal 2^-126, largest finite (2 - 2^-7) 2^127); storage 2 = IEEE
 * binary16 (11 significand bits, smallest normal 2^-14, largest finite 65504); below the
 * smallest normal the spacing is fixed (subnormals). Values beyond the largest finite
 * number by half a spacing or more become infinite. storage 0 returns x unchanged.
 * Pinned by: brute-force nearest-even search over all 2^16 codes of each format, and
 * numpy's binary16 conversion (tests).
 */
static double round_storage(double x, int storage)
{
    if (storage == 0 || x == 0.0 || !isfinite(x)) return x;
    const int p = storage == 1 ? 8 : 11;          /* significand bits */
    const int emin = storage == 1 ? -126 : -14;   /* exponent of the smallest normal */
    const double maxv = storage == 1 ? ldexp(2.0 - ldexp(1.0, -7), 127) : 65504.0;
    int e;
    frexp(x, &e);                /* 2^(e-1) <= |x| < 2^e */
    int q = (e - 1) - (p - 1);   /* exponent of the spacing at |x| */
    if (e - 1 < emin) q = emin - (p - 1);
    double r = ldexp(nearbyint(ldexp(x, -q)), q); /* default mode: nearest, ties to even */
    if (fabs(r) > maxv) return copysign(INFINITY, x);
    return r;
}

void o_round_storage(long n, double *x, int storage)
{
    for (long i = 0; i < n; i++) x[i] = round_storage(x[i], storage);
}

/*
 * CGLS for min ||P x - y||^2 (Appendix 1) from the initial guess in x:
 *   r = y - P x, p = s = P^T r, gamma = ||s||^2; then n_iter times:
 *   q = P p, alpha = gamma / ||q||^2, x += alpha p, r -= alpha q, s = P^T r,
 *   gamma' = ||s||^2, beta = gamma' / gamma, p = s + beta p, gamma = gamma'.
 * The listing's loop l = 0..M performs M+1 such updates; n_iter counts updates. If
 * gamma or ||q||^2 is zero the current x is stationary and the loop stops.
 * resid (optional, n_iter+1 entries) receives ||r||^2 before and after every update.
 * Pinned by: the exact Krylov-subspace least-squares minimiser on small dense systems,
 * monotone residual (tests).
 *
 * storage != 0 is the reduced-precision variant (no counterpart in the paper): the
 * projection-domain vectors r and q are held in a 16-bit format (round_storage) and all
 * else is unchanged. r is rounded where it is formed and after every update; q is
 * rounded after ||q||^2 is taken from the unrounded values. For binary16 q is held as
 * kappa q with kappa = 1 / sqrt(gamma) (keeps it in range) and the update reads
 * r -= (alpha / kappa) (kappa q). Pinned by: a dense-matrix restatement that rounds
 * through a brute-force nearest-even search (tests).
 */
static void cgls_impl(const og_geom *g, const double *y, double *x, int n_iter, double *resid, int storage)
{
    long N = (long)g->nx * g->ny * g->nz, M = (long)g->n_views * g->nv * g->nu;
    double *r = (double *)malloc(sizeof(double) * M), *q = (double *)malloc(sizeof(double) * M);
    double *s = (double *)malloc(sizeof(double) * N), *p = (double *)malloc(sizeof(double) * N);
    o_project(g, x, r);
    for (long i = 0; i < M; i++) r[i] = round_storage(y[i] - r[i], storage);
    o_backproject(g, r, s);
    memcpy(p, s, sizeof(double) * N);
    double gamma = dot(N, s, s);
    if (resid) {
        for (int l = 0; l <= n_iter; l++) resid[l] = NAN;
        resid[0] = dot(M, r, r);
    }
    for (int l = 0; l < n_iter; l++) {
        o_project(g, p, q);
        double delta = dot(M, q, q);
        if (gamma == 0.0 || delta == 0.0) {
            if (resid)
                for (int t = l + 1; t <= n_iter; t++) resid[t] = resid[l];
            break;
        }
        double alpha = gamma / delta;
        for (long j = 0; j < N; j++) x[j] += alpha * p[j];
        if (storage == 0) {
            for (long i = 0; i < M; i++) r[i] -= alpha * q[i];
        } else {
            const double kappa = storage == 2 ? 1.0 / sqrt(gamma) : 1.0;
            for (long i = 0; i < M; i++) {
                const double qs = round_storage(kappa * q[i], storage);
                r[i] = round_storage(r[i] - (alpha / kappa) * qs, storage);
            }
        }
        if (resid) resid[l + 1] = dot(M, r, r);
        o_backproject(g, r, s);
        double gnew = dot(N, s, s);
        double beta = gnew / gamma;
        for (long j = 0; j < N; j++) p[j] = s[j] + beta * p[j];
        gamma = gnew;
    }
    free(r); free(q); free(s); free(p);
}

void o_cgls(const og_geom *g, const double *y, double *x, int n_iter, double *resid)
{
    cgls_impl(g, y, x, n_iter, resid, 0);
}

void o_cgls_storage(const og_geom *g, const double *y, double *x, int n_iter, double *resid, int storage)
{
    cgls_impl(g, y, x, n_iter, resid, storage);
}

/*
 * Algorithm A2 (Section 2.1) on one grid, n_outer iterations. f holds f^(0) on entry
 * (f^(-1) = f^(0), t^(0) = t^(-1) = 1) and f^(n_outer) on exit:
 *   v = f^(k) + (t^(k-1) - 1) / t^(k) (f^(k) - f^(k-1));   [momentum = 0: v = f^(k), i.e. A1]
 *   f^(k+1) = CGLS[v];  f^(k+1) <- D^T T_mu D f^(k+1);  f^(k+1) <- H f^(k+1)  [if positivity];
 *   t^(k+1) = (1 + sqrt(1 + 4 t^(k)^2)) / 2.
 * storage selects the CGLS variant above. coef (optional, n_outer entries) receives the
 * momentum coefficient each iteration applied.
 * Pinned by: the coefficients against hand-evaluated values of the recurrence; with the
 * data step removed (n_cgls = 0, H off) the iterates against the momentum-accelerated
 * shrinkage sequence built from those values; mu = 0 reaches the least-squares solution
 * with and without momentum; a consistent positive constant is a fixed point; momentum
 * converges faster than A1; an independent dense-matrix restatement (tests).
 */
static void a2_impl(const og_geom *g, const double *y, double mu, int n_outer, int n_cgls, int positivity,
                    int momentum, int storage, double *f, double *coef)
{
    long N = (long)g->nx * g->ny * g->nz;
    double *fprev = (double *)malloc(sizeof(double) * N);
    double *x = (double *)malloc(sizeof(double) * N);
    double *alpha = (double *)malloc(sizeof(double) * 27 * N);
    memcpy(fprev, f, sizeof(double) * N);
    double t_prev = 1.0, t = 1.0;
    for (int k = 0; k < n_outer; k++) {
        double c = momentum ? (t_prev - 1.0) / t : 0.0;
        if (coef) coef[k] = c;
        for (long j = 0; j < N; j++) x[j] = f[j] + c * (f[j] - fprev[j]);
        cgls_impl(g, y, x, n_cgls, NULL, storage);
        o_tf_analyze(g->nx, g->ny, g->nz, x, alpha);
        o_tf_shrink(g->nx, g->ny, g->nz, alpha, mu);
        o_tf_synthesize(g->nx, g->ny, g->nz, alpha, x);
        if (positivity) o_positivity(N, x);
        memcpy(fprev, f, sizeof(double) * N);
        memcpy(f, x, sizeof(double) * N);
        double t_next = 0.5 * (1.0 + sqrt(1.0 + 4.0 * t * t));
        t_prev = t;
        t = t_next;
    }
    free(fprev); free(x); free(alpha);
}

void o_a2(const og_geom *g, const double *y, double mu, int n_outer, int n_cgls, int positivity,
          int momentum, double *f, double *coef)
{
    a2_impl(g, y, mu, n_outer, n_cgls, positivity, momentum, 0, f, coef);
}

/*
 * Prolongation between multigrid levels (Section 2.2.3, "linear interpolation"):
 * trilinear interpolation of the coarse grid at every fine voxel centre, both grids
 * centred on the origin, the coarse coordinate clamped to the hull of coarse voxel
 * centres. Pinned by: exactness on linear functions inside the hull, constants (tests).
 */
void o_prolong(int cnx, int cny, int cnz, double cdx, double cdy, double cdz, const double *fc,
               int nx, int ny, int nz, double dx, double dy, double dz, double *ff)
{
    int cn[3] = {cnx, cny, cnz}, fn[3] = {nx, ny, nz};
    double ch[3] = {cdx, cdy, cdz}, fh[3] = {dx, dy, dz};
#pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int fi[3] = {x, y, z}, i0[3], i1[3];
                double w[3];
                for (int a = 0; a < 3; a++) {
                    double pos = -0.5 * fn[a] * fh[a] + (fi[a] + 0.5) * fh[a];
                    double xi = (pos + 0.5 * cn[a] * ch[a]) / ch[a] - 0.5;
                    if (xi < 0.0) xi = 0.0;
                    if (xi > cn[a] - 1) xi = cn[a] - 1;
                    i0[a] = (int)floor(xi);
                    if (i0[a] > cn[a] - 1) i0[a] = cn[a] - 1;
                    i1[a] = i0[a] + 1 < cn[a] ? i0[a] + 1 : cn[a] - 1;
                    w[a] = xi - i0[a];
                }
                double acc = 0.0;
                for (int c = 0; c < 8; c++) {
                    int jx = (c & 1) ? i1[0] : i0[0], jy = (c & 2) ? i1[1] : i0[1], jz = (c & 4) ? i1[2] : i0[2];
                    double wt = ((c & 1) ? w[0] : 1.0 - w[0]) * ((c & 2) ? w[1] : 1.0 - w[1]) *
                                ((c & 4) ? w[2] : 1.0 - w[2]);
                    acc += wt * fc[((long)jz * cny + jy) * cnx + jx];
                }
                ff[((long)z * ny + y) * nx + x] = acc;
            }
}

/*
 * Restriction (fine -> coarse): each coarse voxel takes the mean of the fine voxels
 * whose centres lie inside it (both grids centred on the origin); a coarse voxel with no
 * such fine voxel is 0. Not used by the cascadic multigrid; kept for tests.
 * Pinned by: constants; a linear function, whose mean over the fine centres inside a
 * coarse voxel is its value at their centroid, on aligned and ragged grids (tests).
 */
void o_restrict(int nx, int ny, int nz, double dx, double dy, double dz, const double *ff,
                int cnx, int cny, int cnz, double cdx, double cdy, double cdz, double *fc)
{
    long CN = (long)cnx * cny * cnz;
    double *cnt = (double *)calloc((size_t)CN, sizeof(double));
    for (long j = 0; j < CN; j++) fc[j] = 0.0;
    int fn[3] = {nx, ny, nz}, cn[3] = {cnx, cny, cnz};
    double fh[3] = {dx, dy, dz}, ch[3] = {cdx, cdy, cdz};
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                int fi[3] = {x, y, z}, ci[3], ok = 1;
                for (int a = 0; a < 3; a++) {
                    double pos = -0.5 * fn[a] * fh[a] + (fi[a] + 0.5) * fh[a];
                    ci[a] = (int)floor((pos + 0.5 * cn[a] * ch[a]) / ch[a]);
                    if (ci[a] < 0 || ci[a] >= cn[a]) ok = 0;
                }
                if (!ok) continue;
                long cj = ((long)ci[2] * cny + ci[1]) * cnx + ci[0];
                fc[cj] += ff[((long)z * ny + y) * nx + x];
                cnt[cj] += 1.0;
            }
    for (long j = 0; j < CN; j++)
        if (cnt[j] > 0.0) fc[j] /= cnt[j];
    free(cnt);
}

/*
 * Multigrid reconstruction (Section 2.2.3): levels grids, level l has ceil(n / 2^l)
 * voxels per axis at 2^l times the spacing, same centre; the imager and y are the same
 * on every level. Start with f = 0 on the coarsest grid, run A2 there, prolong the
 * result as the initial guess of the next finer grid, and so on. iters[] lists the A2
 * iteration counts coarsest first.
 * Pinned by: one level equals A2 on that grid; a second level starts from the prolonged
 * coarse result; prolongation is exact on linear functions; an independent dense-matrix
 * restatement of the whole cascade on small grids (tests).
 */
static void reconstruct_impl(const og_geom *g, const double *y, double mu, int levels, const int *iters,
                             int n_cgls, int positivity, int momentum, int storage, double *f_out)
{
    double *fc = NULL;
    og_geom prev = *g;
    for (int lev = levels - 1; lev >= 0; lev--) {
        og_geom gl = *g;
        int s = 1 << lev;
        gl.nx = (g->nx + s - 1) / s; gl.ny = (g->ny + s - 1) / s; gl.nz = (g->nz + s - 1) / s;
        gl.dx = g->dx * s; gl.dy = g->dy * s; gl.dz = g->dz * s;
        long N = (long)gl.nx * gl.ny * gl.nz;
        double *f = (double *)calloc((size_t)N, sizeof(double));
        if (fc) {
            o_prolong(prev.nx, prev.ny, prev.nz, prev.dx, prev.dy, prev.dz, fc,
                      gl.nx, gl.ny, gl.nz, gl.dx, gl.dy, gl.dz, f);
            free(fc);
        }
        a2_impl(&gl, y, mu, iters[levels - 1 - lev], n_cgls, positivity, momentum, storage, f, NULL);
        fc = f;
        prev = gl;
    }
    memcpy(f_out, fc, sizeof(double) * (long)g->nx * g->ny * g->nz);
    free(fc);
}

void o_reconstruct(const og_geom *g, const double *y, double mu, int levels, const int *iters,
                   int n_cgls, int positivity, int momentum, double *f_out)
{
    reconstruct_impl(g, y, mu, levels, iters, n_cgls, positivity, momentum, 0, f_out);
}

/* o_reconstruct with the reduced-precision CGLS variant (storage 1 = bfloat16, 2 = binary16). */
void o_reconstruct_storage(const og_geom *g, const double *y, double mu, int levels, const int *iters,
                           int n_cgls, int positivity, int momentum, int storage, double *f_out)
{
    reconstruct_impl(g, y, mu, levels, iters, n_cgls, positivity, momentum, storage, f_out);
}

int o_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
