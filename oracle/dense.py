"""Brute-force dense system matrix and dense restatements — test infrastructure only.

The dense matrix is built by clipping every ray against every voxel box separately
(slab method, vectorised over voxels). It is an algorithm independent of the Siddon
trace in oracle.c, so A @ f vs the oracle's P f pins the projector on small grids.
"""
from __future__ import annotations

import numpy as np


def _view_frame(geom, theta):
    c, s = np.cos(theta), np.sin(theta)
    S = np.array([geom.sad * c, geom.sad * s, 0.0])
    C = np.array([-(geom.sdd - geom.sad) * c, -(geom.sdd - geom.sad) * s, 0.0])
    eu = np.array([-s, c, 0.0])
    ev = np.array([0.0, 0.0, 1.0])
    return S, C, eu, ev


def system_matrix(geom) -> np.ndarray:
    """Dense A (M x N): A[i, j] = length (mm) of ray i (source to pixel centre) inside
    the half-open voxel box j. Rows ordered (k, iv, iu), columns (iz, iy, ix)."""
    n = np.array([geom.nx, geom.ny, geom.nz])
    h = np.array([geom.dx, geom.dy, geom.dz])
    o = -0.5 * n * h
    lo_axes = [o[a] + np.arange(n[a]) * h[a] for a in range(3)]
    hi_axes = [lo + h[a] for a, lo in enumerate(lo_axes)]
    M = geom.n_views * geom.nv * geom.nu
    N = geom.nx * geom.ny * geom.nz
    A = np.zeros((M, N))
    angles = geom.view_angles()
    row = 0
    for k in range(geom.n_views):
        S, C, eu, ev = _view_frame(geom, angles[k])
        for iv in range(geom.nv):
            for iu in range(geom.nu):
                u = geom.u_off + (iu - 0.5 * (geom.nu - 1)) * geom.du
                v = geom.v_off + (iv - 0.5 * (geom.nv - 1)) * geom.dv
                D = C + u * eu + v * ev
                d = D - S
                amin = [None] * 3
                amax = [None] * 3
                for a in range(3):
                    if d[a] != 0.0:
                        a0 = (lo_axes[a] - S[a]) / d[a]
                        a1 = (hi_axes[a] - S[a]) / d[a]
                        amin[a] = np.minimum(a0, a1)
                        amax[a] = np.maximum(a0, a1)
                    else:
                        inside = (S[a] >= lo_axes[a]) & (S[a] < hi_axes[a])
                        amin[a] = np.where(inside, -np.inf, np.inf)
                        amax[a] = np.where(inside, np.inf, -np.inf)
                lo3 = np.maximum(np.maximum(amin[2][:, None, None], amin[1][None, :, None]),
                                 amin[0][None, None, :])
                hi3 = np.minimum(np.minimum(amax[2][:, None, None], amax[1][None, :, None]),
                                 amax[0][None, None, :])
                lo3 = np.maximum(lo3, 0.0)
                hi3 = np.minimum(hi3, 1.0)
                A[row] = (np.maximum(hi3 - lo3, 0.0) * np.linalg.norm(d)).ravel()
                row += 1
    return A


def format_codes(fmt: str):
    """Every finite value of a 16-bit format, sorted, with its bit pattern: decoded from
    all 2^16 codes (binary16 via numpy's float16 view; bfloat16 as the high half of a
    binary32 pattern)."""
    codes = np.arange(1 << 16, dtype=np.uint32)
    with np.errstate(invalid="ignore"):  # the NaN codes decode to NaN and are dropped below
        if fmt == "f16":
            vals = codes.astype(np.uint16).view(np.float16).astype(np.float64)
        elif fmt == "bf16":
            vals = (codes << 16).view(np.float32).astype(np.float64)
        else:
            raise ValueError(fmt)
    keep = np.isfinite(vals) & ~((vals == 0) & (codes >= 0x8000))  # drop -0 and non-finite
    order = np.argsort(vals[keep], kind="stable")
    return vals[keep][order], codes[keep][order]


def round_nearest_even(x, fmt: str):
    """Brute-force rounding to a 16-bit format: the nearest finite value, ties to the
    code with an even last bit; beyond the largest value by half its spacing or more,
    infinity. A search over all codes, independent of any exponent arithmetic."""
    vals, codes = format_codes(fmt)
    x = np.asarray(x, dtype=np.float64)
    top_gap = vals[-1] - vals[-2]
    ext = np.concatenate([[-vals[-1] - top_gap], vals, [vals[-1] + top_gap]])  # +-inf stand-ins
    ext_codes = np.concatenate([[0], codes, [0]])  # infinities' codes end in 0 (even)
    i = np.clip(np.searchsorted(ext, x), 1, len(ext) - 1)
    lo, hi = ext[i - 1], ext[i]
    dlo, dhi = x - lo, hi - x
    pick_hi = (dhi < dlo) | ((dhi == dlo) & (ext_codes[i] % 2 == 0))
    out = np.where(pick_hi, hi, lo)
    out = np.where(out > vals[-1], np.inf, np.where(out < vals[0], -np.inf, out))
    return np.where(x == 0, x, out)


def cgls_dense(A, y, x0, n_iter, storage=None):
    """Appendix 1 CGLS on a dense matrix (the same listing, numpy vectors). storage
    'bf16' / 'f16': r and q held in that format (rounded by round_nearest_even where
    formed; binary16 holds q / sqrt(gamma))."""
    rnd = (lambda v: v) if storage is None else (lambda v: round_nearest_even(v, storage))
    x = x0.astype(np.float64).copy()
    r = rnd(y - A @ x)
    s = A.T @ r
    p = s.copy()
    gamma = s @ s
    for _ in range(n_iter):
        q = A @ p
        delta = q @ q
        if gamma == 0.0 or delta == 0.0:
            break
        alpha = gamma / delta
        x += alpha * p
        kappa = 1.0 / np.sqrt(gamma) if storage == "f16" else 1.0
        r = rnd(r - (alpha / kappa) * rnd(kappa * q))
        s = A.T @ r
        gnew = s @ s
        p = s + (gnew / gamma) * p
        gamma = gnew
    return x


def krylov_lsq(A, y, x0, n_iter):
    """Minimiser of ||A x - y|| over x0 + span{s, (A^T A) s, ..., (A^T A)^(n-1) s},
    s = A^T (y - A x0): what n CGLS steps compute in exact arithmetic. Solved by
    least squares on an orthonormalised Krylov basis."""
    r0 = y - A @ x0
    s = A.T @ r0
    B = A.T @ A
    vecs = []
    v = s.copy()
    for _ in range(n_iter):
        for w in vecs:  # modified Gram-Schmidt keeps the basis well conditioned
            v = v - (w @ v) * w
        nv = np.linalg.norm(v)
        if nv < 1e-14 * max(1.0, np.linalg.norm(s)):
            break
        v = v / nv
        vecs.append(v)
        v = B @ v
    if not vecs:
        return x0.copy()
    K = np.stack(vecs, axis=1)
    c, *_ = np.linalg.lstsq(A @ K, r0, rcond=None)
    return x0 + K @ c


# ---------------------------------------------------------------------------------------
# Dense restatement of the tight frame, Algorithm A2 and the multigrid cascade
# ---------------------------------------------------------------------------------------

# The paper's piecewise-linear filters (Section 2.1), taps at offsets -1, 0, +1.
_TAPS = (np.array([1.0, 2.0, 1.0]) / 4.0,
         np.sqrt(2.0) / 4.0 * np.array([1.0, 0.0, -1.0]),
         np.array([-1.0, 2.0, -1.0]) / 4.0)


def filter_matrix(n: int, l: int) -> np.ndarray:
    """n x n periodic convolution matrix of filter l: (H f)[x] = sum_a h_l[a] f[x - a]."""
    H = np.zeros((n, n))
    for a, h in zip((-1, 0, 1), _TAPS[l]):
        for x in range(n):
            H[x, (x - a) % n] += h
    return H


def frame_analysis(f: np.ndarray) -> np.ndarray:
    """W f as 27 channels (27, nz, ny, nx), channel i = l + 3m + 9n: the 1-D filter
    matrices applied along x (l), y (m) and z (n)."""
    nz, ny, nx = f.shape
    out = np.empty((27,) + f.shape)
    for i in range(27):
        l, m, n = i % 3, (i // 3) % 3, i // 9
        out[i] = np.einsum("zc,yb,xa,cba->zyx", filter_matrix(nz, n), filter_matrix(ny, m),
                           filter_matrix(nx, l), f)
    return out


def frame_synthesis(alpha: np.ndarray) -> np.ndarray:
    """W^T alpha: the transposed filter matrices applied per channel and summed."""
    _, nz, ny, nx = alpha.shape
    out = np.zeros(alpha.shape[1:])
    for i in range(27):
        l, m, n = i % 3, (i // 3) % 3, i // 9
        out += np.einsum("cz,by,ax,cba->zyx", filter_matrix(nz, n), filter_matrix(ny, m),
                         filter_matrix(nx, l), alpha[i])
    return out


def shrink(alpha: np.ndarray, mu: float) -> np.ndarray:
    """Eq. (2): keep the low-pass channel, scale the 26 high-pass coefficients of each
    voxel by max(1 - mu / ||alpha_h||, 0) (factor 0 where the norm is 0)."""
    nrm = np.sqrt((alpha[1:] ** 2).sum(axis=0))
    with np.errstate(divide="ignore", invalid="ignore"):
        scale = np.where(nrm > mu, 1.0 - mu / np.where(nrm > 0, nrm, 1.0), 0.0)
    out = alpha.copy()
    out[1:] *= scale
    return out


def a2_dense(A, y, shape, mu, n_outer, n_cgls=3, positivity=True, momentum=True, f0=None):
    """Algorithm A2 (Section 2.1) with the dense system matrix A: momentum point, n_cgls
    CGLS updates, frame shrinkage, positivity, then the t recurrence
    t <- (1 + sqrt(1 + 4 t^2)) / 2 from t^(0) = t^(-1) = 1."""
    y = np.asarray(y, dtype=np.float64).ravel()
    f = np.zeros(shape) if f0 is None else np.array(f0, dtype=np.float64)
    f_prev = f.copy()
    t_prev = t = 1.0
    for _ in range(n_outer):
        c = (t_prev - 1.0) / t if momentum else 0.0
        v = f + c * (f - f_prev)
        x = cgls_dense(A, y, v.ravel(), n_cgls).reshape(shape)
        x = frame_synthesis(shrink(frame_analysis(x), mu))
        if positivity:
            x = np.where(x < 0.0, 0.0, x)
        f_prev, f = f, x
        t_prev, t = t, 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
    return f


def interpolation_matrix(nc: int, hc: float, nf: int, hf: float) -> np.ndarray:
    """nf x nc linear interpolation from coarse voxel centres to fine voxel centres along
    one axis (both grids centred on 0), the position clamped to the coarse centres' span."""
    xc = -0.5 * nc * hc + (np.arange(nc) + 0.5) * hc
    xf = -0.5 * nf * hf + (np.arange(nf) + 0.5) * hf
    T = np.zeros((nf, nc))
    for i, x in enumerate(xf):
        if nc == 1 or x <= xc[0]:
            T[i, 0] = 1.0
        elif x >= xc[-1]:
            T[i, -1] = 1.0
        else:
            j = int(np.searchsorted(xc, x, side="right")) - 1
            w = (x - xc[j]) / (xc[j + 1] - xc[j])
            T[i, j] += 1.0 - w
            T[i, j + 1] += w
    return T


def reconstruct_dense(geom, y, mu, levels, iters, n_cgls=3, positivity=True, momentum=True):
    """The multigrid cascade of Section 2.2.3 with dense matrices: level l has
    ceil(n / 2^l) voxels per axis at 2^l times the spacing (same centre, same imager and
    y); A2 from 0 on the coarsest grid, each result interpolated (per axis, trilinear) to
    start the next finer grid. iters is coarsest first."""
    y = np.asarray(y, dtype=np.float64).ravel()
    f = None
    prev = None
    for lev in range(levels - 1, -1, -1):
        gl = geom.level(lev)
        shape = gl.vol_shape
        f0 = None
        if f is not None:
            Tz = interpolation_matrix(prev.nz, prev.dz, gl.nz, gl.dz)
            Ty = interpolation_matrix(prev.ny, prev.dy, gl.ny, gl.dy)
            Tx = interpolation_matrix(prev.nx, prev.dx, gl.nx, gl.dx)
            f0 = np.einsum("zc,yb,xa,cba->zyx", Tz, Ty, Tx, f)
        f = a2_dense(system_matrix(gl), y, shape, mu, iters[levels - 1 - lev], n_cgls,
                     positivity, momentum, f0)
        prev = gl
    return f
