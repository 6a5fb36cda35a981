"""FP64 CPU oracle — test infrastructure only.

Thin ctypes wrapper around ``oracle.c`` (plain C, double precision, optional OpenMP).
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` use
this package; the CUDA library never does, and the two share no code.

Every function takes numpy arrays in the layouts of ``synth.Geometry``: volumes
(nz, ny, nx), projection stacks (n_views, nv, nu), frame coefficients (27, nz, ny, nx).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library with gcc (OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("u_off", ctypes.c_double), ("v_off", ctypes.c_double),
                ("sad", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double))]


_P = ctypes.POINTER(ctypes.c_double)
_PL = ctypes.POINTER(ctypes.c_long)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            G = ctypes.POINTER(_Geom)
            sig = {
                "o_project": (None, [G, _P, _P]),
                "o_project_rays": (None, [G, _P, ctypes.c_long, _PL, _P]),
                "o_backproject": (None, [G, _P, _P]),
                "o_backproject_voxels": (None, [G, _P, ctypes.c_long, _PL, _P]),
                "o_backproject_eq3": (None, [G, _P, _P]),
                "o_count_nnz": (ctypes.c_longlong, [G]),
                "o_trace": (ctypes.c_long, [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, _PL, _P, ctypes.c_long]),
                "o_ray_box_length": (ctypes.c_double, [G, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
                "o_tf_analyze": (None, [ctypes.c_int] * 3 + [_P, _P]),
                "o_tf_synthesize": (None, [ctypes.c_int] * 3 + [_P, _P]),
                "o_tf_shrink": (None, [ctypes.c_int] * 3 + [_P, ctypes.c_double]),
                "o_positivity": (None, [ctypes.c_long, _P]),
                "o_tf_shrink_voxels": (None, [ctypes.c_int] * 3 + [_P, ctypes.c_double, ctypes.c_int, ctypes.c_long, _PL, _P]),
                "o_cgls": (None, [G, _P, _P, ctypes.c_int, _P]),
                "o_cgls_storage": (None, [G, _P, _P, ctypes.c_int, _P, ctypes.c_int]),
                "o_round_storage": (None, [ctypes.c_long, _P, ctypes.c_int]),
                "o_a2": (None, [G, _P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P]),
                "o_prolong": (None, [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_P] + [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_P]),
                "o_restrict": (None, [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_P] + [ctypes.c_int] * 3 + [ctypes.c_double] * 3 + [_P]),
                "o_reconstruct": (None, [G, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
                "o_reconstruct_storage": (None, [G, _P, ctypes.c_double, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _P]),
                "o_num_threads": (ctypes.c_int, []),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


class _GeomHolder:
    """Keeps the angle array alive for as long as the ctypes struct is used."""

    def __init__(self, geom):
        self.angles = np.ascontiguousarray(geom.view_angles(), dtype=np.float64)
        self.s = _Geom(geom.nx, geom.ny, geom.nz, geom.dx, geom.dy, geom.dz,
                       geom.nu, geom.nv, geom.du, geom.dv, geom.u_off, geom.v_off,
                       geom.sad, geom.sdd, geom.n_views, self.angles.ctypes.data_as(_P))

    def ref(self):
        return ctypes.byref(self.s)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == tuple(shape), (a.shape, shape)
    return a


def _ptr(a):
    return a.ctypes.data_as(_P)


def num_threads() -> int:
    return int(_load().o_num_threads())


def project(geom, f):
    """P f — Siddon forward projection (Eq. (1), Section 2.2.1). Returns (K, nv, nu)."""
    lib = _load(); gh = _GeomHolder(geom)
    f = _f64(f, geom.vol_shape)
    out = np.empty(geom.proj_shape)
    lib.o_project(gh.ref(), _ptr(f), _ptr(out))
    return out


def project_rays(geom, f, rays):
    """P f at selected flat ray indices (k*nv + iv)*nu + iu."""
    lib = _load(); gh = _GeomHolder(geom)
    f = _f64(f, geom.vol_shape)
    rays = np.ascontiguousarray(rays, dtype=np.int64)
    out = np.empty(rays.shape[0])
    lib.o_project_rays(gh.ref(), _ptr(f), rays.shape[0], rays.ctypes.data_as(_PL), _ptr(out))
    return out


def backproject(geom, g):
    """P^T g — exact transpose of the Siddon weights. Returns (nz, ny, nx)."""
    lib = _load(); gh = _GeomHolder(geom)
    g = _f64(g, geom.proj_shape)
    out = np.empty(geom.vol_shape)
    lib.o_backproject(gh.ref(), _ptr(g), _ptr(out))
    return out


def backproject_voxels(geom, g, voxels):
    """P^T g at selected flat voxel indices (iz*ny + iy)*nx + ix, by slab clipping."""
    lib = _load(); gh = _GeomHolder(geom)
    g = _f64(g, geom.proj_shape)
    voxels = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(voxels.shape[0])
    lib.o_backproject_voxels(gh.ref(), _ptr(g), voxels.shape[0], voxels.ctypes.data_as(_PL), _ptr(out))
    return out


def backproject_eq3(geom, g):
    """The paper's voxel-driven bilinear backprojector, Eq. (3)."""
    lib = _load(); gh = _GeomHolder(geom)
    g = _f64(g, geom.proj_shape)
    out = np.empty(geom.vol_shape)
    lib.o_backproject_eq3(gh.ref(), _ptr(g), _ptr(out))
    return out


def count_nnz(geom) -> int:
    """Number of non-zero entries of the Siddon system matrix P."""
    lib = _load(); gh = _GeomHolder(geom)
    return int(lib.o_count_nnz(gh.ref()))


def trace(geom, k, iu, iv):
    """Siddon segments of one ray: (flat voxel indices, lengths in mm)."""
    lib = _load(); gh = _GeomHolder(geom)
    cap = geom.nx + geom.ny + geom.nz + 4
    vox = np.empty(cap, dtype=np.int64)
    ln = np.empty(cap)
    m = lib.o_trace(gh.ref(), k, iu, iv, vox.ctypes.data_as(_PL), _ptr(ln), cap)
    return vox[:m].copy(), ln[:m].copy()


def ray_box_length(geom, k, iu, iv, lo, hi):
    lib = _load(); gh = _GeomHolder(geom)
    lo = _f64(lo, (3,)); hi = _f64(hi, (3,))
    return float(lib.o_ray_box_length(gh.ref(), k, iu, iv, _ptr(lo), _ptr(hi)))


def tf_analyze(f):
    """W f: 27 channels (27, nz, ny, nx), periodic boundary."""
    lib = _load()
    f = _f64(f)
    nz, ny, nx = f.shape
    out = np.empty((27, nz, ny, nx))
    lib.o_tf_analyze(nx, ny, nz, _ptr(f), _ptr(out))
    return out


def tf_synthesize(alpha):
    """W^T alpha."""
    lib = _load()
    alpha = _f64(alpha)
    _, nz, ny, nx = alpha.shape
    out = np.empty((nz, ny, nx))
    lib.o_tf_synthesize(nx, ny, nz, _ptr(alpha), _ptr(out))
    return out


def tf_shrink(alpha, mu):
    """T_mu alpha (Eq. (2)); returns a new array."""
    lib = _load()
    a = _f64(alpha).copy()
    _, nz, ny, nx = a.shape
    lib.o_tf_shrink(nx, ny, nz, _ptr(a), float(mu))
    return a


def positivity(f):
    lib = _load()
    a = _f64(f).copy()
    lib.o_positivity(a.size, _ptr(a))
    return a


def tf_shrink_voxels(f, mu, positive, voxels):
    """H(W^T T_mu W f) at selected flat voxel indices (z*ny + y)*nx + x."""
    lib = _load()
    f = _f64(f)
    nz, ny, nx = f.shape
    voxels = np.ascontiguousarray(voxels, dtype=np.int64)
    out = np.empty(voxels.shape[0])
    lib.o_tf_shrink_voxels(nx, ny, nz, _ptr(f), float(mu), int(bool(positive)), voxels.shape[0],
                           voxels.ctypes.data_as(_PL), _ptr(out))
    return out


def tf_synthesize_shrink(alpha, mu, positive):
    """H(W^T T_mu alpha) (H only if ``positive``)."""
    f = tf_synthesize(tf_shrink(alpha, mu))
    return positivity(f) if positive else f


# storage codes of the reduced-precision variant: 0 none (FP64), 1 bfloat16, 2 binary16
STORAGE = {"f32": 0, "f64": 0, "bf16": 1, "f16": 2}


def _storage(storage) -> int:
    return STORAGE[storage] if isinstance(storage, str) else int(storage)


def round_storage(x, storage):
    """Round every value to the 16-bit storage format (nearest, ties to even)."""
    lib = _load()
    a = np.array(x, dtype=np.float64, copy=True)
    flat = np.ascontiguousarray(a.ravel())
    lib.o_round_storage(flat.size, _ptr(flat), _storage(storage))
    return flat.reshape(a.shape)


def cgls(geom, y, x0, n_iter, return_resid=False, storage=0):
    """n_iter CGLS updates from x0 (Appendix 1). Returns x (and ||r||^2 history).
    storage 'bf16' / 'f16' holds r and q in that 16-bit format (reduced-precision variant)."""
    lib = _load(); gh = _GeomHolder(geom)
    y = _f64(y, geom.proj_shape)
    x = _f64(x0, geom.vol_shape).copy()
    res = np.empty(n_iter + 1)
    lib.o_cgls_storage(gh.ref(), _ptr(y), _ptr(x), int(n_iter), _ptr(res), _storage(storage))
    return (x, res) if return_resid else x


def a2(geom, y, mu, n_outer, n_cgls=3, positivity=True, momentum=True, f0=None,
       return_coefficients=False):
    """Algorithm A2 (A1 with momentum=False) on one grid from f0 (default 0). With
    return_coefficients, also the momentum coefficient each iteration applied."""
    lib = _load(); gh = _GeomHolder(geom)
    y = _f64(y, geom.proj_shape)
    f = np.zeros(geom.vol_shape) if f0 is None else _f64(f0, geom.vol_shape).copy()
    coef = np.full(max(int(n_outer), 1), np.nan)
    lib.o_a2(gh.ref(), _ptr(y), float(mu), int(n_outer), int(n_cgls), int(bool(positivity)),
             int(bool(momentum)), _ptr(f), _ptr(coef))
    return (f, coef[:int(n_outer)]) if return_coefficients else f


def prolong(fc, coarse_spacing, fine_shape, fine_spacing):
    """Trilinear prolongation coarse (nz, ny, nx) -> fine grid (both centred)."""
    lib = _load()
    fc = _f64(fc)
    cnz, cny, cnx = fc.shape
    nz, ny, nx = fine_shape
    out = np.empty((nz, ny, nx))
    cdx, cdy, cdz = coarse_spacing
    dx, dy, dz = fine_spacing
    lib.o_prolong(cnx, cny, cnz, cdx, cdy, cdz, _ptr(fc), nx, ny, nz, dx, dy, dz, _ptr(out))
    return out


def restrict(ff, fine_spacing, coarse_shape, coarse_spacing):
    """Mean of fine voxels whose centres fall in each coarse voxel."""
    lib = _load()
    ff = _f64(ff)
    nz, ny, nx = ff.shape
    cnz, cny, cnx = coarse_shape
    out = np.empty((cnz, cny, cnx))
    dx, dy, dz = fine_spacing
    cdx, cdy, cdz = coarse_spacing
    lib.o_restrict(nx, ny, nz, dx, dy, dz, _ptr(ff), cnx, cny, cnz, cdx, cdy, cdz, _ptr(out))
    return out


def reconstruct(geom, y, mu, levels, iters, n_cgls=3, positivity=True, momentum=True, storage=0):
    """Multigrid A2 reconstruction (Section 2.2.3); iters coarsest first. storage selects
    the reduced-precision CGLS variant ('bf16' / 'f16'; 0 = plain FP64)."""
    lib = _load(); gh = _GeomHolder(geom)
    y = _f64(y, geom.proj_shape)
    it = (ctypes.c_int * levels)(*[int(v) for v in iters])
    out = np.empty(geom.vol_shape)
    lib.o_reconstruct_storage(gh.ref(), _ptr(y), float(mu), int(levels), it, int(n_cgls),
                              int(bool(positivity)), int(bool(momentum)), _storage(storage), _ptr(out))
    return out
