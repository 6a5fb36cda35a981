"""Python binding of the cbcttf C ABI (include/cbcttf.h).

Argument marshalling only: every step runs in the CUDA library ``libcbcttf.so``, built
in-tree by ``paper_1008_2042_gb300.build.build()``. PyTorch supplies device memory and
the current stream. There is no CPU fallback: if the library is missing or no GPU is
present, calls raise.

Layouts follow the C ABI: volumes (nz, ny, nx) float32, projection stacks
(n_views, nv, nu), frame coefficients (27, nz, ny, nx), all contiguous CUDA tensors on
the device the geometry was created on. Projection stacks and frame coefficients may be
float32, bfloat16 or float16 (storage only: the arithmetic is FP32).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libcbcttf.so")

_lib = None


class CbctError(RuntimeError):
    """A non-OK status returned by the library."""

    def __init__(self, status: int, message: str):
        super().__init__(f"cbcttf status {status}: {message}")
        self.status = status


class GeometryDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("dx", ctypes.c_double), ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("du", ctypes.c_double), ("dv", ctypes.c_double),
                ("u_off", ctypes.c_double), ("v_off", ctypes.c_double),
                ("sad", ctypes.c_double), ("sdd", ctypes.c_double),
                ("n_views", ctypes.c_int), ("angles", ctypes.POINTER(ctypes.c_double))]


class ReconOpts(ctypes.Structure):
    _fields_ = [("n_cgls", ctypes.c_int), ("momentum", ctypes.c_int), ("positivity", ctypes.c_int),
                ("storage", ctypes.c_int)]


# cbct_dtype codes of the storage types
DTYPES = {torch.float32: 0, torch.bfloat16: 1, torch.float16: 2}
_DTYPE_NAMES = {"f32": torch.float32, "fp32": torch.float32, "float32": torch.float32,
                "bf16": torch.bfloat16, "bfloat16": torch.bfloat16,
                "f16": torch.float16, "fp16": torch.float16, "float16": torch.float16}


def storage_dtype(d) -> torch.dtype:
    """A storage type given as a torch dtype or a name ('f32', 'bf16', 'f16')."""
    if isinstance(d, str):
        if d.lower() not in _DTYPE_NAMES:
            raise ValueError(f"unknown storage type {d!r}")
        return _DTYPE_NAMES[d.lower()]
    if d not in DTYPES:
        raise ValueError(f"unsupported storage type {d}")
    return d


_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double
_f = ctypes.c_float

_SIGNATURES = {
    "cbct_geometry_create": [ctypes.POINTER(GeometryDesc), ctypes.POINTER(_vp)],
    "cbct_geometry_destroy": [_vp],
    "cbct_project": [_vp, _vp, _vp, _vp],
    "cbct_project_static": [_vp, _vp, _vp, _vp],
    "cbct_backproject": [_vp, _vp, _vp, _vp],
    "cbct_project_ex": [_vp, _vp, _vp, _i, _vp],
    "cbct_backproject_ex": [_vp, _vp, _i, _vp, _vp],
    "cbct_tf_analyze_ex": [_i, _i, _i, _vp, _vp, _i, _vp],
    "cbct_tf_synthesize_shrink_ex": [_i, _i, _i, _vp, _i, _f, _i, _vp, _vp],
    "cbct_backproject_eq3": [_vp, _vp, _vp, _vp],
    "cbct_project_batch": [_vp, _i, _vp, _vp, _vp],
    "cbct_backproject_batch": [_vp, _i, _vp, _vp, _vp],
    "cbct_tf_analyze": [_i, _i, _i, _vp, _vp, _vp],
    "cbct_tf_synthesize_shrink": [_i, _i, _i, _vp, _f, _i, _vp, _vp],
    "cbct_tf_shrink": [_i, _i, _i, _vp, _f, _i, _vp, _vp],
    "cbct_cgls": [_vp, _vp, _vp, _i, _vp],
    "cbct_reconstruct": [_vp, _vp, _f, _f, _i, ctypes.POINTER(_i), _vp, _vp],
    "cbct_reconstruct_ex": [_vp, _vp, _f, _f, _i, ctypes.POINTER(_i), ctypes.POINTER(ReconOpts),
                            _vp, ctypes.c_size_t, _vp, _vp],
    "cbct_reconstruct_workspace_size": [_vp, ctypes.POINTER(ctypes.c_size_t)],
    "cbct_prolong": [_i, _i, _i, _d, _d, _d, _vp, _i, _i, _i, _d, _d, _d, _vp, _vp],
    "cbct_restrict": [_i, _i, _i, _d, _d, _d, _vp, _i, _i, _i, _d, _d, _d, _vp, _vp],
    "cbct_count_nnz": [_vp, _i, ctypes.POINTER(ctypes.c_ulonglong), _vp],
    "cbct_set_project_group": [_i],
    "cbct_project_group": [_vp, _i, ctypes.POINTER(ctypes.c_int)],
    "cbct_server_create": [ctypes.c_void_p, ctypes.POINTER(_vp)],
    "cbct_server_submit": [_vp, ctypes.POINTER(GeometryDesc), _vp, _f, _f, _i, ctypes.POINTER(_i),
                           ctypes.POINTER(ReconOpts), _vp, ctypes.POINTER(ctypes.c_longlong)],
    "cbct_server_wait": [_vp, ctypes.c_longlong, _d, _vp],
    "cbct_server_stats_get": [_vp, _vp],
    "cbct_server_destroy": [_vp],
    "cbct_profiling_enable": [_i],
    "cbct_profiling_select": [ctypes.c_uint],
    "cbct_profiling_reset": [],
    "cbct_kernel_time": [_i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_ulonglong)],
}

KERNEL_KINDS = {"project": 0, "backproject": 1, "tf_analyze": 2, "tf_synth": 3, "other": 4}


def load_library(path: str = LIB_PATH):
    """Load libcbcttf.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1008_2042_gb300.build.build()")
        lib = ctypes.CDLL(path)
        for name, args in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lib.cbct_last_error.restype = ctypes.c_char_p
        lib.cbct_last_error.argtypes = []
        lib.cbct_version.restype = ctypes.c_char_p
        lib.cbct_version.argtypes = []
        lib.cbct_launch_count.restype = ctypes.c_ulonglong
        lib.cbct_launch_count.argtypes = []
        _lib = lib
    return _lib


def _check(status: int):
    if status != 0:
        raise CbctError(status, load_library().cbct_last_error().decode())


def _stream(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t: torch.Tensor, shape, name: str, typed: bool = False) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if typed:
        if t.dtype not in DTYPES or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous float32, bfloat16 or float16 tensor")
    elif t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return ctypes.c_void_p(t.data_ptr())


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load_library().cbct_launch_count())


def version() -> str:
    return load_library().cbct_version().decode()


def make_desc(desc=None, **kw):
    """A GeometryDesc from any object with the fields of cbct_geometry_desc (nx, ny, nz,
    dx, dy, dz, nu, nv, du, dv, n_views and optionally u_off, v_off, sad, sdd, angles), or
    from keyword arguments. Returns (desc, angle array to keep alive while desc is used)."""
    get = (lambda k, d=None: getattr(desc, k, d)) if desc is not None else (lambda k, d=None: kw.get(k, d))
    n_views = int(get("n_views"))
    angles = get("angles", None)
    keep, ap = None, None
    if angles is not None:
        keep = (ctypes.c_double * n_views)(*[float(a) for a in angles])
        ap = ctypes.cast(keep, ctypes.POINTER(ctypes.c_double))
    d = GeometryDesc(int(get("nx")), int(get("ny")), int(get("nz")), float(get("dx")), float(get("dy")),
                     float(get("dz")), int(get("nu")), int(get("nv")), float(get("du")), float(get("dv")),
                     float(get("u_off", 0.0)), float(get("v_off", 0.0)), float(get("sad", 1000.0)),
                     float(get("sdd", 1500.0)), n_views, ap)
    return d, keep


class Geometry:
    """Owns a cbct_geometry handle. Accepts any object with the fields of
    cbct_geometry_desc (nx, ny, nz, dx, dy, dz, nu, nv, du, dv, sad, sdd, n_views, and
    optionally u_off, v_off, angles), or the same as keyword arguments."""

    def __init__(self, desc=None, **kw):
        lib = load_library()
        d, self._angles = make_desc(desc, **kw)
        self.nx, self.ny, self.nz = d.nx, d.ny, d.nz
        self.dx, self.dy, self.dz = d.dx, d.dy, d.dz
        self.nu, self.nv = d.nu, d.nv
        self.du, self.dv = d.du, d.dv
        self.u_off, self.v_off = d.u_off, d.v_off
        self.sad, self.sdd = d.sad, d.sdd
        self.n_views = d.n_views
        h = ctypes.c_void_p()
        _check(lib.cbct_geometry_create(ctypes.byref(d), ctypes.byref(h)))
        self._h = h
        self.device = torch.cuda.current_device()

    @property
    def handle(self):
        return self._h

    @property
    def vol_shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def proj_shape(self):
        return (self.n_views, self.nv, self.nu)

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().cbct_geometry_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def project(geom: Geometry, f: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None,
            dtype=torch.float32) -> torch.Tensor:
    """g = P f (Siddon forward projection). The projections are stored as `out.dtype` when
    `out` is given, else as `dtype` (float32, bfloat16 or float16)."""
    if out is None:
        out = torch.empty(geom.proj_shape, dtype=storage_dtype(dtype), device=f.device)
    po = _dev(out, geom.proj_shape, "out", typed=True)
    lib = load_library()
    if out.dtype == torch.float32:
        _check(lib.cbct_project(geom.handle, _dev(f, geom.vol_shape, "f"), po, _stream(stream)))
    else:
        _check(lib.cbct_project_ex(geom.handle, _dev(f, geom.vol_shape, "f"), po, DTYPES[out.dtype],
                                   _stream(stream)))
    return out


def project_static(geom: Geometry, f: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    """g = P f like project(), using the library's fixed device scratch instead of
    allocating: for callers that cannot allocate device memory while running. `out` must
    be supplied (nothing is allocated here either)."""
    _check(load_library().cbct_project_static(geom.handle, _dev(f, geom.vol_shape, "f"),
                                              _dev(out, geom.proj_shape, "out"), _stream(stream)))
    return out


def backproject(geom: Geometry, g: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """f = P^T g (exact adjoint); g may be float32, bfloat16 or float16."""
    if out is None:
        out = torch.empty(geom.vol_shape, dtype=torch.float32, device=g.device)
    pg = _dev(g, geom.proj_shape, "g", typed=True)
    lib = load_library()
    if g.dtype == torch.float32:
        _check(lib.cbct_backproject(geom.handle, pg, _dev(out, geom.vol_shape, "out"), _stream(stream)))
    else:
        _check(lib.cbct_backproject_ex(geom.handle, pg, DTYPES[g.dtype], _dev(out, geom.vol_shape, "out"),
                                       _stream(stream)))
    return out


def backproject_eq3(geom: Geometry, g: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """The paper's Eq. (3) backprojector (voxel-driven, bilinear): approximates P^T g."""
    if out is None:
        out = torch.empty(geom.vol_shape, dtype=torch.float32, device=g.device)
    _check(load_library().cbct_backproject_eq3(geom.handle, _dev(g, geom.proj_shape, "g"),
                                               _dev(out, geom.vol_shape, "out"), _stream(stream)))
    return out


def project_batch(geom: Geometry, f: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """P of a batch of volumes (B, nz, ny, nx) -> (B, n_views, nv, nu)."""
    b = f.shape[0]
    if out is None:
        out = torch.empty((b,) + geom.proj_shape, dtype=torch.float32, device=f.device)
    _check(load_library().cbct_project_batch(geom.handle, int(b), _dev(f, (b,) + geom.vol_shape, "f"),
                                             _dev(out, (b,) + geom.proj_shape, "out"), _stream(stream)))
    return out


def backproject_batch(geom: Geometry, g: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Exact P^T of a batch of stacks (B, n_views, nv, nu) -> (B, nz, ny, nx)."""
    b = g.shape[0]
    if out is None:
        out = torch.empty((b,) + geom.vol_shape, dtype=torch.float32, device=g.device)
    _check(load_library().cbct_backproject_batch(geom.handle, int(b), _dev(g, (b,) + geom.proj_shape, "g"),
                                                 _dev(out, (b,) + geom.vol_shape, "out"), _stream(stream)))
    return out


def tf_analyze(f: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None, dtype=torch.float32) -> torch.Tensor:
    """alpha = W f, 27 channels, stored as `out.dtype` (or `dtype` when out is None)."""
    nz, ny, nx = f.shape
    if out is None:
        out = torch.empty((27, nz, ny, nx), dtype=storage_dtype(dtype), device=f.device)
    pa = _dev(out, (27, nz, ny, nx), "out", typed=True)
    lib = load_library()
    if out.dtype == torch.float32:
        _check(lib.cbct_tf_analyze(nx, ny, nz, _dev(f, None, "f"), pa, _stream(stream)))
    else:
        _check(lib.cbct_tf_analyze_ex(nx, ny, nz, _dev(f, None, "f"), pa, DTYPES[out.dtype], _stream(stream)))
    return out


def tf_synthesize_shrink(alpha: torch.Tensor, mu: float, positivity: bool = True,
                         out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """f = H(W^T T_mu alpha) (H only if positivity); alpha may be float32, bfloat16 or float16."""
    _, nz, ny, nx = alpha.shape
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=alpha.device)
    pa = _dev(alpha, None, "alpha", typed=True)
    lib = load_library()
    if alpha.dtype == torch.float32:
        _check(lib.cbct_tf_synthesize_shrink(nx, ny, nz, pa, float(mu), int(bool(positivity)),
                                             _dev(out, (nz, ny, nx), "out"), _stream(stream)))
    else:
        _check(lib.cbct_tf_synthesize_shrink_ex(nx, ny, nz, pa, DTYPES[alpha.dtype], float(mu),
                                                int(bool(positivity)), _dev(out, (nz, ny, nx), "out"),
                                                _stream(stream)))
    return out


def tf_shrink(f: torch.Tensor, mu: float, positivity: bool = True, out: Optional[torch.Tensor] = None,
              stream=None) -> torch.Tensor:
    """f_out = H(W^T T_mu W f) in one fused pass (coefficients never stored)."""
    nz, ny, nx = f.shape
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=f.device)
    _check(load_library().cbct_tf_shrink(nx, ny, nz, _dev(f, None, "f"), float(mu), int(bool(positivity)),
                                         _dev(out, (nz, ny, nx), "out"), _stream(stream)))
    return out


def cgls(geom: Geometry, y: torch.Tensor, x: torch.Tensor, n_iter: int, stream=None) -> torch.Tensor:
    """n_iter CGLS updates of x in place (Appendix 1); returns x."""
    _check(load_library().cbct_cgls(geom.handle, _dev(y, geom.proj_shape, "y"), _dev(x, geom.vol_shape, "x"),
                                    int(n_iter), _stream(stream)))
    return x


def reconstruct(geom: Geometry, y: torch.Tensor, mu: float, levels: int, iters: Sequence[int],
                lam: float = 0.0, n_cgls: int = 3, momentum: bool = True, positivity: bool = True,
                workspace: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None,
                stream=None, storage=torch.float32) -> torch.Tensor:
    """Multigrid A2 reconstruction; iters lists the outer iterations per level, coarsest first.
    `storage` is the type of the CGLS residual and projected direction (float32, bfloat16,
    float16, or 'f32' / 'bf16' / 'f16')."""
    lib = load_library()
    if len(iters) != levels:
        raise ValueError("iters must have one entry per level")
    if out is None:
        out = torch.empty(geom.vol_shape, dtype=torch.float32, device=y.device)
    it = (ctypes.c_int * levels)(*[int(v) for v in iters])
    opts = ReconOpts(int(n_cgls), int(bool(momentum)), int(bool(positivity)), DTYPES[storage_dtype(storage)])
    ws, ws_bytes = None, 0
    if workspace is not None:
        if not workspace.is_cuda or not workspace.is_contiguous():
            raise TypeError("workspace must be a contiguous CUDA tensor")
        ws = ctypes.c_void_p(workspace.data_ptr())
        ws_bytes = workspace.numel() * workspace.element_size()
    _check(lib.cbct_reconstruct_ex(_dev(y, geom.proj_shape, "y"), geom.handle, float(mu), float(lam), int(levels),
                                   it, ctypes.byref(opts), ws, ctypes.c_size_t(ws_bytes),
                                   _dev(out, geom.vol_shape, "out"), _stream(stream)))
    return out


def reconstruct_workspace_size(geom: Geometry) -> int:
    n = ctypes.c_size_t()
    _check(load_library().cbct_reconstruct_workspace_size(geom.handle, ctypes.byref(n)))
    return int(n.value)


def prolong(fc: torch.Tensor, coarse_spacing, fine_shape, fine_spacing, out=None, stream=None) -> torch.Tensor:
    """Trilinear prolongation coarse (nz, ny, nx) -> fine grid, both centred on the origin."""
    cnz, cny, cnx = fc.shape
    nz, ny, nx = fine_shape
    if out is None:
        out = torch.empty((nz, ny, nx), dtype=torch.float32, device=fc.device)
    cdx, cdy, cdz = coarse_spacing
    dx, dy, dz = fine_spacing
    _check(load_library().cbct_prolong(cnx, cny, cnz, cdx, cdy, cdz, _dev(fc, None, "fc"), nx, ny, nz, dx, dy, dz,
                                       _dev(out, (nz, ny, nx), "out"), _stream(stream)))
    return out


def restrict(ff: torch.Tensor, fine_spacing, coarse_shape, coarse_spacing, out=None, stream=None) -> torch.Tensor:
    """Mean of the fine voxels whose centres fall in each coarse voxel."""
    nz, ny, nx = ff.shape
    cnz, cny, cnx = coarse_shape
    if out is None:
        out = torch.empty((cnz, cny, cnx), dtype=torch.float32, device=ff.device)
    dx, dy, dz = fine_spacing
    cdx, cdy, cdz = coarse_spacing
    _check(load_library().cbct_restrict(nx, ny, nz, dx, dy, dz, _dev(ff, None, "ff"), cnx, cny, cnz, cdx, cdy, cdz,
                                        _dev(out, (cnz, cny, cnx), "out"), _stream(stream)))
    return out


def count_nnz(geom: Geometry, level: int = 0, stream=None) -> int:
    """Non-zeros of P on a multigrid level, counted by the projector itself."""
    n = ctypes.c_ulonglong()
    _check(load_library().cbct_count_nnz(geom.handle, int(level), ctypes.byref(n), _stream(stream)))
    return int(n.value)


PROJECT_GROUP_SIZES = (16, 24, 32, 40, 48, 56, 64, 80, 96)


def set_project_group(segments: int) -> None:
    """Force the projector's column-group size (one of PROJECT_GROUP_SIZES); 0 restores
    the automatic per-launch choice. Process-wide."""
    _check(load_library().cbct_set_project_group(int(segments)))


def project_group(geom: Geometry, level: int = 0) -> int:
    """The column-group size an FP32 projection of `level` uses on the current device."""
    n = ctypes.c_int()
    _check(load_library().cbct_project_group(geom.handle, int(level), ctypes.byref(n)))
    return int(n.value)


def profiling(enable: bool) -> None:
    """Bracket every library kernel launch with CUDA events (measurement support)."""
    _check(load_library().cbct_profiling_enable(int(bool(enable))))


def profiling_select(kinds) -> None:
    """Time only the named kernel families (names of KERNEL_KINDS); an empty list stops."""
    mask = 0
    for k in kinds:
        mask |= 1 << KERNEL_KINDS[k]
    _check(load_library().cbct_profiling_select(mask))


def profiling_reset() -> None:
    _check(load_library().cbct_profiling_reset())


def kernel_times() -> dict:
    """Per kernel family: (summed device ms, launches) since the last reset."""
    lib = load_library()
    out = {}
    for name, kind in KERNEL_KINDS.items():
        ms, n = ctypes.c_double(), ctypes.c_ulonglong()
        _check(lib.cbct_kernel_time(kind, ctypes.byref(ms), ctypes.byref(n)))
        out[name] = (float(ms.value), int(n.value))
    return out


# ---------------------------------------------------------------------------------------
# Request server (cbct_server_*): continuous batching of whole reconstructions
# ---------------------------------------------------------------------------------------

class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_size_t), ("max_active", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("l2_budget_bytes", ctypes.c_size_t), ("size_priority", ctypes.c_int),
                ("max_bypass_s", ctypes.c_double)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("done", ctypes.c_int), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double), ("device_bytes", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("queued", ctypes.c_int), ("active", ctypes.c_int), ("max_active_seen", ctypes.c_int),
                ("bytes_in_use", ctypes.c_size_t), ("max_bytes_seen", ctypes.c_size_t),
                ("budget_bytes", ctypes.c_size_t), ("l2_budget_bytes", ctypes.c_size_t),
                ("bypassed", ctypes.c_longlong)]


def _host(t: torch.Tensor, numel: int, name: str) -> ctypes.c_void_p:
    if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous float32 CPU tensor")
    if not t.is_pinned():
        raise TypeError(f"{name} must be in page-locked memory (tensor.pin_memory())")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} values, expected {numel}")
    return ctypes.c_void_p(t.data_ptr())


class Server:
    """A cbct_server on the current device: submit() queues a reconstruction with pinned
    host buffers and returns at once; wait() blocks until it is done. Requests run
    concurrently on the GPU, admitted by slots and by the device-memory budget."""

    PRIORITIES = {"none": 0, "size": 1, "age": 2}

    def __init__(self, budget_bytes: int = 0, max_active: int = 16, use_graphs: bool = True,
                 l2_budget_bytes: int = 0, size_priority: bool = True, max_bypass_s: float = 0.0,
                 priority: Optional[str] = None):
        """priority: "size" (smallest requests first), "age" (oldest first, re-ranked after
        every A2 iteration) or "none"; None takes "size" or "none" from size_priority."""
        lib = load_library()
        if priority is None:
            priority = "size" if size_priority else "none"
        if priority not in self.PRIORITIES:
            raise ValueError(f"priority must be one of {sorted(self.PRIORITIES)}")
        o = ServerOpts(int(budget_bytes), int(max_active), int(bool(use_graphs)), int(l2_budget_bytes),
                       self.PRIORITIES[priority], float(max_bypass_s))
        h = ctypes.c_void_p()
        _check(lib.cbct_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._keep = {}  # id -> host tensors that must outlive the request

    def submit(self, geom, y_host: torch.Tensor, mu: float, levels: int, iters: Sequence[int],
               out: torch.Tensor, lam: float = 0.0, n_cgls: int = 3, momentum: bool = True,
               positivity: bool = True, storage=torch.float32) -> int:
        d, angles = make_desc(geom)
        if len(iters) != levels:
            raise ValueError("iters must have one entry per level")
        it = (ctypes.c_int * levels)(*[int(v) for v in iters])
        opts = ReconOpts(int(n_cgls), int(bool(momentum)), int(bool(positivity)), DTYPES[storage_dtype(storage)])
        py = _host(y_host, d.n_views * d.nv * d.nu, "y_host")
        pf = _host(out, d.nx * d.ny * d.nz, "out")
        rid = ctypes.c_longlong()
        _check(load_library().cbct_server_submit(self._h, ctypes.byref(d), py, float(mu), float(lam), int(levels),
                                                 it, ctypes.byref(opts), pf, ctypes.byref(rid)))
        self._keep[rid.value] = (y_host, out, angles)
        return int(rid.value)

    def wait(self, rid: int, timeout: Optional[float] = None) -> dict:
        """Blocks until request rid is done (raises CbctError on failure or timeout)."""
        info = RequestInfo()
        st = load_library().cbct_server_wait(self._h, int(rid), -1.0 if timeout is None else float(timeout),
                                             ctypes.byref(info))
        if st != 6:  # a timed-out request keeps its buffers alive
            self._keep.pop(int(rid), None)
        _check(st)
        return {"status": info.status, "t_submit": info.t_submit, "t_admit": info.t_admit, "t_done": info.t_done,
                "device_bytes": int(info.device_bytes)}

    def stats(self) -> dict:
        s = ServerStats()
        _check(load_library().cbct_server_stats_get(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _check(load_library().cbct_server_destroy(self._h))
            self._h = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
