"""Python binding of the GB300 FLD solver library (argument marshalling only).

Every function here forwards to the C ABI declared in ``include/fld.h``, with
the same name; all computation runs in the CUDA kernels of
``libfld_gb300.so``.  There is no CPU fallback: if the library cannot be
loaded, or no GPU is present, the calls raise.

Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); CUDA tensors are passed to the library as device pointers.
Unpadded fields are float32 of shape (nz, ny, nx); padded state fields
(phi, D) are float64 of shape (nz+2, ny+2, nx+2).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

__all__ = [
    "FLD_OK", "FLD_ERR_INVALID_ARG", "FLD_ERR_OOM", "FLD_ERR_CUDA", "FLD_ERR_STATE",
    "FLD_ERR_NOT_CONVERGED", "FLD_ERR_DIVERGED", "FLD_ERR_NO_DEVICE", "FLD_ERR_TIMEOUT",
    "LIMITERS", "PRECISIONS", "FldError", "SolveParams", "SolveResult",
    "load", "library_path", "fld_default_params", "fld_create_grid", "fld_set_medium", "fld_set_source",
    "fld_get_source", "fld_bake_directional", "fld_bake_point", "fld_set_state", "fld_get_state",
    "fld_iterate", "fld_solve", "fld_solve_batch", "fld_residual", "fld_residual_noalloc", "fld_destroy",
    "fld_server_create", "fld_server_add", "fld_server_step", "fld_server_active", "fld_server_destroy",
    "fld_server_updates",
    "Server", "fld_status_string",
    "fld_last_error", "Grid", "params",
]

FLD_OK, FLD_ERR_INVALID_ARG, FLD_ERR_OOM, FLD_ERR_CUDA, FLD_ERR_STATE = 0, 1, 2, 3, 4
FLD_ERR_NOT_CONVERGED, FLD_ERR_DIVERGED, FLD_ERR_NO_DEVICE, FLD_ERR_TIMEOUT = 5, 6, 7, 8
FLD_MEM_HOST, FLD_MEM_DEVICE = 0, 1
LIMITERS = {"cda": 0, "sum": 1, "max": 2, "kershaw": 3, "larsen": 4, "lp": 5}
PRECISIONS = {"fp64": 0, "fp32": 1, "mixed": 2, "pair": 3}
SCHEMES = {"red_black": 0, "rb": 0, "jacobi": 1}


class SolveParams(ctypes.Structure):
    """Mirror of fld_solve_params (fld.h)."""
    _fields_ = [
        ("limiter", ctypes.c_int), ("larsen_n", ctypes.c_double), ("omega", ctypes.c_double),
        ("local_iters", ctypes.c_int), ("tol", ctypes.c_double), ("max_iters", ctypes.c_int),
        ("check_every", ctypes.c_int), ("sigma_eps", ctypes.c_double), ("eps", ctypes.c_double),
        ("precision", ctypes.c_int), ("fp32_switch", ctypes.c_double), ("residual_margin", ctypes.c_int),
        ("warm_start", ctypes.c_int), ("phi0", ctypes.c_double), ("D0", ctypes.c_double),
        ("phi_b", ctypes.c_double), ("D_b", ctypes.c_double), ("warmup_iters", ctypes.c_int),
        ("medium_bf16", ctypes.c_int), ("scheme", ctypes.c_int), ("nested", ctypes.c_int),
        ("anderson", ctypes.c_int), ("fp64_verify", ctypes.c_int), ("temporal_depth", ctypes.c_int),
        ("tile_y", ctypes.c_int), ("cells_per_thread", ctypes.c_int), ("batch_launch", ctypes.c_int),
    ]


class SolveResult(ctypes.Structure):
    """Mirror of fld_solve_result (fld.h)."""
    _fields_ = [
        ("status", ctypes.c_int), ("iterations", ctypes.c_int), ("iterations_fp32", ctypes.c_int),
        ("iterations_corr", ctypes.c_int), ("checks", ctypes.c_int), ("rel_residual", ctypes.c_double),
        ("jbar", ctypes.c_double), ("omega", ctypes.c_double), ("ms", ctypes.c_double),
        ("ms_sweep_fp32", ctypes.c_double), ("ms_sweep_corr", ctypes.c_double), ("kernels", ctypes.c_longlong),
        ("omega_backoffs", ctypes.c_int), ("iterations_mid", ctypes.c_int), ("ms_sweep_mid", ctypes.c_double),
        ("iterations_coarse", ctypes.c_int), ("ms_coarse", ctypes.c_double), ("updates_coarse", ctypes.c_longlong),
        ("anderson_steps", ctypes.c_int), ("anderson_resets", ctypes.c_int),
        ("iterations_fp64", ctypes.c_int), ("ms_sweep_fp64", ctypes.c_double),
        ("rel_residual_single", ctypes.c_double),
    ]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Camera(ctypes.Structure):
    """Mirror of fld_camera (fld.h)."""
    _fields_ = [
        ("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
        ("fov_deg", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int),
        ("step", ctypes.c_double), ("background", ctypes.c_double), ("t_min", ctypes.c_double),
    ]


def camera(eye, target, up=(0.0, 1.0, 0.0), fov_deg=40.0, width=1024, height=1024, step=0.0, background=0.0,
           t_min=-1.0) -> Camera:
    c = Camera()
    c.eye[:] = [float(v) for v in eye]
    c.target[:] = [float(v) for v in target]
    c.up[:] = [float(v) for v in up]
    c.fov_deg, c.width, c.height = float(fov_deg), int(width), int(height)
    c.step, c.background, c.t_min = float(step), float(background), float(t_min)
    return c


class FldError(RuntimeError):
    def __init__(self, status: int, func: str, detail: str):
        self.status = status
        super().__init__(f"{func}: {_STATUS_NAMES.get(status, status)}: {detail}")


_STATUS_NAMES = {0: "FLD_OK", 1: "FLD_ERR_INVALID_ARG", 2: "FLD_ERR_OOM", 3: "FLD_ERR_CUDA",
                 4: "FLD_ERR_STATE", 5: "FLD_ERR_NOT_CONVERGED", 6: "FLD_ERR_DIVERGED", 7: "FLD_ERR_NO_DEVICE",
                 8: "FLD_ERR_TIMEOUT"}

_lib = None
_lock = threading.Lock()
_vp = ctypes.c_void_p
_dp3 = ctypes.c_double * 3


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libfld_gb300.so (building it with nvcc if it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"FLD CUDA library not built: {path}")
            _build.build()
        lib = ctypes.CDLL(path)
        c_int, c_double = ctypes.c_int, ctypes.c_double
        P, R = ctypes.POINTER(SolveParams), ctypes.POINTER(SolveResult)
        sig = {
            "fld_default_params": (None, [P]),
            "fld_create_grid": (c_int, [c_int, c_int, c_int, c_double, _vp, ctypes.POINTER(_vp)]),
            "fld_set_medium": (c_int, [_vp, _vp, _vp, c_int]),
            "fld_set_source": (c_int, [_vp, _vp, c_int]),
            "fld_get_source": (c_int, [_vp, _vp, c_int]),
            "fld_bake_directional": (c_int, [_vp, _dp3, c_double, c_double, c_int]),
            "fld_bake_point": (c_int, [_vp, _dp3, c_double, c_double, c_int]),
            "fld_set_state": (c_int, [_vp, _vp, _vp, c_int]),
            "fld_get_state": (c_int, [_vp, _vp, _vp, c_int]),
            "fld_iterate": (c_int, [_vp, P, c_int]),
            "fld_solve": (c_int, [_vp, P, R]),
            "fld_solve_batch": (c_int, [ctypes.POINTER(_vp), c_int, P, R]),
            "fld_server_create": (c_int, [P, _vp, ctypes.POINTER(_vp)]),
            "fld_server_add": (c_int, [_vp, _vp, ctypes.c_longlong]),
            "fld_server_step": (c_int, [_vp, ctypes.POINTER(ctypes.c_longlong), R, c_int,
                                        ctypes.POINTER(c_int)]),
            "fld_server_active": (c_int, [_vp, ctypes.POINTER(c_int)]),
            "fld_server_updates": (c_int, [_vp, ctypes.POINTER(ctypes.c_longlong)]),
            "fld_server_destroy": (None, [_vp]),
            "fld_residual": (c_int, [_vp, P, ctypes.POINTER(c_double)]),
            "fld_residual_noalloc": (c_int, [c_int, c_int, c_int, c_double, P, _vp, _vp, _vp, _vp, _vp,
                                             ctypes.POINTER(c_double), _vp]),
            "fld_render": (c_int, [_vp, _vp, ctypes.POINTER(Camera), _vp, _vp, c_double, c_double, c_int]),
            "fld_downsample": (c_int, [_vp, _vp, c_int]),
            "fld_destroy": (None, [_vp]),
            "fld_status_string": (ctypes.c_char_p, [c_int]),
            "fld_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _check(status: int, func: str, allow=(FLD_OK,)):
    if status not in allow:
        raise FldError(status, func, fld_last_error())
    return status


def _ptr(a, dtype):
    """(pointer, where, keepalive) of a numpy array or torch tensor."""
    try:
        import torch  # noqa: F401
        is_tensor = type(a).__module__.startswith("torch")
    except ImportError:  # pragma: no cover
        is_tensor = False
    if is_tensor:
        import torch
        want = {np.float32: torch.float32, np.float64: torch.float64, np.uint8: torch.uint8}[dtype]
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {want} tensor")
        return ctypes.c_void_p(a.data_ptr()), (FLD_MEM_DEVICE if a.is_cuda else FLD_MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return ctypes.c_void_p(arr.ctypes.data), FLD_MEM_HOST, arr


# ---------------------------------------------------------------------------
# The ABI, one wrapper per entry point
# ---------------------------------------------------------------------------

def fld_default_params() -> SolveParams:
    p = SolveParams()
    load().fld_default_params(ctypes.byref(p))
    return p


def fld_status_string(status: int) -> str:
    return load().fld_status_string(int(status)).decode()


def fld_last_error() -> str:
    return load().fld_last_error().decode()


def fld_create_grid(nx: int, ny: int, nz: int, h: float, stream=None) -> ctypes.c_void_p:
    out = _vp()
    s = None if stream is None else _vp(int(stream))
    _check(load().fld_create_grid(int(nx), int(ny), int(nz), float(h), s, ctypes.byref(out)), "fld_create_grid")
    return out


def fld_set_medium(g, sigma_t, albedo) -> None:
    ps, w1, k1 = _ptr(sigma_t, np.float32)
    pa, w2, k2 = _ptr(albedo, np.float32)
    if w1 != w2:
        raise ValueError("sigma_t and albedo must live in the same kind of memory")
    _check(load().fld_set_medium(g, ps, pa, w1), "fld_set_medium")


def fld_set_source(g, j) -> None:
    pj, w, k = _ptr(j, np.float32)
    _check(load().fld_set_source(g, pj, w), "fld_set_source")


def fld_get_source(g, out) -> None:
    pj, w, k = _ptr(out, np.float32)
    _check(load().fld_get_source(g, pj, w), "fld_get_source")


def fld_downsample(fine, coarse, factor: int = 4) -> None:
    _check(load().fld_downsample(fine, coarse, int(factor)), "fld_downsample")


def fld_render(g, phi_grid, cam: Camera, radiance=None, codes=None, exposure: float = 1.0,
               gamma: float = 2.2) -> None:
    pr, w1, k1 = _ptr(radiance, np.float32) if radiance is not None else (None, None, None)
    pc, w2, k2 = _ptr(codes, np.uint8) if codes is not None else (None, None, None)
    ws = {w for w in (w1, w2) if w is not None}
    if len(ws) > 1:
        raise ValueError("radiance and codes must live in the same kind of memory")
    _check(load().fld_render(g, phi_grid, ctypes.byref(cam), pr, pc, float(exposure), float(gamma),
                             ws.pop() if ws else FLD_MEM_HOST), "fld_render")


def fld_bake_directional(g, direction, radiance: float = 1.0, step: float = 0.0, accumulate: int = 0) -> None:
    _check(load().fld_bake_directional(g, _dp3(*map(float, direction)), float(radiance), float(step),
                                       int(accumulate)), "fld_bake_directional")


def fld_bake_point(g, pos, power: float = 1.0, step: float = 0.0, accumulate: int = 0) -> None:
    _check(load().fld_bake_point(g, _dp3(*map(float, pos)), float(power), float(step), int(accumulate)),
           "fld_bake_point")


def fld_set_state(g, phi=None, D=None) -> None:
    pp, w1, k1 = _ptr(phi, np.float64) if phi is not None else (None, None, None)
    pd, w2, k2 = _ptr(D, np.float64) if D is not None else (None, None, None)
    ws = {w for w in (w1, w2) if w is not None}
    if len(ws) > 1:
        raise ValueError("phi and D must live in the same kind of memory")
    _check(load().fld_set_state(g, pp, pd, ws.pop() if ws else FLD_MEM_HOST), "fld_set_state")


def fld_get_state(g, phi=None, D=None) -> None:
    pp, w1, k1 = _ptr(phi, np.float64) if phi is not None else (None, None, None)
    pd, w2, k2 = _ptr(D, np.float64) if D is not None else (None, None, None)
    if phi is not None and w1 == FLD_MEM_HOST and not isinstance(phi, np.ndarray):
        raise TypeError("host outputs must be numpy arrays or CPU tensors")
    ws = {w for w in (w1, w2) if w is not None}
    if len(ws) > 1:
        raise ValueError("phi and D must live in the same kind of memory")
    _check(load().fld_get_state(g, pp, pd, ws.pop() if ws else FLD_MEM_HOST), "fld_get_state")
    for out, keep in ((phi, k1), (D, k2)):
        if out is not None and isinstance(out, np.ndarray) and keep is not out:
            out[...] = keep


def fld_iterate(g, p: SolveParams, iterations: int) -> None:
    _check(load().fld_iterate(g, ctypes.byref(p), int(iterations)), "fld_iterate")


def fld_solve(g, p: SolveParams, check: bool = True) -> SolveResult:
    r = SolveResult()
    st = load().fld_solve(g, ctypes.byref(p), ctypes.byref(r))
    if check:
        _check(st, "fld_solve", allow=(FLD_OK, FLD_ERR_NOT_CONVERGED, FLD_ERR_DIVERGED))
    r.status = st
    return r


def fld_solve_batch(grids, p: SolveParams, check: bool = True):
    """Solve several grids together; returns (status, [SolveResult per grid])."""
    n = len(grids)
    arr = (_vp * n)(*[g.handle if isinstance(g, Grid) else g for g in grids])
    out = (SolveResult * n)()
    st = load().fld_solve_batch(arr, n, ctypes.byref(p), out)
    if check:
        _check(st, "fld_solve_batch", allow=(FLD_OK, FLD_ERR_NOT_CONVERGED, FLD_ERR_DIVERGED))
    return st, list(out)


def fld_server_create(p: SolveParams, stream=None):
    out = _vp()
    s = None if stream is None else _vp(int(stream))
    _check(load().fld_server_create(ctypes.byref(p), s, ctypes.byref(out)), "fld_server_create")
    return out


def fld_server_add(s, g, tag: int) -> None:
    _check(load().fld_server_add(s, g.handle if isinstance(g, Grid) else g, int(tag)), "fld_server_add")


def fld_server_step(s, capacity: int = 256):
    """One step; returns [(tag, SolveResult)] of the grids that finished."""
    tags = (ctypes.c_longlong * max(1, capacity))()
    res = (SolveResult * max(1, capacity))()
    n = ctypes.c_int(0)
    _check(load().fld_server_step(s, tags, res, int(capacity), ctypes.byref(n)), "fld_server_step")
    return [(int(tags[i]), res[i]) for i in range(n.value)]


def fld_server_updates(s) -> int:
    n = ctypes.c_longlong(0)
    _check(load().fld_server_updates(s, ctypes.byref(n)), "fld_server_updates")
    return n.value


def fld_server_active(s) -> int:
    n = ctypes.c_int(0)
    _check(load().fld_server_active(s, ctypes.byref(n)), "fld_server_active")
    return n.value


def fld_server_destroy(s) -> None:
    if s:
        load().fld_server_destroy(s)


class Server:
    """Owning wrapper of an fld_server handle."""

    def __init__(self, p: SolveParams, stream=None):
        self.handle = fld_server_create(p, stream)

    def add(self, grid, tag: int):
        fld_server_add(self.handle, grid, tag)

    def step(self, capacity: int = 256):
        return fld_server_step(self.handle, capacity)

    @property
    def active(self) -> int:
        return fld_server_active(self.handle)

    @property
    def updates(self) -> int:
        return fld_server_updates(self.handle)

    def close(self):
        if self.handle:
            fld_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fld_residual(g, p: SolveParams) -> float:
    rel = ctypes.c_double(0.0)
    _check(load().fld_residual(g, ctypes.byref(p), ctypes.byref(rel)), "fld_residual")
    return rel.value


def fld_residual_noalloc(nx: int, ny: int, nz: int, h: float, p: SolveParams, sigma_t, albedo, j, phi, D,
                         stream=None) -> float:
    """Allocation-free FP64 residual from caller-owned CUDA tensors (float32
    sigma_t, albedo, j of shape (nz, ny, nx); float64 phi, D padded)."""
    args = []
    for a, dt in ((sigma_t, np.float32), (albedo, np.float32), (j, np.float32), (phi, np.float64),
                  (D, np.float64)):
        ptr, where, keep = _ptr(a, dt)
        if where != FLD_MEM_DEVICE:
            raise TypeError("fld_residual_noalloc takes device buffers (CUDA tensors)")
        args.append(ptr)
    rel = ctypes.c_double(0.0)
    s = None if stream is None else _vp(int(stream))
    _check(load().fld_residual_noalloc(int(nx), int(ny), int(nz), float(h), ctypes.byref(p), *args,
                                       ctypes.byref(rel), s), "fld_residual_noalloc")
    return rel.value


def fld_destroy(g) -> None:
    if g:
        load().fld_destroy(g)


# ---------------------------------------------------------------------------
# Convenience
# ---------------------------------------------------------------------------

def params(**kw) -> SolveParams:
    """fld_default_params() with fields overridden by keyword; `limiter` and
    `precision` also accept their names ("lp", "mixed", ...)."""
    p = fld_default_params()
    for k, v in kw.items():
        if k == "limiter" and isinstance(v, str):
            v = LIMITERS[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "scheme" and isinstance(v, str):
            v = SCHEMES[v]
        if not hasattr(p, k):
            raise AttributeError(f"SolveParams has no field {k!r}")
        setattr(p, k, v)
    return p


class Grid:
    """Owning wrapper of an fld_grid handle."""

    def __init__(self, nx: int, ny: int, nz: int, h: float, stream=None):
        self.shape = (nz, ny, nx)
        self.h = h
        self.handle = fld_create_grid(nx, ny, nz, h, stream)

    def close(self):
        if self.handle:
            fld_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    @property
    def padded_shape(self):
        nz, ny, nx = self.shape
        return (nz + 2, ny + 2, nx + 2)

    def set_medium(self, sigma_t, albedo):
        fld_set_medium(self.handle, sigma_t, albedo)

    def set_source(self, j):
        fld_set_source(self.handle, j)

    def get_source(self):
        out = np.empty(self.shape, np.float32)
        fld_get_source(self.handle, out)
        return out

    def bake_directional(self, direction=(0.0, 0.0, -1.0), radiance=1.0, step=0.0, accumulate=0):
        fld_bake_directional(self.handle, direction, radiance, step, accumulate)

    def bake_point(self, pos, power=1.0, step=0.0, accumulate=0):
        fld_bake_point(self.handle, pos, power, step, accumulate)

    def render(self, cam: Camera, exposure=1.0, gamma=2.2, codes=False, phi_grid=None):
        """(radiance, codes or None) as host arrays of shape (height, width);
        phi_grid: a coarser solved Grid to take phi from (upsampled)."""
        rad = np.empty((cam.height, cam.width), np.float32)
        cod = np.empty((cam.height, cam.width), np.uint8) if codes else None
        fld_render(self.handle, phi_grid.handle if phi_grid is not None else None, cam, rad, cod, exposure, gamma)
        return rad, cod

    def downsample_to(self, coarse: "Grid", factor: int = 4):
        """Set coarse's medium and source from this grid's (box averages)."""
        fld_downsample(self.handle, coarse.handle, factor)

    def set_state(self, phi=None, D=None):
        fld_set_state(self.handle, phi, D)

    def get_state(self):
        phi = np.empty(self.padded_shape, np.float64)
        D = np.empty(self.padded_shape, np.float64)
        fld_get_state(self.handle, phi, D)
        return phi, D

    def iterate(self, p: SolveParams, iterations: int):
        fld_iterate(self.handle, p, iterations)

    def solve(self, p: SolveParams, check: bool = True) -> SolveResult:
        return fld_solve(self.handle, p, check)

    def residual(self, p: SolveParams) -> float:
        return fld_residual(self.handle, p)
