"""FP64 CPU oracle for the FLD solver -- TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It shares no code with the CUDA path
(`paper_1403_8105_gb300`), and the CUDA path never imports it.

The arithmetic lives in `fld_oracle.c` (plain C, double precision, written
from Koerner et al. 2014, Sec. 3-5 and Algorithm 1); this module compiles it
with gcc on first use and wraps it with numpy arrays.

Array conventions (same as `fld_inputs`): unpadded fields are shape
(nz, ny, nx); padded fields (phi, D) are shape (nz+2, ny+2, nx+2) with the
Dirichlet ghost layer on the outside.

Parity notes: every function here follows the paper's formula or algorithm
step by step; "parity unpinned" items are listed in the design notes (the
heterogeneous fixed points have no printed values in the paper and are pinned
only through the tiny-grid brute-force solves, invariants and closed forms in
`tests/test_oracle_*.py`).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fld_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libfld_oracle.so")
_lock = threading.Lock()
_lib = None

LIMITERS = {"cda": 0, "sum": 1, "max": 2, "kershaw": 3, "larsen": 4, "lp": 5}
EPS = 1e-20          # epsilon of Eq. 35
_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)
_ip = ctypes.POINTER(ctypes.c_int)


class _Camera(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_double * 3), ("target", ctypes.c_double * 3), ("up", ctypes.c_double * 3),
                ("fov_deg", ctypes.c_double), ("width", ctypes.c_int), ("height", ctypes.c_int),
                ("step", ctypes.c_double), ("background", ctypes.c_double), ("t_min", ctypes.c_double)]


class _Cfg(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
                ("h", ctypes.c_double), ("limiter", ctypes.c_int), ("larsen_n", ctypes.c_double),
                ("eps", ctypes.c_double), ("jbar", ctypes.c_double), ("omega", ctypes.c_double),
                ("nthreads", ctypes.c_int), ("local_iters", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE double, no FMA contraction so the
    x86 and Arm builds round identically)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off", "-fno-fast-math",
               "-shared", "-fPIC", "-o", tmp, _SRC, "-lpthread", "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.fldo_limiter.restype = ctypes.c_double
            lib.fldo_limiter.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.fldo_prep.restype = None
            lib.fldo_prep.argtypes = [ctypes.c_long, _fp, _fp, ctypes.c_double, _dp, _dp]
            lib.fldo_prep_bf16.restype = None
            lib.fldo_prep_bf16.argtypes = [ctypes.c_long, _fp, _fp, ctypes.c_double, _dp, _dp]
            lib.fldo_rms.restype = ctypes.c_double
            lib.fldo_rms.argtypes = [ctypes.c_long, _dp]
            lib.fldo_rb_iteration.restype = None
            lib.fldo_rb_iteration.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp]
            lib.fldo_render.restype = None
            lib.fldo_render.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp,
                                        _dp, ctypes.POINTER(_Camera), _dp, ctypes.c_int]
            lib.fldo_render_pixels.restype = None
            lib.fldo_render_pixels.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp,
                                               _dp, _dp, ctypes.POINTER(_Camera), _ip, _ip, ctypes.c_long, _dp]
            lib.fldo_downsample.restype = None
            lib.fldo_downsample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _fp, _fp, _dp,
                                            _dp, _dp, _dp]
            lib.fldo_upsample.restype = None
            lib.fldo_upsample.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                          _dp, _dp]
            lib.fldo_jacobi_iteration.restype = None
            lib.fldo_jacobi_iteration.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp, _dp]
            lib.fldo_pass.restype = None
            lib.fldo_pass.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp, ctypes.c_int]
            lib.fldo_residual.restype = ctypes.c_double
            lib.fldo_residual.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp, ctypes.c_int,
                                          _dp, ctypes.POINTER(ctypes.c_long), _dp]
            lib.fldo_residual_at.restype = ctypes.c_double
            lib.fldo_residual_at.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_int]
            lib.fldo_solve.restype = ctypes.c_int
            lib.fldo_solve.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp, _dp, _dp, ctypes.c_double,
                                       ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                       ctypes.POINTER(ctypes.c_int)]
            lib.fldo_bake_directional.restype = None
            lib.fldo_bake_directional.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                  _fp, _fp, _dp, ctypes.c_double, ctypes.c_double,
                                                  ctypes.c_int, _dp]
            lib.fldo_limiter_array.restype = None
            lib.fldo_limiter_array.argtypes = [ctypes.c_int, ctypes.c_double, _dp, _dp, ctypes.c_long]
            lib.fldo_flux.restype = None
            lib.fldo_flux.argtypes = [ctypes.POINTER(_Cfg), _dp, _dp, _dp]
            lib.fldo_bake_point.restype = None
            lib.fldo_bake_point.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                            _fp, _fp, _dp, ctypes.c_double, ctypes.c_double,
                                            ctypes.c_int, _dp]
            _lib = lib
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags.c_contiguous
    return a.ctypes.data_as(_fp)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


# --------------------------------------------------------------------------
# Limiters (Table 2)
# --------------------------------------------------------------------------

def limiter(kind: str, R, larsen_n: float = 2.0):
    """F(R) for one of "cda", "sum", "max", "kershaw", "larsen", "lp"."""
    lib = _load()
    k = LIMITERS[kind]
    Rs = np.ascontiguousarray(R, dtype=np.float64)
    if Rs.ndim == 0:
        return float(lib.fldo_limiter(k, float(larsen_n), float(Rs)))
    out = np.empty_like(Rs)
    lib.fldo_limiter_array(k, float(larsen_n), _d(Rs), _d(out), Rs.size)
    return out


# --------------------------------------------------------------------------
# Problem state
# --------------------------------------------------------------------------

@dataclasses.dataclass
class Problem:
    """Inputs of Algorithm 1 after its first three steps, plus the state."""
    nx: int
    ny: int
    nz: int
    h: float
    sp: np.ndarray      # sigma' = max(sigma_t, sigma_eps), (nz, ny, nx) float64
    sa: np.ndarray      # sigma_a' = (1 - albedo) sigma'
    j: np.ndarray       # emission incl. q_ri
    jbar: float
    limiter: str = "lp"
    larsen_n: float = 2.0
    omega: float = 1.0
    eps: float = EPS
    phi: np.ndarray | None = None   # padded
    D: np.ndarray | None = None     # padded
    nthreads: int = 1
    local_iters: int = 1

    def cfg(self) -> _Cfg:
        return _Cfg(self.nx, self.ny, self.nz, float(self.h), LIMITERS[self.limiter], float(self.larsen_n),
                    float(self.eps), float(self.jbar), float(self.omega), int(self.nthreads),
                    int(self.local_iters))


def sigma_eps_default(nx: int, ny: int, nz: int, h: float) -> float:
    """sigma_eps = 1e-3 / L with L the largest grid extent (Sec. 5)."""
    return 1e-3 / (max(nx, ny, nz) * h)


def omega_default(nx: int, ny: int, nz: int) -> float:
    """SOR factor used when none is given: the Laplacian estimate
    2 / (1 + sin(pi / (n + 1))) for the largest extent n, clamped to
    [1, 1.95].  The paper only requires 0 < omega < 2 (Eq. 36)."""
    n = max(nx, ny, nz)
    w = 2.0 / (1.0 + np.sin(np.pi / (n + 1)))
    return float(min(1.95, max(1.0, w)))


def make_problem(sigma_t: np.ndarray, albedo: np.ndarray, j: np.ndarray, h: float, *,
                 limiter: str = "lp", larsen_n: float = 2.0, omega: float | None = None,
                 sigma_eps: float | None = None, eps: float = EPS, nthreads: int | None = None,
                 local_iters: int = 1, medium_bf16: bool = False) -> Problem:
    """Algorithm 1, first three steps: floor sigma, compute sigma_a' and jbar.
    medium_bf16: sigma' and sigma_a' formed in single precision and rounded
    to bfloat16 (nearest, ties to even), then used exactly."""
    lib = _load()
    sigma_t = np.ascontiguousarray(sigma_t, dtype=np.float32)
    albedo = np.ascontiguousarray(albedo, dtype=np.float32)
    nz, ny, nx = sigma_t.shape
    if sigma_eps is None:
        sigma_eps = sigma_eps_default(nx, ny, nz, h)
    sp = np.empty(sigma_t.shape, dtype=np.float64)
    sa = np.empty(sigma_t.shape, dtype=np.float64)
    prep = lib.fldo_prep_bf16 if medium_bf16 else lib.fldo_prep
    prep(sigma_t.size, _f(sigma_t), _f(albedo), float(sigma_eps), _d(sp), _d(sa))
    jd = np.ascontiguousarray(j, dtype=np.float64)
    jbar = lib.fldo_rms(jd.size, _d(jd))
    if omega is None:
        omega = omega_default(nx, ny, nz)
    return Problem(nx, ny, nz, float(h), sp, sa, jd, float(jbar), limiter, larsen_n, float(omega), eps,
                   None, None, nthreads or default_threads(), int(local_iters))


def init_state(p: Problem, phi0: float | None = None, D0: float | None = None,
               phi_b: float | None = None, D_b: float | None = None) -> None:
    """Algorithm 1 initialisation: phi = eps*jbar*dl, D = eps*dl everywhere,
    including the Dirichlet ghost layer, unless values are given."""
    pd = p.eps * p.jbar * p.h
    dd = p.eps * p.h
    shape = (p.nz + 2, p.ny + 2, p.nx + 2)
    p.phi = np.full(shape, pd if phi_b is None else phi_b, dtype=np.float64)
    p.D = np.full(shape, dd if D_b is None else D_b, dtype=np.float64)
    p.phi[1:-1, 1:-1, 1:-1] = pd if phi0 is None else phi0
    p.D[1:-1, 1:-1, 1:-1] = dd if D0 is None else D0


def rb_iteration(p: Problem, iters: int = 1) -> None:
    lib = _load()
    c = p.cfg()
    for _ in range(iters):
        lib.fldo_rb_iteration(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(p.phi), _d(p.D))


def colour_pass(p: Problem, colour: int) -> None:
    lib = _load()
    c = p.cfg()
    lib.fldo_pass(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(p.phi), _d(p.D), int(colour))


def jacobi_iteration(p: Problem, iters: int = 1):
    """Jacobi iterations (D^k from phi^k everywhere, then phi^{k+1} from
    phi^k and D^k, damped by p.omega); p.phi and p.D are updated."""
    lib = _load()
    c = p.cfg()
    nxt = np.empty_like(p.phi)
    for _ in range(iters):
        lib.fldo_jacobi_iteration(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(p.phi), _d(p.D), _d(nxt))
        p.phi, nxt = nxt, p.phi


def render(sigma_t: np.ndarray, albedo: np.ndarray, q: np.ndarray, phi: np.ndarray, h: float, *,
           eye, target, up=(0.0, 1.0, 0.0), fov_deg: float = 40.0, width: int = 64, height: int = 64,
           step: float | None = None, background: float = 0.0, t_min: float = 1e-6,
           nthreads: int | None = None, pixels=None) -> np.ndarray:
    """Primary ray march (Sec. 3): radiance per pixel, shape (height, width),
    row 0 at the top (or, with pixels = [(px, py), ...], of those pixels
    only).  sigma_t, albedo, q (the solver's source: q_ri + j) are unpadded;
    phi is unpadded or padded (the ghost layer is dropped)."""
    lib = _load()
    sigma_t = np.asarray(sigma_t, dtype=np.float32)
    nz, ny, nx = sigma_t.shape
    st = np.ascontiguousarray(sigma_t, dtype=np.float64)
    ss = np.ascontiguousarray(np.asarray(albedo, dtype=np.float32).astype(np.float64) * st)
    qd = np.ascontiguousarray(q, dtype=np.float64)
    ph = np.asarray(phi, dtype=np.float64)
    if ph.shape == (nz + 2, ny + 2, nx + 2):
        ph = ph[1:-1, 1:-1, 1:-1]
    ph = np.ascontiguousarray(ph)
    cam = _Camera()
    cam.eye[:] = [float(v) for v in eye]
    cam.target[:] = [float(v) for v in target]
    cam.up[:] = [float(v) for v in up]
    cam.fov_deg, cam.width, cam.height = float(fov_deg), int(width), int(height)
    cam.step = float(step) if step else 0.5 * h
    cam.background, cam.t_min = float(background), float(t_min)
    if pixels is not None:
        pxs = np.ascontiguousarray([p[0] for p in pixels], dtype=np.int32)
        pys = np.ascontiguousarray([p[1] for p in pixels], dtype=np.int32)
        out = np.zeros(len(pxs), dtype=np.float64)
        lib.fldo_render_pixels(nx, ny, nz, float(h), _d(st), _d(ss), _d(qd), _d(ph), ctypes.byref(cam),
                               pxs.ctypes.data_as(_ip), pys.ctypes.data_as(_ip), len(pxs), _d(out))
        return out
    img = np.zeros((height, width), dtype=np.float64)
    lib.fldo_render(nx, ny, nz, float(h), _d(st), _d(ss), _d(qd), _d(ph), ctypes.byref(cam), _d(img),
                    int(nthreads or default_threads()))
    return img


def downsample(sigma_t: np.ndarray, albedo: np.ndarray, q: np.ndarray, factor: int = 4):
    """Box averages over factor^3 blocks (Sec. 6.2's quarter-resolution solve):
    returns (sigma_t_c, albedo_c, q_c) on the ceil(n / factor) grid."""
    lib = _load()
    sigma_t = np.ascontiguousarray(sigma_t, dtype=np.float32)
    albedo = np.ascontiguousarray(albedo, dtype=np.float32)
    qd = np.ascontiguousarray(q, dtype=np.float64)
    nz, ny, nx = sigma_t.shape
    f = int(factor)
    shp = ((nz + f - 1) // f, (ny + f - 1) // f, (nx + f - 1) // f)
    st, al, qc = (np.zeros(shp), np.zeros(shp), np.zeros(shp))
    lib.fldo_downsample(nx, ny, nz, f, _f(sigma_t), _f(albedo), _d(qd), _d(st), _d(al), _d(qc))
    return st, al, qc


def upsample(phi_c: np.ndarray, fine_shape, h: float, factor: int = 4) -> np.ndarray:
    """phi of the coarse grid (unpadded or padded) at the fine voxel centres."""
    lib = _load()
    nz, ny, nx = fine_shape
    f = int(factor)
    shp = ((nz + f - 1) // f, (ny + f - 1) // f, (nx + f - 1) // f)
    pc = np.asarray(phi_c, dtype=np.float64)
    if pc.shape == tuple(s + 2 for s in shp):
        pc = pc[1:-1, 1:-1, 1:-1]
    pc = np.ascontiguousarray(pc)
    out = np.zeros((nz, ny, nx))
    lib.fldo_upsample(nx, ny, nz, float(h), f, _d(pc), _d(out))
    return out


def tonemap(radiance: np.ndarray, exposure: float = 1.0, gamma: float = 2.2, dtype=np.float64) -> np.ndarray:
    """Gamma compression to 8 bits (Sec. 6.2): round(255 clamp((e L)^(1/gamma), 0, 1)).
    dtype: the precision the rounding decision is taken in (the paper fixes
    none; comparisons with the GPU's codes take it in float32, the kernel's)."""
    t = np.dtype(dtype).type
    v = np.clip(t(exposure) * np.asarray(radiance, dtype=dtype), t(0.0), None) ** t(1.0 / gamma)
    return np.floor(t(255.0) * np.clip(v, t(0.0), t(1.0)) + t(0.5)).astype(np.uint8)


def residual(p: Problem, phi: np.ndarray | None = None, margin: int = 0, field: bool = False):
    """Relative residual Rbar/jbar with D recomputed from phi (Eq. 37).

    Returns (rel, sum_R2, count[, R field])."""
    lib = _load()
    c = p.cfg()
    ph = p.phi if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    s = ctypes.c_double(0.0)
    cnt = ctypes.c_long(0)
    R = np.empty((p.nz, p.ny, p.nx), dtype=np.float64) if field else None
    rel = lib.fldo_residual(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(ph), _d(p.D), int(margin),
                            ctypes.byref(s), ctypes.byref(cnt), _d(R) if field else None)
    if field:
        return rel, s.value, cnt.value, R
    return rel, s.value, cnt.value


def residual_at(p: Problem, phi: np.ndarray, i: int, j: int, k: int) -> float:
    """R_p at one unknown with D recomputed locally (Eq. 37)."""
    lib = _load()
    c = p.cfg()
    ph = np.ascontiguousarray(phi, dtype=np.float64)
    return lib.fldo_residual_at(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(ph), _d(p.D),
                                int(i), int(j), int(k))


def solve(p: Problem, tol: float = 1e-10, max_iters: int = 100000, check_every: int = 10,
          margin: int = 0):
    """Algorithm 1 until Rbar/jbar <= tol.  Returns (iterations, rel, history)."""
    lib = _load()
    c = p.cfg()
    nh_max = max_iters // max(1, check_every) + 2
    hist = np.zeros(nh_max, dtype=np.float64)
    rel = ctypes.c_double(0.0)
    nh = ctypes.c_int(0)
    it = lib.fldo_solve(ctypes.byref(c), _d(p.sp), _d(p.sa), _d(p.j), _d(p.phi), _d(p.D), float(tol),
                        int(max_iters), int(check_every), int(margin), ctypes.byref(rel), _d(hist),
                        ctypes.byref(nh))
    return it, rel.value, hist[: nh.value].copy()


def solve_anderson(p: Problem, tol: float, sweeps_per_block: int = 16, m: int = 8,
                   max_sweeps: int = 400000):
    """The fixed point of Algorithm 1 reached faster, for reference solutions
    of grids where plain SOR takes too long (not in the paper).

    A block of `sweeps_per_block` red-black iterations (`rb_iteration`) is a
    map G whose fixed point is the solution of Eq. 31.  Each block starts
    from the affine combination x = sum a_i G(x_i) of the last m block images
    with sum a_i = 1 and the a minimising |sum a_i (G(x_i) - x_i)| (Anderson
    mixing, Walker & Ni 2011); the unknowns only are mixed, the Dirichlet
    ghosts stay as set.  Stops when the fresh-D residual of Eq. 37 is <= tol,
    so the result is judged by the same definition as `solve`.  Returns
    (sweeps, rel)."""
    inner = (slice(1, -1),) * 3
    x = p.phi[inner].copy()
    G, F = [], []
    sweeps = 0
    while sweeps < max_sweeps:
        rb_iteration(p, sweeps_per_block)
        sweeps += sweeps_per_block
        rel = residual(p)[0]
        if rel <= tol:
            return sweeps, rel
        g = p.phi[inner].copy()
        G.append(g)
        F.append(g - x)
        G, F = G[-m:], F[-m:]
        gram = np.array([[np.vdot(a, b) for b in F] for a in F])
        y = np.linalg.solve(gram + 1e-12 * np.trace(gram) / len(F) * np.eye(len(F)), np.ones(len(F)))
        a = y / y.sum()
        x = sum(ai * gi for ai, gi in zip(a, G))
        p.phi[inner] = x
    return sweeps, residual(p)[0]


# --------------------------------------------------------------------------
# Single-scatter source (Sec. 3 after Eq. 6; Sec. 6.2)
# --------------------------------------------------------------------------

def bake_directional(sigma_t: np.ndarray, albedo: np.ndarray, h: float, direction=(0.0, 0.0, -1.0),
                     radiance: float = 1.0, step: float | None = None, nthreads: int | None = None):
    """q_ri = L sigma_s T for a directional light travelling along `direction`."""
    lib = _load()
    sigma_t = np.ascontiguousarray(sigma_t, dtype=np.float32)
    albedo = np.ascontiguousarray(albedo, dtype=np.float32)
    nz, ny, nx = sigma_t.shape
    q = np.empty(sigma_t.shape, dtype=np.float64)
    d = np.asarray(direction, dtype=np.float64)
    lib.fldo_bake_directional(nx, ny, nz, float(h), _f(sigma_t), _f(albedo), _d(d), float(radiance),
                              float(0.5 * h if step is None else step), int(nthreads or default_threads()),
                              _d(q))
    return q


def bake_point(sigma_t: np.ndarray, albedo: np.ndarray, h: float, pos, power: float = 1.0,
               step: float | None = None, nthreads: int | None = None):
    """q_ri = P sigma_s T / (4 pi max(r, h/2)^2) for a point light at `pos`."""
    lib = _load()
    sigma_t = np.ascontiguousarray(sigma_t, dtype=np.float32)
    albedo = np.ascontiguousarray(albedo, dtype=np.float32)
    nz, ny, nx = sigma_t.shape
    q = np.empty(sigma_t.shape, dtype=np.float64)
    pp = np.asarray(pos, dtype=np.float64)
    lib.fldo_bake_point(nx, ny, nz, float(h), _f(sigma_t), _f(albedo), _d(pp), float(power),
                        float(0.5 * h if step is None else step), int(nthreads or default_threads()), _d(q))
    return q


def flux_magnitude(p: Problem, phi: np.ndarray | None = None) -> np.ndarray:
    """|E_p| = D_p |grad phi_p| with D_p recomputed from phi (Eq. 15, 33-35),
    for the flux-limiting constraint |E| <= phi (Eq. 14)."""
    lib = _load()
    c = p.cfg()
    ph = p.phi if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
    E = np.empty((p.nz, p.ny, p.nx), dtype=np.float64)
    lib.fldo_flux(ctypes.byref(c), _d(p.sp), _d(ph), _d(E))
    return E


# --------------------------------------------------------------------------
# Picard iteration with an aggregation-multigrid linear solver: a reference
# solver for the nonlinear-multigrid direction (not in the paper; the paper
# names multigrid only as future work).  Test infrastructure like the rest.
# --------------------------------------------------------------------------

def fresh_D_field(p: Problem, phi: np.ndarray) -> np.ndarray:
    """D = F(R(phi))/sigma' at every unknown from phi (Eq. 33-35), ghost D as
    in p.D: the D^k of one Jacobi iteration (`fldo_jacobi_iteration`), taken
    on a copy of the state."""
    q = dataclasses.replace(p, phi=np.array(phi, dtype=np.float64), D=p.D.copy(), omega=1.0)
    jacobi_iteration(q, 1)
    return q.D


def lagged_system(p: Problem, D: np.ndarray):
    """Eq. 31 with D frozen: A phi = b over the unknowns (x fastest), with
    D_ps = (D_p + D_s)/2, A_pp = sigma_a' h^2 + sum_s D_ps, A_ps = -D_ps for
    unknown neighbours, and the Dirichlet ghosts' D_ps phi_s moved into b = j h^2 + ...
    Returns (A as scipy CSR, b)."""
    import scipy.sparse as sps
    nz, ny, nx = p.nz, p.ny, p.nx
    h2 = p.h * p.h
    n = nx * ny * nz
    idx = np.arange(n).reshape(nz, ny, nx)
    Dp = D[1:-1, 1:-1, 1:-1]
    diag = (p.sa * h2).ravel().copy()
    b = (p.j * h2).ravel().copy()
    rows, cols, vals = [idx.ravel()], [idx.ravel()], []
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    off = []
    for dz, dy, dx in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
        Dn = D[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        Dps = 0.5 * (Dp + Dn)
        diag += Dps.ravel()
        kk, jj, ii = k + dz, j + dy, i + dx
        inside = (kk >= 0) & (kk < nz) & (jj >= 0) & (jj < ny) & (ii >= 0) & (ii < nx)
        rows.append(idx[inside])
        cols.append((kk[inside] * ny + jj[inside]) * nx + ii[inside])
        off.append(-Dps[inside])
        ghost_phi = p.phi[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]
        np.add.at(b, idx[~inside], (Dps * ghost_phi)[~inside])
    vals = [diag] + off
    A = sps.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))
    return A, b


class AggregationMG:
    """V-cycle over Galerkin coarse operators P^T A P of 2x2x2 aggregates
    (P piecewise constant, or with `smooth` one damped-Jacobi step applied
    to it -- smoothed aggregation; either way the coarse operators follow the
    fine coefficients across their jumps), damped-Jacobi smoothing (2 + 2
    sweeps, weight 2/3) and a direct solve on the coarsest level; symmetric,
    so it preconditions CG."""

    def __init__(self, A, shape, coarsest: int = 2000, smooth: bool = False):
        import scipy.sparse as sps
        import scipy.sparse.linalg as spla
        self.A, self.P = [A.tocsr()], []
        while self.A[-1].shape[0] > coarsest and min(shape) > 1:
            nz, ny, nx = shape
            cz, cy, cx = (nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2
            k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
            agg = (((k // 2) * cy + j // 2) * cx + i // 2).ravel()
            P = sps.csr_matrix((np.ones(agg.size), (np.arange(agg.size), agg)), shape=(agg.size, cz * cy * cx))
            if smooth:
                # smoothed aggregation: P = (I - w D^-1 A) P_tent, w = 4 / (3 rho(D^-1 A)),
                # rho bounded by the largest absolute row sum of D^-1 A
                Af = self.A[-1]
                dinv = 1.0 / Af.diagonal()
                DA = sps.diags(dinv) @ Af
                rho = float(np.abs(DA).sum(axis=1).max())
                P = (P - (4.0 / (3.0 * rho)) * (DA @ P)).tocsr()
            self.P.append(P)
            self.A.append((P.T @ self.A[-1] @ P).tocsr())
            shape = (cz, cy, cx)
        self.dinv = [1.0 / M.diagonal() for M in self.A]
        self.lu = spla.splu(self.A[-1].tocsc())

    def vcycle(self, b, level: int = 0):
        if level == len(self.A) - 1:
            return self.lu.solve(b)
        A, dinv = self.A[level], self.dinv[level]
        x = np.zeros_like(b)
        for _ in range(2):
            x = x + (2.0 / 3.0) * dinv * (b - A @ x)
        x = x + self.P[level] @ self.vcycle(self.P[level].T @ (b - A @ x), level + 1)
        for _ in range(2):
            x = x + (2.0 / 3.0) * dinv * (b - A @ x)
        return x


def solve_picard_mg(p: Problem, tol: float, m: int = 5, inner_tol: float = 1e-4, max_steps: int = 400,
                    smooth: bool = True):
    """The fixed point of Eq. 31 by Picard steps -- D from the current phi,
    then the linear system with that D (`lagged_system`) solved by CG
    preconditioned with one `AggregationMG` V-cycle to `inner_tol` relative
    -- with Anderson mixing of the last m steps.  Stops when the fresh-D
    residual of Eq. 37 is <= tol (the definition `solve` uses).  Returns
    (picard_steps, cg_iterations, rel)."""
    import scipy.sparse.linalg as spla
    inner = (slice(1, -1),) * 3
    shape = (p.nz, p.ny, p.nx)
    x = p.phi[inner].copy()
    G, F = [], []
    cg_its = 0
    for step in range(1, max_steps + 1):
        A, b = lagged_system(p, fresh_D_field(p, p.phi))
        mg = AggregationMG(A, shape, smooth=smooth)
        count = [0]
        M = spla.LinearOperator(A.shape, matvec=mg.vcycle)
        r0 = float(np.linalg.norm(b - A @ x.ravel()))
        g, _ = spla.cg(A, b, x0=x.ravel(), rtol=0.0, atol=inner_tol * r0, maxiter=500, M=M,
                       callback=lambda _xk: count.__setitem__(0, count[0] + 1))
        cg_its += count[0]
        g = g.reshape(shape)
        G.append(g)
        F.append(g - x)
        G, F = G[-m:], F[-m:]
        gram = np.array([[np.vdot(a, c) for c in F] for a in F])
        if np.trace(gram) > 0.0:
            y = np.linalg.solve(gram + 1e-12 * np.trace(gram) / len(F) * np.eye(len(F)), np.ones(len(F)))
            a = y / y.sum()
            x = sum(ai * gi for ai, gi in zip(a, G))
        else:
            x = g
        p.phi[inner] = x
        rel = residual(p)[0]
        if rel <= tol:
            return step, cg_its, rel
    return max_steps, cg_its, residual(p)[0]


def solve_newton_mg(p: Problem, tol: float, start_tol: float = 1e-2, max_newton: int = 30, smooth: bool = True):
    """Newton's method on the residual of Eq. 37 (with D recomputed from phi),
    started from `solve_picard_mg` to `start_tol`: each step solves J d = -R
    by GMRES with Jacobian-vector products by forward differences of the
    residual field (`residual`) and one `AggregationMG` V-cycle of the lagged
    operator (J ~ -A / h^2) as preconditioner, then backtracks on |R|.
    Stops when the relative residual is <= tol.  Returns
    (picard_steps, newton_steps, v_cycles, residual_evaluations, rel_history)."""
    import scipy.sparse.linalg as spla
    inner = (slice(1, -1),) * 3
    shape = (p.nz, p.ny, p.nx)
    pic, cg_its, rel = solve_picard_mg(p, start_tol, smooth=smooth)
    counts = {"v": cg_its, "f": 0}
    history = [rel]

    def field(x):
        ph = p.phi.copy()
        ph[inner] = x.reshape(shape)
        counts["f"] += 1
        return residual(p, ph, field=True)[3].ravel()

    x = p.phi[inner].ravel().copy()
    for step in range(1, max_newton + 1):
        if rel <= tol:
            return pic, step - 1, counts["v"], counts["f"], history
        R = field(x)
        A, _ = lagged_system(p, fresh_D_field(p, p.phi))
        mg = AggregationMG(A, shape, smooth=smooth)
        scale = np.linalg.norm(x)

        def jv(v):
            nv = np.linalg.norm(v)
            if nv == 0.0:
                return np.zeros_like(v)
            e = 1e-7 * (1.0 + scale) / nv
            return (field(x + e * v) - R) / e

        def pre(r):
            counts["v"] += 1
            return -p.h * p.h * mg.vcycle(r)

        n = x.size
        d, _ = spla.gmres(spla.LinearOperator((n, n), matvec=jv), -R, rtol=1e-2, restart=30, maxiter=3,
                          M=spla.LinearOperator((n, n), matvec=pre))
        r0, lam = np.linalg.norm(R), 1.0
        while True:
            xn = x + lam * d
            if np.linalg.norm(field(xn)) < r0 or lam < 1e-3:
                break
            lam *= 0.5
        x = xn
        p.phi[inner] = x.reshape(shape)
        rel = residual(p)[0]
        history.append(rel)
    return pic, max_newton, counts["v"], counts["f"], history
