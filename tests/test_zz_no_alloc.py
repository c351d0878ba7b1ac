"""The allocation-free residual entry point, called through the C ABI.

fld_residual_noalloc serves callers that may not allocate device memory when
they evaluate the residual (a renderer's frame loop where cudaMalloc is
banned after start-up, a host application that lends the library buffers from
its own pool).  It must give the same relative residual as fld_residual in
FP64 on the same state, on two calls in a row (its fixed scratch array is
shared by every call and keeps the previous call's contents).

This file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1403_8105_gb300 as fld  # noqa: E402


def _state(shape, seed):
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    sig = rng.uniform(0.5, 30.0, shape).astype(np.float32)
    sig[rng.uniform(size=shape) < 0.2] = 0.0
    alb = rng.uniform(0.3, 0.99, shape).astype(np.float32)
    j = rng.uniform(0.0, 4.0, shape).astype(np.float32)
    phi = rng.uniform(0.1, 2.0, (nz + 2, ny + 2, nx + 2))
    phi[0, :, :] = phi[-1, :, :] = 0.05            # ghost values
    D = np.full(phi.shape, 0.02)
    D[1:-1, 1:-1, 1:-1] = rng.uniform(0.001, 0.3, shape)
    return sig, alb, j, phi, D, 1.0 / max(shape)


@pytest.mark.parametrize("shape,margin,limiter", [((20, 17, 33), 0, "lp"), ((9, 40, 12), 2, "kershaw")])
def test_noalloc_residual_matches_fld_residual_twice(shape, margin, limiter):
    sig, alb, j, phi, D, h = _state(shape, 3)
    nz, ny, nx = shape
    p = fld.params(precision="fp64", limiter=limiter, residual_margin=margin)
    with fld.Grid(nx, ny, nz, h) as g:
        g.set_medium(sig, alb)
        g.set_source(j)
        g.set_state(phi, D)
        want = g.residual(p)

    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(a).to(dev) for a in (sig, alb, j, phi, D)]
    torch.cuda.synchronize()
    lib = fld.load()                      # the C ABI, called directly through ctypes
    fn = lib.fld_residual_noalloc
    got = []
    for _ in range(2):
        rel = ctypes.c_double(-1.0)
        st = fn(nx, ny, nz, h, ctypes.byref(p), *[ctypes.c_void_p(b.data_ptr()) for b in bufs],
                ctypes.byref(rel), None)
        assert st == fld.FLD_OK, fld.fld_last_error()
        got.append(rel.value)
    for v in got:
        assert abs(v - want) <= 1e-12 * want, (v, want)
    assert got[0] == got[1]


def test_noalloc_rejects_grids_beyond_its_scratch():
    p = fld.params(precision="fp64")
    dev = torch.device("cuda", 0)
    one = torch.zeros(1, device=dev)
    rel = ctypes.c_double(0.0)
    # ceil(512/32) * ceil(512/8) * 512 blocks > 65536 partial-sum slots
    st = fld.load().fld_residual_noalloc(512, 512, 512, 1.0 / 512, ctypes.byref(p),
                                         *[ctypes.c_void_p(one.data_ptr())] * 5, ctypes.byref(rel), None)
    assert st == fld.FLD_ERR_INVALID_ARG
    assert "FLD_NOALLOC_MAX_BLOCKS" in fld.fld_last_error()


def test_noalloc_allocates_nothing_and_runs_on_a_given_stream():
    # the entry point's claim itself: after a first call, further calls leave
    # the device's free memory unchanged (no cudaMalloc, no pool growth), and
    # the call is ordered on the stream it is given
    shape = (18, 21, 25)
    sig, alb, j, phi, D, h = _state(shape, 5)
    nz, ny, nx = shape
    p = fld.params(precision="fp64")
    dev = torch.device("cuda", 0)
    bufs = [torch.from_numpy(a).to(dev) for a in (sig, alb, j, phi, D)]
    torch.cuda.synchronize()
    fn = fld.load().fld_residual_noalloc
    args = [ctypes.c_void_p(b.data_ptr()) for b in bufs]
    rel = ctypes.c_double(-1.0)
    assert fn(nx, ny, nz, h, ctypes.byref(p), *args, ctypes.byref(rel), None) == fld.FLD_OK
    first = rel.value
    # the test's own stream is made (and used once) before the measurement:
    # torch's first stream request sets up its stream pool, which takes
    # device memory of its own
    side = torch.cuda.Stream(device=dev)
    assert fn(nx, ny, nz, h, ctypes.byref(p), *args, ctypes.byref(rel), ctypes.c_void_p(side.cuda_stream)) == fld.FLD_OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(dev)
    for k in range(6):
        rel = ctypes.c_double(-1.0)
        stream = ctypes.c_void_p(side.cuda_stream) if k % 2 else None
        assert fn(nx, ny, nz, h, ctypes.byref(p), *args, ctypes.byref(rel), stream) == fld.FLD_OK
        assert rel.value == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(dev)
    assert free1 == free0, (free0, free1)
