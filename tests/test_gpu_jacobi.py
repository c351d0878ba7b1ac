"""GPU parity of the Jacobi scheme (scheme = "jacobi"): D^k from phi^k at
every unknown, then phi^{k+1} from phi^k and D^k into a second buffer,
against the oracle's Jacobi iteration; its fixed point against the oracle's
red-black phi*."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_parity import INNER, gpu_grid, random_case, rel_el  # noqa: E402


@pytest.mark.parametrize("limiter", ["lp", "kershaw", "larsen", "sum", "max", "cda"])
@pytest.mark.parametrize("omega", [1.0, 0.7])
@pytest.mark.parametrize("iters", [1, 5])
def test_jacobi_fp64_matches_oracle(limiter, omega, iters):
    sig, alb, j, h = random_case((9, 11, 13), 3)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, limiter=limiter, omega=omega, nthreads=1)
    oracle.init_state(ref)
    oracle.jacobi_iteration(ref, 4)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    oracle.jacobi_iteration(ref, iters)
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(phi0, D0)
        g.iterate(fld.params(limiter=limiter, precision="fp64", scheme="jacobi", omega=omega, warm_start=1), iters)
        phi, D = g.get_state()
    e_phi, e_D = rel_el(phi, ref.phi, also=phi0), rel_el(D, ref.D, also=D0)
    print(f"jacobi fp64 {limiter} omega={omega} x{iters}: per-element phi {e_phi:.2e} D {e_D:.2e}")
    assert e_phi <= 1e-12
    assert e_D <= 1e-12


@pytest.mark.parametrize("limiter", ["lp", "kershaw"])
def test_jacobi_fp32_matches_oracle(limiter):
    sig, alb, j, h = random_case((16, 12, 20), 5)
    ref = oracle.make_problem(sig, alb, j.astype(np.float64), h, limiter=limiter, omega=0.9, nthreads=1)
    oracle.init_state(ref)
    oracle.jacobi_iteration(ref, 6)
    ref.phi[...] = ref.phi.astype(np.float32)
    ref.D[...] = ref.D.astype(np.float32)
    phi0, D0 = ref.phi.copy(), ref.D.copy()
    oracle.jacobi_iteration(ref, 3)
    with gpu_grid(sig, alb, j, h) as g:
        g.set_state(phi0, D0)
        g.iterate(fld.params(limiter=limiter, precision="fp32", scheme="jacobi", omega=0.9, warm_start=1), 3)
        phi, D = g.get_state()
    e_phi, e_D = rel_el(phi, ref.phi, also=phi0), rel_el(D, ref.D, also=D0)
    print(f"jacobi fp32 {limiter}: per-element phi {e_phi:.2e} D {e_D:.2e}")
    assert e_phi <= 3e-6
    assert e_D <= 3e-5


def test_jacobi_fixed_point_is_the_red_black_one():
    n = 12
    sig, alb = fld_inputs.cloud_medium(n, seed=4, albedo=0.9)
    h = 1.0 / n
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0).astype(np.float32)
    ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, omega=1.5, local_iters=2)
    oracle.init_state(ref)
    it, rel, _ = oracle.solve(ref, tol=1e-12, max_iters=200000, check_every=20)
    assert rel <= 1e-12
    with gpu_grid(sig, alb, q, h) as g:
        r = g.solve(fld.params(precision="fp64", scheme="jacobi", tol=1e-10, check_every=500, max_iters=2000000))
        assert r.status == fld.FLD_OK, r.as_dict()
        phi, _ = g.get_state()
        r32 = g.solve(fld.params(precision="fp32", scheme="jacobi", tol=1e-4, check_every=500, max_iters=2000000))
        assert r32.status == fld.FLD_OK, r32.as_dict()
        phi32, _ = g.get_state()
    err = np.linalg.norm(phi[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
    assert err <= 1e-8
    err32 = np.linalg.norm(phi32[INNER] - ref.phi[INNER]) / np.linalg.norm(ref.phi[INNER])
    assert err32 <= 1e-3


def test_jacobi_batch_equals_solo_and_invalid_combinations():
    # batched solves run the single-precision families: Jacobi in FP32
    p = fld.params(precision="fp32", scheme="jacobi", tol=1e-4, check_every=200, max_iters=400000)
    shapes = [(8, 8, 8), (7, 9, 5)]
    ins = []
    for s, (nz, ny, nx) in enumerate(shapes):
        sig, alb = fld_inputs.cloud_medium(nx, seed=30 + s, albedo=0.9, ny=ny, nz=nz)
        ins.append((sig, alb, 1.0 / max(nx, ny, nz)))

    def grid(sig, alb, h):
        nz, ny, nx = sig.shape
        g = fld.Grid(nx, ny, nz, h)
        g.set_medium(sig, alb)
        g.bake_directional((0.0, 0.0, -1.0), 1.0)
        return g

    solo = []
    for sig, alb, h in ins:
        with grid(sig, alb, h) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK, r.as_dict()
            solo.append((r.iterations, g.get_state()[0]))
    grids = [grid(*x) for x in ins]
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for a, g in enumerate(grids):
            assert rs[a].status == fld.FLD_OK and rs[a].iterations == solo[a][0]
            assert np.array_equal(g.get_state()[0], solo[a][1]), a
        for bad in (dict(precision="mixed"), dict(precision="pair"), dict(omega=1.5), dict(scheme=7)):
            kw = dict(precision="fp64", scheme="jacobi")
            kw.update(bad)
            with pytest.raises(fld.FldError) as e:
                grids[0].solve(fld.params(**kw))
            assert e.value.status == fld.FLD_ERR_INVALID_ARG
    finally:
        for g in grids:
            g.close()
