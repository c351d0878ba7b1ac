"""Anderson mixing of blocks of sweeps (fld_solve_params.anderson): the mix
changes the iteration path only, so every accelerated solve must land on the
oracle's fixed point like a plain one -- and do so in fewer sweeps."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

INNER = (slice(1, -1),) * 3


def cloud(shape, seed=5, albedo=0.95):
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=seed, albedo=albedo, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    q = oracle.bake_directional(sig, alb, h, (0, 0, -1), 1.0).astype(np.float32)
    return sig, alb, q, h


_FIXED_POINTS = {}


def oracle_fixed_point(sig, alb, q, h):
    key = (sig.shape, float(sig.sum()), float(q.sum()))
    if key not in _FIXED_POINTS:
        ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, omega=1.6, local_iters=2)
        oracle.init_state(ref)
        it, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
        assert rel <= 1e-11
        _FIXED_POINTS[key] = ref.phi
    return _FIXED_POINTS[key]


def rel_l2(a, b):
    return np.linalg.norm(a[INNER] - b[INNER]) / np.linalg.norm(b[INNER])


@pytest.mark.parametrize("shape", [(24, 24, 24), (29, 17, 23)])
@pytest.mark.parametrize("precision,tol,bound", [("mixed", 1e-6, 1e-5), ("fp64", 1e-10, 1e-8)])
@pytest.mark.parametrize("m", [3, 8])
def test_anderson_solve_reaches_the_oracle_fixed_point(shape, precision, tol, bound, m):
    sig, alb, q, h = cloud(shape)
    ref = oracle_fixed_point(sig, alb, q, h)
    nz, ny, nx = shape
    with fld.Grid(nx, ny, nz, h) as g:
        g.set_medium(sig, alb)
        g.set_source(q)
        r = g.solve(fld.params(precision=precision, tol=tol, check_every=16, max_iters=400000, anderson=m))
        assert r.status == fld.FLD_OK, r.as_dict()
        assert r.anderson_steps > 0
        phi, D = g.get_state()
    assert rel_l2(phi, ref) <= bound
    assert np.all(phi[INNER] > 0)


def test_anderson_cuts_the_sweeps_of_a_cloud_solve():
    sig, alb, q, h = cloud((32, 32, 32), seed=0)
    iters = {}
    phis = {}
    for m in (0, 8):
        with fld.Grid(32, 32, 32, h) as g:
            g.set_medium(sig, alb)
            g.set_source(q)
            r = g.solve(fld.params(tol=1e-6, check_every=32, max_iters=400000, anderson=m))
            assert r.status == fld.FLD_OK, r.as_dict()
            iters[m] = r.iterations
            phis[m] = g.get_state()[0]
    assert iters[8] * 2 < iters[0], iters
    # both stop at rel. residual 1e-6 of the same discrete equation
    assert rel_l2(phis[8], phis[0]) <= 2e-5


def test_anderson_with_a_nested_start():
    sig, alb, q, h = cloud((20, 20, 20), seed=3)
    ref = oracle_fixed_point(sig, alb, q, h)
    with fld.Grid(20, 20, 20, h) as g:
        g.set_medium(sig, alb)
        g.set_source(q)
        r = g.solve(fld.params(tol=1e-6, check_every=16, max_iters=400000, anderson=6, nested=1))
        assert r.status == fld.FLD_OK, r.as_dict()
        assert r.iterations_coarse > 0
        phi, _ = g.get_state()
    assert rel_l2(phi, ref) <= 1e-5


def test_anderson_argument_checks():
    sig, alb, q, h = cloud((8, 8, 8))
    with fld.Grid(8, 8, 8, h) as g:
        g.set_medium(sig, alb)
        g.set_source(q)
        for bad in (dict(anderson=17), dict(anderson=-1), dict(anderson=4, scheme="jacobi", precision="fp64")):
            with pytest.raises(fld.FldError) as e:
                g.solve(fld.params(**bad))
            assert e.value.status == fld.FLD_ERR_INVALID_ARG, bad
        with pytest.raises(fld.FldError) as e:
            fld.fld_solve_batch([g], fld.params(anderson=17))
        assert e.value.status == fld.FLD_ERR_INVALID_ARG
    with pytest.raises(fld.FldError) as e:
        fld.fld_server_create(fld.params(anderson=-1))
    assert e.value.status == fld.FLD_ERR_INVALID_ARG


def test_anderson_batch_and_server_equal_solo_solves():
    # the mix runs per grid in the batched and served paths too, with the same
    # kernels at the same points of each grid's solve: every result equals its
    # solo solve bit for bit, and the oracle's fixed point
    p = fld.params(precision="mixed", tol=1e-6, check_every=16, max_iters=400000, anderson=6)
    shapes = [(16, 16, 16), (12, 20, 18), (21, 13, 9)]
    cases = [cloud(s) for s in shapes]

    def grid(sig, alb, q, h):
        nz, ny, nx = sig.shape
        g = fld.Grid(nx, ny, nz, h)
        g.set_medium(sig, alb)
        g.set_source(q)
        return g

    solo = []
    for c in cases:
        with grid(*c) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK and r.anderson_steps > 0, r.as_dict()
            solo.append((r.iterations, r.anderson_steps, g.get_state()[0]))
    grids = [grid(*c) for c in cases]
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for a, g in enumerate(grids):
            assert (rs[a].iterations, rs[a].anderson_steps) == solo[a][:2]
            assert np.array_equal(g.get_state()[0], solo[a][2]), a
    finally:
        for g in grids:
            g.close()
    grids = [grid(*c) for c in cases]
    try:
        done = {}
        with fld.Server(p) as srv:
            srv.add(grids[0], 0)
            steps = 0
            while srv.active > 0 or len(done) < len(grids):
                if steps in (2, 5):
                    srv.add(grids[1 if steps == 2 else 2], 1 if steps == 2 else 2)
                for tag, r in srv.step():
                    done[tag] = r
                steps += 1
                assert steps < 100000
        for a, g in enumerate(grids):
            assert done[a].iterations == solo[a][0]
            assert np.array_equal(g.get_state()[0], solo[a][2]), a
    finally:
        for g in grids:
            g.close()
