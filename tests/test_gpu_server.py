"""Continuous batching on the GPU: solves admitted to a running server at
different steps finish with exactly the result of their solo solve."""
import numpy as np
import pytest

import fld_inputs

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

SHAPES = [(16, 16, 16), (24, 20, 18), (12, 12, 12), (20, 20, 20), (10, 30, 14)]


def _grid(a, shape):
    nz, ny, nx = shape
    sig, alb = fld_inputs.cloud_medium(nx, seed=40 + a, albedo=0.85 + 0.03 * a, ny=ny, nz=nz)
    g = fld.Grid(nx, ny, nz, 1.0 / max(shape))
    g.set_medium(sig, alb)
    if a % 2:
        g.bake_point((0.2, 0.8, 1.4), 3.0)
    else:
        g.bake_directional((0.2, -0.1, -1.0), 1.0)
    return g


def test_server_admissions_mid_stream_equal_solo_solves():
    p = fld.params(limiter="lp", precision="mixed", tol=1e-7, check_every=32, max_iters=200000)
    solo = []
    for a, shape in enumerate(SHAPES):
        with _grid(a, shape) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK
            solo.append((r.iterations, g.get_state()[0]))
    grids = [_grid(a, shape) for a, shape in enumerate(SHAPES)]
    done = {}
    try:
        with fld.Server(p) as srv:
            srv.add(grids[0], 0)
            srv.add(grids[1], 1)
            steps = 0
            nxt = 2
            while srv.active > 0 or nxt < len(grids):
                if nxt < len(grids) and steps in (3, 7, 11):
                    srv.add(grids[nxt], nxt)          # joins the running set
                    nxt += 1
                for tag, r in srv.step():
                    done[tag] = r
                steps += 1
                assert steps < 100000
        assert sorted(done) == list(range(len(grids)))
        for a, g in enumerate(grids):
            assert done[a].status == fld.FLD_OK
            assert done[a].iterations == solo[a][0]
            assert np.array_equal(g.get_state()[0], solo[a][1]), a
    finally:
        for g in grids:
            g.close()


def test_serving_loop_runs_a_small_stream():
    from paper_1403_8105_gb300 import serve
    p = fld.params(limiter="lp", precision="mixed", tol=1e-6, check_every=64, max_iters=200000)
    arr = serve.poisson_arrivals(8, 40.0, 5)
    reqs = []
    for i in range(8):
        n = [12, 16, 20, 24][i % 4]
        sig, alb = fld_inputs.cloud_medium(n, seed=i, albedo=0.9)
        reqs.append(serve.Request(rid=i, arrival=float(arr[i]), n=n, medium=(sig, alb),
                                  light=fld_inputs.Light(kind="directional"), footprint=serve.footprint_bytes(n)))
    be = serve.GpuBackend(p)
    try:
        reqs, st = serve.serve(reqs, be, max_active=4)
    finally:
        be.close()
    assert st["requests"] == 8
    assert all(r.result.status == fld.FLD_OK for r in reqs)
    assert st["max_in_flight"] <= 4


def test_served_results_match_the_oracle_fixed_point():
    # each result of the continuous-batching server, not only its solo twin,
    # against the oracle's FP64 fixed point of the same inputs (the source is
    # the oracle's bake, rounded to float, given to both sides)
    import oracle
    from test_gpu_parity import rel_el, rel_l2
    p = fld.params(limiter="lp", precision="mixed", tol=1e-6, omega=1.7, check_every=32, max_iters=200000)
    shapes = [(16, 16, 16), (12, 20, 18), (10, 14, 12)]
    grids, refs = [], []
    try:
        for a, (nz, ny, nx) in enumerate(shapes):
            sig, alb = fld_inputs.cloud_medium(nx, seed=70 + a, albedo=0.9, ny=ny, nz=nz)
            h = 1.0 / max(nx, ny, nz)
            q = oracle.bake_directional(sig, alb, h, (0.1, 0.2, -1.0), 1.0).astype(np.float32)
            ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, limiter="lp", omega=1.7, local_iters=2)
            oracle.init_state(ref)
            _, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
            assert rel <= 1e-11
            refs.append(ref.phi[1:-1, 1:-1, 1:-1].copy())
            g = fld.Grid(nx, ny, nz, h)
            g.set_medium(sig, alb)
            g.set_source(q)
            grids.append(g)
        done = {}
        with fld.Server(p) as srv:
            srv.add(grids[0], 0)
            srv.add(grids[1], 1)
            steps = 0
            while srv.active > 0 or len(done) < len(grids):
                if steps == 2:
                    srv.add(grids[2], 2)
                for tag, r in srv.step():
                    done[tag] = r
                steps += 1
                assert steps < 100000
        for a, g in enumerate(grids):
            r = done[a]
            assert r.status == fld.FLD_OK and r.rel_residual <= 1e-6, r.as_dict()
            phi = g.get_state()[0][1:-1, 1:-1, 1:-1]
            l2, el = rel_l2(phi, refs[a]), rel_el(phi, refs[a], floor=1e-3)
            print(f"served {shapes[a]}: rel L2 {l2:.2e} per-element {el:.2e} fp64 sweeps {r.iterations_fp64}")
            assert l2 <= 1e-5 and el <= 1e-4
    finally:
        for g in grids:
            g.close()
