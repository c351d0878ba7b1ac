"""Per-channel (RGB) albedo (Sec. 6.2, the CT scene's colour transfer
function): the same extinction with one albedo per channel gives three
independent FLD problems (sigma_s = albedo_c sigma_t bakes a different source
and sigma_a' = (1 - albedo_c) sigma' a different absorption per channel).
They run as one batched solve; each channel must equal its solo solve bit for
bit and land on the oracle's fixed point of that channel."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

from test_gpu_parity import INNER, rel_el, rel_l2  # noqa: E402


def test_rgb_channels_batched_match_solo_and_oracle():
    shape = (18, 22, 20)
    nz, ny, nx = shape
    sig, _ = fld_inputs.cloud_medium(nx, seed=8, albedo=0.9, ny=ny, nz=nz)
    h = 1.0 / max(shape)
    # a colour transfer function: albedo varies with density differently per channel
    dens = sig / max(float(sig.max()), 1e-6)
    albs = [np.clip(a0 + a1 * dens, 0.0, 0.995).astype(np.float32)
            for a0, a1 in ((0.75, 0.2), (0.85, 0.1), (0.95, -0.1))]
    p = fld.params(limiter="lp", precision="mixed", tol=1e-6, omega=1.7, check_every=32, max_iters=400000)
    qs, refs = [], []
    for alb in albs:
        q = oracle.bake_directional(sig, alb, h, (0.2, -0.1, -1.0), 1.0).astype(np.float32)
        ref = oracle.make_problem(sig, alb, q.astype(np.float64), h, limiter="lp", omega=1.7, local_iters=2)
        oracle.init_state(ref)
        _, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
        assert rel <= 1e-11
        qs.append(q)
        refs.append(ref.phi[INNER].copy())
    # the channels really differ
    assert rel_l2(refs[0], refs[2]) > 1e-2

    def grid(alb, q):
        g = fld.Grid(nx, ny, nz, h)
        g.set_medium(sig, alb)
        g.set_source(q)
        return g

    solo = []
    for alb, q in zip(albs, qs):
        with grid(alb, q) as g:
            r = g.solve(p)
            assert r.status == fld.FLD_OK
            solo.append(g.get_state()[0])
    grids = [grid(a, q) for a, q in zip(albs, qs)]
    try:
        st, rs = fld.fld_solve_batch(grids, p)
        assert st == fld.FLD_OK
        for c, g in enumerate(grids):
            phi = g.get_state()[0]
            assert np.array_equal(phi, solo[c]), c
            l2, el = rel_l2(phi[INNER], refs[c]), rel_el(phi[INNER], refs[c], floor=1e-3)
            print(f"channel {c}: rel L2 {l2:.2e} per-element {el:.2e} residual {rs[c].rel_residual:.2e}")
            assert rs[c].rel_residual <= 1e-6
            assert l2 <= 1e-5 and el <= 1e-4
    finally:
        for g in grids:
            g.close()
