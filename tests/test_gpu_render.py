"""GPU parity of the primary ray march (fld_render, Sec. 3) against the
oracle's renderer on the same fields: the medium, the oracle's baked source
and the oracle's solved phi, given to the GPU grid (set_source / set_state),
so nothing the oracle reads comes from the GPU."""
import math

import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)


def solved_cloud(n, seed, shape=None):
    """A GPU grid holding the oracle's source and the oracle's fixed point."""
    nz, ny, nx = shape or (n, n, n)
    sig, alb = fld_inputs.cloud_medium(nx, seed=seed, albedo=0.9, ny=ny, nz=nz)
    h = 1.0 / max(nx, ny, nz)
    q = oracle.bake_directional(sig, alb, h, (0.3, -0.2, -1.0), 1.0)
    ref = oracle.make_problem(sig, alb, q, h, omega=1.6, local_iters=2)
    oracle.init_state(ref)
    _, rel, _ = oracle.solve(ref, tol=1e-9, max_iters=200000, check_every=20)
    assert rel <= 1e-9
    g = fld.Grid(nx, ny, nz, h)
    g.set_medium(sig, alb)
    g.set_source(q.astype(np.float32))
    g.set_state(ref.phi, ref.D)
    return g, sig, alb, h, q.astype(np.float32).astype(np.float64), ref.phi


@pytest.mark.parametrize("shape", [(24, 24, 24), (17, 23, 29)])
@pytest.mark.parametrize("step_frac,t_min", [(0.5, 1e-6), (0.37, 0.0), (1.3, 1e-3)])
def test_render_matches_oracle(shape, step_frac, t_min):
    g, sig, alb, h, q, phi = solved_cloud(0, 8, shape)
    try:
        cam = dict(eye=(0.35, 1.2, -1.1), target=(0.5, 0.4, 0.55), up=(0.1, 1.0, 0.0), fov_deg=45.0, width=48,
                   height=40, step=step_frac * h, background=0.3, t_min=t_min)
        rad, _ = g.render(fld.camera(**cam))
    finally:
        g.close()
    want = oracle.render(sig, alb, q, phi, h, **cam)
    assert np.abs(rad - want).max() <= 2e-5 * np.abs(want).max()
    assert rad.std() > 0.01 * rad.mean()


def test_homogeneous_axis_ray_closed_form():
    n, h = 10, 0.1
    shape = (n, n, n)
    with fld.Grid(n, n, n, h) as g:
        g.set_medium(np.full(shape, 3.0, np.float32), np.full(shape, 0.25, np.float32))
        g.set_source(np.full(shape, 2.0, np.float32))
        g.set_state(np.zeros((n + 2,) * 3), np.full((n + 2,) * 3, 0.1))
        rad, _ = g.render(fld.camera(eye=(0.5, 0.5, -2.0), target=(0.5, 0.5, 0.5), width=1, height=1,
                                     step=0.3 * h, background=0.7, t_min=0.0))
    L, T, length = 0.0, 1.0, 1.0
    for m in range(math.ceil(length / (0.3 * h) - 1e-9)):
        seg = min(0.3 * h, length - m * 0.3 * h)
        L += T * 2.0 / (4 * math.pi) * seg
        T *= math.exp(-3.0 * seg)
    assert rad[0, 0] == pytest.approx(L + 0.7 * T, rel=2e-6)


def test_device_outputs_codes_and_errors():
    g, sig, alb, h, q, phi = solved_cloud(16, 2)
    try:
        cam = fld.camera(eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), width=33, height=17, background=0.1)
        rad, codes = g.render(cam, exposure=3.0, gamma=2.2, codes=True)
        drad = torch.empty((17, 33), dtype=torch.float32, device="cuda")
        dcod = torch.empty((17, 33), dtype=torch.uint8, device="cuda")
        fld.fld_render(g.handle, None, cam, drad, dcod, 3.0, 2.2)
        torch.cuda.synchronize()
        assert np.array_equal(drad.cpu().numpy(), rad)
        assert np.array_equal(dcod.cpu().numpy(), codes)
        # the codes against the oracle's tone map of its own radiance: +-1 where
        # the two radiances straddle a half-integer code boundary
        want = oracle.render(sig, alb, q, phi, h, eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), width=33,
                             height=17, background=0.1)
        mine = oracle.tonemap(want, exposure=3.0, gamma=2.2, dtype=np.float32)
        assert np.abs(mine.astype(int) - codes.astype(int)).max() <= 1
        for bad in (dict(width=0), dict(fov_deg=180.0), dict(eye=(0.5, 0.5, 0.5)), dict(up=(0.0, 0.0, 1.0))):
            kw = dict(eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), width=8, height=8)
            kw.update(bad)
            with pytest.raises(fld.FldError) as e:
                g.render(fld.camera(**kw))
            assert e.value.status == fld.FLD_ERR_INVALID_ARG
        with pytest.raises(fld.FldError) as e:
            g.render(cam, exposure=0.0)
        assert e.value.status == fld.FLD_ERR_INVALID_ARG
    finally:
        g.close()
    with fld.Grid(4, 4, 4, 0.25) as g2:
        with pytest.raises(fld.FldError) as e:
            g2.render(fld.camera(eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), width=4, height=4))
        assert e.value.status == fld.FLD_ERR_STATE


def test_quarter_resolution_pipeline_matches_oracle():
    # fine 40 x 36 x 30 (not divisible by 4: partial blocks), phi solved at
    # 10 x 9 x 8 with spacing 4h, rendered at full resolution
    nx, ny, nz, f = 40, 36, 30, 4
    sig, alb = fld_inputs.cloud_medium(nx, seed=12, albedo=0.9, ny=ny, nz=nz)
    h = 1.0 / max(nx, ny, nz)
    cx, cy, cz = (nx + f - 1) // f, (ny + f - 1) // f, (nz + f - 1) // f
    q = oracle.bake_directional(sig, alb, h, (0.2, -0.3, -1.0), 1.0).astype(np.float32).astype(np.float64)
    with fld.Grid(nx, ny, nz, h) as g, fld.Grid(cx, cy, cz, f * h) as c:
        g.set_medium(sig, alb)
        g.set_source(q.astype(np.float32))
        g.downsample_to(c, f)
        qc_gpu = c.get_source()
        r = c.solve(fld.params(tol=1e-7, check_every=32, max_iters=200000))
        assert r.status == fld.FLD_OK, r.as_dict()
        phic, _ = c.get_state()
        cam = dict(eye=(0.4, 1.1, -1.2), target=(0.5, 0.4, 0.4), fov_deg=45.0, width=40, height=32, background=0.2)
        rad, _ = g.render(fld.camera(**cam), phi_grid=c)
    # the oracle's own chain: downsample, coarse fixed point, upsample, render
    stc, alc, qc = oracle.downsample(sig, alb, q, f)
    assert np.abs(qc_gpu - qc).max() <= 1e-6 * np.abs(qc).max()
    ref = oracle.make_problem(stc.astype(np.float32), alc.astype(np.float32), qc.astype(np.float32).astype(np.float64),
                              f * h, omega=1.6, local_iters=2)
    oracle.init_state(ref)
    it, rel, _ = oracle.solve(ref, tol=1e-11, max_iters=400000, check_every=20)
    assert rel <= 1e-11
    inner = (slice(1, -1),) * 3
    err = np.linalg.norm(phic[inner] - ref.phi[inner]) / np.linalg.norm(ref.phi[inner])
    assert err <= 1e-5
    up = oracle.upsample(ref.phi, (nz, ny, nx), h, f)
    want = oracle.render(sig, alb, q, up, h, **cam)
    assert np.abs(rad - want).max() <= 2e-5 * np.abs(want).max()


def test_downsample_rejects_mismatched_grids():
    with fld.Grid(16, 16, 16, 1 / 16) as g, fld.Grid(5, 4, 4, 0.25) as bad, fld.Grid(4, 4, 4, 0.3) as bad_h:
        sig, alb = fld_inputs.cloud_medium(16, seed=1, albedo=0.9)
        g.set_medium(sig, alb)
        for other in (bad, bad_h):
            with pytest.raises(fld.FldError) as e:
                g.downsample_to(other, 4)
            assert e.value.status == fld.FLD_ERR_INVALID_ARG


def test_host_render_loop_allocates_nothing_after_the_first_frame():
    # host outputs go through the grid's own staging image, grown only for a
    # larger image: repeated frames give the same pixels and leave the free
    # device memory as it was after the first frame
    g, sig, alb, h, q, phi = solved_cloud(16, 3)
    kw = dict(eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), up=(0.0, 1.0, 0.0), fov_deg=40.0, width=48, height=40,
              step=0.5 * h, background=0.2, t_min=1e-6)
    try:
        cam = fld.camera(**kw)
        small = fld.camera(**{**kw, "width": 20, "height": 12})
        rad0, cod0 = g.render(cam, exposure=2.0, codes=True)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(4):
            rad, cod = g.render(cam, exposure=2.0, codes=True)
            assert np.array_equal(rad, rad0) and np.array_equal(cod, cod0)
            g.render(small, exposure=2.0)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        want = oracle.render(sig, alb, q, phi, h, **kw)
        assert np.abs(rad0 - want).max() <= 2e-5 * np.abs(want).max()
    finally:
        g.close()
