"""Full-size checks on the 128^3 cloud (the benchmark workload), in the
benchmark's launch configuration: properties the oracle can check at any size
(its FP64 residual of the GPU solution, |E| <= phi, positivity, per-voxel
residuals computed one by one), one-iteration parity from a shared seeded
state, and sampled pixels of the full-size render.  The source is the oracle's
bake, given to the GPU grid; no oracle input comes from the GPU."""
import numpy as np
import pytest

import fld_inputs
import oracle

pytestmark = pytest.mark.gpu

fld = pytest.importorskip("paper_1403_8105_gb300")
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

N = 128
INNER = (slice(1, -1),) * 3


@pytest.fixture(scope="module")
def c2():
    case = fld_inputs.cloud_case(N, seed=0, albedo=0.95)
    j = oracle.bake_directional(case.sigma_t, case.alb, case.h, (0.0, 0.0, -1.0), 1.0).astype(np.float32)
    g = fld.Grid(N, N, N, case.h)
    g.set_medium(case.sigma_t, case.alb)
    g.set_source(j)
    yield case, g, j
    g.close()


def _seeded_state(seed):
    """A smooth positive phi (a product of cosines over the padded grid) and a
    positive D, both seeded: a state for one-iteration parity and the render."""
    rng = np.random.default_rng(seed)
    ax = [np.linspace(0.0, 1.0, N + 2)] * 3
    kz, ky, kx = rng.uniform(1.0, 3.0, 3)
    z, y, x = np.meshgrid(*ax, indexing="ij")
    phi = 0.05 + np.cos(kx * x) ** 2 * np.cos(ky * y) ** 2 * np.cos(kz * z) ** 2
    phi *= 1.0 + 0.05 * rng.standard_normal(phi.shape)
    D = rng.uniform(0.002, 0.3, phi.shape)
    return np.abs(phi), D


def test_converged_solution_satisfies_the_fp64_discrete_equation(c2):
    case, g, j = c2
    p = fld.params(limiter="lp", precision="mixed", tol=1e-6, check_every=256, max_iters=600000)
    r = g.solve(p)
    assert r.status == fld.FLD_OK, r.as_dict()
    phi, D = g.get_state()
    ref = oracle.make_problem(case.sigma_t, case.alb, j.astype(np.float64), case.h, limiter="lp")
    ref.phi, ref.D = phi, D
    rel64, _, _ = oracle.residual(ref)
    print(f"GPU rel residual {r.rel_residual:.3e} (single-precision D {r.rel_residual_single:.3e}, "
          f"FP64 sweeps {r.iterations_fp64}), FP64 oracle residual of the GPU phi {rel64:.3e}")
    # the stop test is taken in FP64 (fp64_verify): the returned phi satisfies
    # the FP64 discrete equation to the tolerance, as the oracle evaluates it
    assert r.rel_residual <= 1e-6
    assert rel64 <= 1e-6 * (1 + 1e-9)
    inner = phi[INNER]
    assert np.all(inner > 0)
    E = oracle.flux_magnitude(ref)
    assert np.all(E <= inner * (1 + 1e-6))                    # Eq. 14
    # per-voxel residuals computed one by one agree with the field reduction
    rng = np.random.default_rng(0)
    idx = rng.integers(0, N, size=(400, 3))
    _, _, _, R = oracle.residual(ref, field=True)
    for i, jj, k in idx:
        at = oracle.residual_at(ref, phi, int(i), int(jj), int(k))
        assert abs(at - R[k, jj, i]) <= 1e-9 * (abs(R[k, jj, i]) + ref.jbar)


def test_one_iteration_parity_at_full_size(c2):
    # from a seeded smooth positive state, in the bench's launch configuration
    case, g, j = c2
    phi0, D0 = _seeded_state(17)
    D0 = D0.astype(np.float32).astype(np.float64)
    ref = oracle.make_problem(case.sigma_t, case.alb, j.astype(np.float64), case.h, limiter="lp",
                              omega=1.93, local_iters=2)
    ref.phi, ref.D = phi0.copy(), D0.copy()
    oracle.rb_iteration(ref, 1)
    g.set_state(phi0, D0)
    g.iterate(fld.params(limiter="lp", precision="mixed", omega=1.93, local_iters=2, warm_start=1), 1)
    phi, D = g.get_state()
    from test_gpu_parity import rel_el
    e_phi, e_D = rel_el(phi, ref.phi, also=phi0), rel_el(D, ref.D, also=D0)
    print(f"128^3 one iteration: per-element phi {e_phi:.2e} D {e_D:.2e}")
    assert e_phi <= 1e-6
    assert e_D <= 3e-5


def test_render_at_full_size_matches_oracle_pixels(c2):
    # the bench's 1024^2 view of the 128^3 cloud, sampled pixels rendered one
    # by one by the oracle from the same fields
    case, g, j = c2
    cam = dict(eye=(0.5, 1.1, -1.3), target=(0.5, 0.45, 0.5), up=(0.0, 1.0, 0.0), fov_deg=40.0, width=1024,
               height=1024, background=0.05)
    # the render of a seeded phi (the oracle's renderer reads no GPU output)
    phi, D = _seeded_state(5)
    g.set_state(phi, D)
    rad, codes = g.render(fld.camera(**cam), exposure=2.0, codes=True)
    rng = np.random.default_rng(3)
    pix = [(int(x), int(y)) for x, y in rng.integers(0, 1024, size=(300, 2))]
    pix += [(512, 512), (0, 0), (1023, 1023), (300, 700)]
    want = oracle.render(case.sigma_t, case.alb, j.astype(np.float64), phi, case.h, pixels=pix, t_min=1e-6, **cam)
    got = np.array([rad[y, x] for x, y in pix], dtype=np.float64)
    scale = float(np.abs(want).max())
    assert np.abs(got - want).max() <= 1e-4 * scale
    # the cloud covers part of the view (seen from below it is darker than the background)
    assert (np.abs(rad - cam["background"]) > 0.01 * cam["background"]).mean() > 0.05
    # tone map at the sampled pixels: the oracle's codes of its own radiance
    # (+-1 where the two radiances straddle a half-integer code boundary)
    mine = oracle.tonemap(want, exposure=2.0, dtype=np.float32)
    got_codes = np.array([codes[y, x] for x, y in pix])
    assert np.abs(mine.astype(int) - got_codes.astype(int)).max() <= 1
