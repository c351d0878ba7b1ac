"""The seeded input generator: deterministic, in range, vacuum outside the
sphere, FP32 output."""
import numpy as np

import fld_inputs


def test_fbm_deterministic_and_in_range():
    a = fld_inputs.fbm_noise(24, 20, 16, 1.0 / 24, seed=3)
    b = fld_inputs.fbm_noise(24, 20, 16, 1.0 / 24, seed=3)
    c = fld_inputs.fbm_noise(24, 20, 16, 1.0 / 24, seed=4)
    assert a.shape == (16, 20, 24)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, c)
    assert a.min() >= 0.0 and a.max() <= 1.0


def test_cloud_medium_recipe():
    sig, alb = fld_inputs.cloud_medium(32, seed=0, albedo=0.95)
    assert sig.dtype == np.float32 and alb.dtype == np.float32
    n = 32
    x = (np.arange(n) + 0.5) / n - 0.5
    r2 = x[:, None, None] ** 2 + x[None, :, None] ** 2 + x[None, None, :] ** 2
    assert np.all(sig[r2 > 0.45 ** 2] == 0.0)
    assert sig.max() <= 200.0 * 0.65 ** 1.5 + 1e-3
    assert (sig > 0).mean() > 0.05
    assert np.all(alb == np.float32(0.95))


def test_point_source_unit_power():
    ps = fld_inputs.point_source_medium(32)
    assert ps.centre == (16, 16, 16)
    assert ps.j.sum() * ps.h ** 3 == 1.0
    assert ps.j[16, 16, 16] == 32768.0


def test_batch_cases_reproducible():
    a = fld_inputs.batch_cases(64, seed=7)
    b = fld_inputs.batch_cases(64, seed=7)
    assert [x["n"] for x in a] == [x["n"] for x in b]
    assert set(x["n"] for x in a) <= {32, 48, 64, 96, 128, 160}
    assert all(0.8 <= x["albedo"] <= 0.99 for x in a)
