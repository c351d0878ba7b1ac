"""Pins of the oracle's primary ray march (Sec. 3: the radiance at the camera
is the attenuated background plus the sum over march segments of the
transmittance to the camera times Q times the segment length, with
4 pi Q = q_ri + sigma_s phi + j).

* Homogeneous medium, ray along an axis: the sum is a geometric series,
  written out here (with the clipped last segment), to rounding.
* No extinction: every segment sees T = 1, so L = Q x chord length + background.
* The scattered part of the source is sigma_s phi.
* Step -> 0: Beer-Lambert, L -> Q/sigma_t (1 - e^{-sigma_t d}) + L_bg e^{-sigma_t d}, first order.
* A medium and camera symmetric under x -> 1 - x give a mirror-symmetric image.
* Early stop at transmittance t_min changes L by at most t_min x the rest.
"""
import math

import numpy as np
import pytest

import fld_inputs
import oracle

AXIS_CAM = dict(eye=(0.5, 0.5, -2.0), target=(0.5, 0.5, 0.5), width=1, height=1)


def homogeneous(n, sigma, albedo, q, phi):
    shape = (n, n, n)
    return (np.full(shape, sigma, np.float32), np.full(shape, albedo, np.float32), np.full(shape, q),
            np.full(shape, phi))


def axis_series(sigma, Q, length, step, background):
    nseg = math.ceil(length / step - 1e-12)
    L, T = 0.0, 1.0
    for m in range(nseg):
        seg = min(step, length - m * step)
        L += T * Q * seg
        T *= math.exp(-sigma * seg)
    return L + background * T


@pytest.mark.parametrize("step_frac", [0.5, 0.3, 1.0])
def test_homogeneous_axis_ray_is_a_geometric_series(step_frac):
    n, h = 10, 0.1
    st, al, q, ph = homogeneous(n, 3.0, 0.25, 2.0, 0.0)
    img = oracle.render(st, al, q, ph, h, step=step_frac * h, background=0.7, t_min=0.0, **AXIS_CAM)
    want = axis_series(3.0, 2.0 / (4 * math.pi), 1.0, step_frac * h, 0.7)
    assert img[0, 0] == pytest.approx(want, rel=1e-13)


def test_scattered_fluence_enters_the_source():
    n, h = 10, 0.1
    st, al, q, ph = homogeneous(n, 3.0, 0.25, 0.0, 5.0)
    img = oracle.render(st, al, q, ph, h, t_min=0.0, **AXIS_CAM)
    want = axis_series(3.0, 0.25 * 3.0 * 5.0 / (4 * math.pi), 1.0, 0.5 * h, 0.0)
    assert img[0, 0] == pytest.approx(want, rel=1e-13)


def test_no_extinction_gives_source_times_chord():
    n, h = 12, 1.0 / 12
    st, al, q, ph = homogeneous(n, 0.0, 0.5, 1.5, 3.0)
    eye = np.array([-0.7, 0.2, 1.9])
    target = np.array([0.6, 0.55, 0.4])
    img = oracle.render(st, al, q, ph, h, eye=eye, target=target, width=1, height=1, background=0.25)
    d = (target - eye) / np.linalg.norm(target - eye)
    ta = (0.0 - eye) / d
    tb = (1.0 - eye) / d
    t0 = max(np.minimum(ta, tb).max(), 0.0)
    t1 = np.maximum(ta, tb).min()
    assert img[0, 0] == pytest.approx(1.5 / (4 * math.pi) * (t1 - t0) + 0.25, rel=1e-13)


def test_continuum_limit_is_beer_lambert():
    n, h, sigma, Qv, bg = 16, 1.0 / 16, 4.0, 1.0, 0.3
    st, al, q, ph = homogeneous(n, sigma, 0.5, 4 * math.pi * Qv, 0.0)
    exact = Qv / sigma * (1 - math.exp(-sigma)) + bg * math.exp(-sigma)
    errs = []
    for frac in (0.5, 0.25, 0.125, 0.0625):
        img = oracle.render(st, al, q, ph, h, step=frac * h, background=bg, t_min=0.0, **AXIS_CAM)
        errs.append(abs(img[0, 0] - exact))
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < a / b < 2.2          # first order in the step
    assert errs[-1] < 1e-2 * exact


def test_mirror_symmetric_scene_gives_mirror_symmetric_image():
    n = 14
    sig, alb = fld_inputs.cloud_medium(n, seed=3, albedo=0.9)
    sig = 0.5 * (sig + sig[:, :, ::-1])
    alb = 0.5 * (alb + alb[:, :, ::-1])
    rng = np.random.default_rng(1)
    q = rng.uniform(0, 1, sig.shape)
    q = 0.5 * (q + q[:, :, ::-1])
    ph = rng.uniform(0, 2, sig.shape)
    ph = 0.5 * (ph + ph[:, :, ::-1])
    img = oracle.render(sig, alb, q, ph, 1.0 / n, eye=(0.5, 1.3, -1.4), target=(0.5, 0.45, 0.5), width=32,
                        height=24, fov_deg=50.0, background=0.1)
    np.testing.assert_allclose(img, img[:, ::-1], rtol=1e-12, atol=1e-15)
    assert img.std() > 0.01 * img.mean()        # the image is not trivially flat


def test_early_stop_bound():
    n = 16
    sig, alb = fld_inputs.cloud_medium(n, seed=5, albedo=0.9)
    sig = sig * 20
    q = np.ones(sig.shape)
    ph = np.ones(sig.shape)
    kw = dict(eye=(0.5, 0.5, -1.5), target=(0.5, 0.5, 0.5), width=16, height=16, background=1.0)
    full = oracle.render(sig, alb, q, ph, 1.0 / n, t_min=0.0, **kw)
    cut = oracle.render(sig, alb, q, ph, 1.0 / n, t_min=1e-3, **kw)
    qmax = (1.0 + float((alb * sig).max()) * 1.0) / (4 * math.pi)
    bound = 1e-3 * (qmax * math.sqrt(3.0) + 1.0)
    assert np.abs(full - cut).max() <= bound
    assert np.abs(full - cut).max() > 0.0


def test_tonemap_codes():
    L = np.array([0.0, 1.0, 4.0, 0.5 ** 2.2, -1.0])
    np.testing.assert_array_equal(oracle.tonemap(L), [0, 255, 255, 128, 0])
    np.testing.assert_array_equal(oracle.tonemap(np.array([0.25]), exposure=4.0, gamma=1.0), [255])
    # the same codes with the decision taken in single precision
    np.testing.assert_array_equal(oracle.tonemap(L, dtype=np.float32), [0, 255, 255, 128, 0])
    np.testing.assert_array_equal(oracle.tonemap(np.array([0.25]), exposure=4.0, gamma=1.0, dtype=np.float32),
                                  [255])
