"""Pins of the oracle's quarter-resolution path (Sec. 6.2: phi solved on a grid
with a quarter of the data's resolution per axis, used at full resolution in
the ray march).

* Box averages: a field linear in the voxel index averages, over a full
  block, to its value at the block centre; constants stay constant; a partial
  block at the far face averages the voxels that exist (written out by hand).
* The coarse albedo is mean(albedo sigma_t) / mean(sigma_t).
* Trilinear upsampling reproduces a coarse field that is linear in space at
  every fine centre between the outermost coarse centres, and constants
  everywhere.
* The per-pixel renderer equals the full-image renderer.
"""
import numpy as np
import pytest

import fld_inputs
import oracle


def test_linear_field_averages_to_block_centre():
    nz, ny, nx, f = 8, 12, 16, 4
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = 1.0 + 0.5 * i - 0.25 * j + 2.0 * k
    st = np.full((nz, ny, nx), 3.0, np.float32)
    al = np.full((nz, ny, nx), 0.5, np.float32)
    stc, alc, qc = oracle.downsample(st, al, q, f)
    K, J, I = np.meshgrid(np.arange(nz // f), np.arange(ny // f), np.arange(nx // f), indexing="ij")
    ci, cj, ck = f * I + (f - 1) / 2, f * J + (f - 1) / 2, f * K + (f - 1) / 2
    np.testing.assert_allclose(qc, 1.0 + 0.5 * ci - 0.25 * cj + 2.0 * ck, rtol=1e-14)
    np.testing.assert_allclose(stc, 3.0, rtol=1e-15)
    np.testing.assert_allclose(alc, 0.5, rtol=1e-15)


def test_partial_blocks_and_albedo_weighting():
    st = np.array([[[1.0, 3.0, 2.0, 0.0, 5.0]]], np.float32)       # nx = 5, ny = nz = 1
    al = np.array([[[0.5, 1.0, 0.25, 0.9, 0.2]]], np.float32)
    q = np.array([[[2.0, 4.0, 6.0, 8.0, 10.0]]])
    stc, alc, qc = oracle.downsample(st, al, q, 4)
    assert stc.shape == (1, 1, 2)
    assert stc[0, 0, 0] == pytest.approx((1 + 3 + 2 + 0) / 4)
    assert alc[0, 0, 0] == pytest.approx((0.5 * 1 + 1.0 * 3 + 0.25 * 2 + 0.9 * 0) / (1 + 3 + 2 + 0))
    assert qc[0, 0, 0] == pytest.approx(5.0)
    # the partial block holds one fine voxel
    assert (stc[0, 0, 1], qc[0, 0, 1]) == (pytest.approx(5.0), pytest.approx(10.0))
    assert alc[0, 0, 1] == pytest.approx(np.float32(0.2), rel=1e-7)
    # vacuum block: albedo 0
    st0 = np.zeros((4, 4, 4), np.float32)
    _, al0, _ = oracle.downsample(st0, np.full((4, 4, 4), 0.7, np.float32), np.zeros((4, 4, 4)), 4)
    assert al0[0, 0, 0] == 0.0


def test_upsample_reproduces_linear_and_constant_fields():
    f, h = 4, 1.0 / 32
    shape = (32, 24, 28)
    cshape = tuple((s + f - 1) // f for s in shape)
    K, J, I = np.meshgrid(*[np.arange(s) for s in cshape], indexing="ij")
    H = f * h
    lin = lambda x, y, z: 0.3 + 1.5 * x - 0.7 * y + 2.2 * z
    pc = lin((I + 0.5) * H, (J + 0.5) * H, (K + 0.5) * H)
    fine = oracle.upsample(pc, shape, h, f)
    k, j, i = np.meshgrid(*[np.arange(s) for s in shape], indexing="ij")
    x, y, z = (i + 0.5) * h, (j + 0.5) * h, (k + 0.5) * h
    inside = ((x >= 0.5 * H) & (x <= (cshape[2] - 0.5) * H) & (y >= 0.5 * H) & (y <= (cshape[1] - 0.5) * H)
              & (z >= 0.5 * H) & (z <= (cshape[0] - 0.5) * H))
    np.testing.assert_allclose(fine[inside], lin(x, y, z)[inside], rtol=1e-13)
    assert inside.mean() > 0.5
    np.testing.assert_allclose(oracle.upsample(np.full(cshape, 2.5), shape, h, f), 2.5, rtol=1e-15)
    # padded coarse input is accepted
    padded = np.pad(pc, 1, constant_values=-1.0)
    np.testing.assert_array_equal(oracle.upsample(padded, shape, h, f), fine)


def test_render_pixels_equal_full_image():
    n = 14
    sig, alb = fld_inputs.cloud_medium(n, seed=3, albedo=0.9)
    rng = np.random.default_rng(1)
    q, ph = rng.uniform(0, 1, sig.shape), rng.uniform(0, 2, sig.shape)
    kw = dict(eye=(0.5, 1.3, -1.4), target=(0.5, 0.45, 0.5), width=32, height=24, fov_deg=50.0, background=0.1)
    img = oracle.render(sig, alb, q, ph, 1.0 / n, **kw)
    pix = [(3, 4), (31, 23), (0, 0), (17, 11)]
    got = oracle.render(sig, alb, q, ph, 1.0 / n, pixels=pix, **kw)
    np.testing.assert_array_equal(got, [img[y, x] for x, y in pix])
