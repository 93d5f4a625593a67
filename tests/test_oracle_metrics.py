"""Pins of the oracle's tiled, mask-aware PSNR / SSIM (supplement S4.2: 128 x 128
tiles, the valid region from the mask, the dynamic range per tile):

- PSNR against its closed form for a known error on the valid texels, with
  arbitrary values on the masked-out ones (which must not count);
- SSIM of a map with itself is 1;
- SSIM against an independent evaluation of Wang et al.'s index through
  SciPy's Gaussian filter (sigma 1.5, radius 5, windows inside the tile),
  averaged over the valid centres;
- empty tiles give NaN, partial tiles keep their own size.
"""
import numpy as np
import pytest

import oracle


def test_psnr_closed_form_ignores_masked_texels():
    rng = np.random.default_rng(1)
    ref = rng.uniform(0.5, 4.0, (2, 40, 56, 3))
    mask = rng.random((2, 40, 56)) < 0.7
    pred = ref + np.where(mask[..., None], 0.01, 0.0) * np.array([1.0, -1.0, 1.0])
    pred[~mask] += 100.0                                   # garbage outside the valid region
    ps, _ = oracle.tile_metrics(pred, ref, mask, tile=16)
    for mi in range(2):
        for ty in range(3):
            for tx in range(4):
                sl = (mi, slice(16 * ty, 16 * ty + 16), slice(16 * tx, 16 * tx + 16))
                vr = ref[sl][mask[sl]]
                L = vr.max() - vr.min()
                assert abs(ps[mi, ty, tx] - 20 * np.log10(L / 0.01)) < 1e-9


def test_ssim_of_identity_and_empty_tiles():
    rng = np.random.default_rng(2)
    ref = rng.uniform(0, 3, (1, 48, 70, 3))
    mask = np.ones((1, 48, 70), bool)
    mask[0, :16, :16] = False                              # tile (0, 0) empty
    ps, ss = oracle.tile_metrics(ref, ref, mask, tile=16)
    assert np.isnan(ps[0, 0, 0]) and np.isnan(ss[0, 0, 0])
    assert np.all(np.isinf(ps[0][~np.isnan(ps[0])]))
    assert np.allclose(ss[0, :, :4][~np.isnan(ss[0, :, :4])], 1.0, atol=1e-12)
    assert np.all(np.isnan(ss[0, :, 4]))                   # the 6-texel-wide partial tiles hold no full window


def ssim_scipy(x, y, valid, L):
    ndimage = pytest.importorskip("scipy.ndimage")

    def g(a):
        return ndimage.gaussian_filter(a, sigma=1.5, truncate=5 / 1.5, mode="constant")

    C1, C2 = (0.01 * L) ** 2, (0.03 * L) ** 2
    vals = []
    for k in range(x.shape[-1]):
        a, b = x[..., k], y[..., k]
        mx, my = g(a), g(b)
        vx, vy, cxy = g(a * a) - mx * mx, g(b * b) - my * my, g(a * b) - mx * my
        s = ((2 * mx * my + C1) * (2 * cxy + C2)) / ((mx * mx + my * my + C1) * (vx + vy + C2))
        vals.append(s[5:-5, 5:-5][valid[5:-5, 5:-5]])
    return float(np.mean(np.concatenate(vals)))


def test_ssim_against_scipy_gaussian_windows():
    rng = np.random.default_rng(3)
    ref = rng.uniform(0, 2, (1, 64, 96, 3)) + np.linspace(0, 3, 96)[None, None, :, None]
    pred = ref + rng.normal(0, 0.15, ref.shape) + 0.05
    mask = rng.random((1, 64, 96)) < 0.8
    ps, ss = oracle.tile_metrics(pred, ref, mask, tile=32)
    for ty in range(2):
        for tx in range(3):
            sl = (slice(32 * ty, 32 * ty + 32), slice(32 * tx, 32 * tx + 32))
            x, y, v = pred[0][sl], ref[0][sl], mask[0][sl]
            L = y[v].max() - y[v].min()
            assert abs(ss[0, ty, tx] - ssim_scipy(x, y, v, L)) < 1e-10
            assert 0.0 < ss[0, ty, tx] < 1.0
