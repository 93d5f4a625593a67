"""GPU tiled mask-aware PSNR / SSIM (supplement S4.2) against the oracle's
(pinned on its own against closed forms and SciPy's Gaussian filter):
ragged maps with partial tiles, masks with empty tiles, HDR values."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.mark.parametrize("masked", [False, True])
def test_tile_metrics_match_oracle(ndgi, masked):
    rng = np.random.default_rng(5)
    n, h, w, c = 3, 300, 260, 3
    ref = (rng.gamma(2.0, 0.5, (n, h, w, c)) + np.linspace(0, 4, w)[None, None, :, None]).astype(np.float32)
    pred = (ref + rng.normal(0, 0.05, ref.shape) * (1 + ref)).astype(np.float32)
    mask = None
    if masked:
        mask = (rng.random((n, h, w)) < 0.75).astype(np.uint8)
        mask[0, :128, :128] = 0                             # one empty tile
    ps, ss = ndgi.ndgi_tile_metrics(torch.from_numpy(pred).cuda(), torch.from_numpy(ref).cuda(),
                                    None if mask is None else torch.from_numpy(mask).cuda(), tile=128)
    ps, ss = ps.cpu().numpy(), ss.cpu().numpy()
    rp, rs = oracle.tile_metrics(pred, ref, mask, tile=128)
    assert np.array_equal(np.isnan(ps), np.isnan(rp)) and np.array_equal(np.isnan(ss), np.isnan(rs))
    ok = ~np.isnan(rp)
    assert np.max(np.abs(ps[ok] - rp[ok])) <= 1e-6 * np.max(np.abs(rp[ok]))
    ok = ~np.isnan(rs)
    print(f"masked={masked}: max |dPSNR| {np.max(np.abs(ps - rp)[~np.isnan(rp)]):.2e} dB, "
          f"max |dSSIM| {np.max(np.abs(ss[ok] - rs[ok])):.2e}")
    assert np.max(np.abs(ss[ok] - rs[ok])) <= 1e-5


def test_tile_metrics_identical_maps(ndgi):
    ref = torch.rand((1, 128, 256, 3), device="cuda") * 4
    ps, ss = ndgi.ndgi_tile_metrics(ref, ref.clone(), tile=128)
    assert torch.all(torch.isinf(ps)) and torch.allclose(ss, torch.ones_like(ss), atol=1e-6)
