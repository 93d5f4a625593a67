"""GPU parity of the point decode's decoded-texel cache path.

With many queries per feature texel, a tensor-core point decode first
decodes every BC4 texel of the map once into an FP16 cache (the value
fl32(P35) * fl32(1/8925) rounded to FP16, as the page decode's feature ring)
and then blends each query's four cached taps in half2 arithmetic.

- The gather is checked bit for bit against an independent NumPy statement
  of that arithmetic (taps and fractions from the texel-centre convention,
  weights (1 - f) and f rounded to FP16, the four weight products and the
  three blend steps each rounded once to FP16), and against the oracle's
  FP64 features within the bound that arithmetic implies.
- The decode is checked against the FP64 oracle on the stored FP16 / BF16
  parameters at the FP16 gate (2e-3 of range; BF16 sanity 2e-2), for clamp
  and mirror addressing, and the library's path query reports each path.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import edge_queries, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def h(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


def cache_blend_reference(m, q):
    """The cache path's spatial features, stated independently in NumPy (FP16 roundings made explicit)."""
    _, p35 = oracle.features(m, q)                                   # [n][4][cs], taps (x0,y0),(x1,y0),(x0,y1),(x1,y1)
    f = h(p35.astype(np.float32) * (np.float32(1) / np.float32(8925)))
    fx = q[:, 0].astype(np.float64) * m["feat_w"] - 0.5
    fy = q[:, 1].astype(np.float64) * m["feat_h"] - 0.5
    fx, fy = (fx - np.floor(fx))[:, None], (fy - np.floor(fy))[:, None]
    wx0, wx1, wy0, wy1 = h(1 - fx), h(fx), h(1 - fy), h(fy)
    w = [h(wx0 * wy0), h(wx1 * wy0), h(wx0 * wy1), h(wx1 * wy1)]
    v = h(w[0] * f[:, 0])
    for k in (1, 2, 3):
        v = h(w[k] * f[:, k] + v)                                    # exact in FP64, one rounding: an FMA
    return v


@pytest.mark.parametrize("shape", [(16, 8, 64, 0), (8, 8, 32, 1), (4, 4, 16, 0), (16, 16, 64, 1)])
def test_cache_gather_exact_arithmetic_and_bound(ndgi, shape):
    cs, ct, H, mode = shape
    m = synth.model(91, 512, 512, 256, 128, cs, 24, ct, H, temporal_dtype="f16", address_mode=mode)
    q = edge_queries(40_000, 92)
    if mode == 1:
        q[:4000, :2] = np.random.default_rng(93).uniform(-1.5, 2.5, (4000, 2)).astype(np.float32)
    model = ndgi.Model.from_arrays(m)
    x = ndgi.ndgi_debug_features_cache(model, torch.from_numpy(q).cuda()).cpu().numpy().astype(np.float64)
    want = cache_blend_reference(m, q)
    assert np.array_equal(x[:, :cs], want)
    xr, _ = oracle.features(m, q)
    # features lie in [0, 1]: the FP16 rounding of each tap value (2^-12), of the four weights (3 roundings each,
    # relative 2^-11 of a weight <= 1) and of the four blend steps (2^-12 each) bound the error by 17 * 2^-12
    assert np.abs(x[:, :cs] - xr[:, :cs]).max() <= 17 * 2.0 ** -12
    assert np.abs(x[:, cs:] - xr[:, cs:]).max() <= 4e-6 * max(1.0, np.abs(xr[:, cs:]).max())   # temporal: FP32


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
@pytest.mark.parametrize("mode", [0, 1])
def test_cache_path_decode_matches_oracle(ndgi, prec, mode):
    m = synth.model(94 + mode, 512, 512, 256, 256, 16, 24, 8, 64, temporal_dtype="f16", address_mode=mode)
    model = ndgi.Model.from_arrays(m)
    q = edge_queries(70_001, 95)
    assert ndgi.ndgi_decode_points_path(model, prec, q.shape[0]) == "cache_ws"
    assert ndgi.ndgi_decode_points_path(model, prec, 1000) == "direct"
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), prec).cpu().numpy()
    st, word = ndgi.ndgi_workspace_check(model, prec)
    assert st == 0 and word == 0
    ref = oracle.decode_points(m, q, precision=prec)
    err = rel_err(got, ref)
    print(f"cache path {prec} mode {mode}: max|err|/range = {err:.3e}")
    assert err <= (2e-3 if prec == "fp16" else 2e-2)
    # the direct gather of the same queries (fewer per call) agrees within the same gate
    direct = np.concatenate([ndgi.ndgi_decode_points(model, torch.from_numpy(q[i:i + 1000]).cuda(), prec).cpu().numpy()
                             for i in range(0, 5000, 1000)])
    assert rel_err(direct, ref[:5000], float(np.ptp(ref))) <= (2e-3 if prec == "fp16" else 2e-2)


def test_cache_path_full_size_sampled(ndgi):
    # the benchmark workload: 2^24 queries of the 2048^2 atlas (1024^2 x 16 planes, a 32 MiB cache)
    m = synth.points_model_2048(2)
    model = ndgi.Model.from_arrays(m)
    q = synth.random_queries(2, 1 << 24)
    assert ndgi.ndgi_decode_points_path(model, "fp16", q.shape[0]) == "cache_ws"
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), "fp16").cpu().numpy()
    assert ndgi.ndgi_workspace_check(model, "fp16") == (0, 0)
    idx = np.random.default_rng(7).choice(q.shape[0], 1 << 15, replace=False)
    ref = oracle.decode_points(m, q[idx], precision="fp16")
    assert rel_err(got[idx], ref) <= 2e-3
    assert np.all(np.isfinite(got))


def test_map_too_large_for_the_cache_gathers_directly(ndgi):
    # 2048^2 x 16 planes would need a 128 MiB cache: no cache in the workspace, the direct gather runs
    m = synth.model(96, 4096, 4096, 2048, 2048, 16, 24, 8, 64, temporal_dtype="f16")
    model = ndgi.Model.from_arrays(m)
    assert ndgi.ndgi_decode_points_path(model, "fp16", 1 << 24) == "direct"
    q = synth.random_queries(97, 1 << 16)
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), "fp16").cpu().numpy()
    assert rel_err(got, oracle.decode_points(m, q, precision="fp16")) <= 2e-3


@pytest.mark.parametrize("shape", [(16, 8, 64), (16, 16, 64), (8, 8, 32), (4, 4, 16), (16, 8, 16)])
@pytest.mark.parametrize("n", [600, 5000, 70_001])
def test_cache_path_shapes_and_tails(ndgi, shape, n):
    # the warp-specialised kernel (shapes whose slot fits the merged layout) and the four-lane kernel both
    # run the cache path; n = 600 leaves most lanes without a tile, odd n a ragged last tile
    cs, ct, H = shape
    m = synth.model(98, 128, 128, 32, 32, cs, 12, ct, H, temporal_dtype="f32")
    model = ndgi.Model.from_arrays(m)
    q = edge_queries(n - 216, 99)
    path = ndgi.ndgi_decode_points_path(model, "fp16", q.shape[0])
    assert path == ("cache" if shape == (16, 16, 64) else "cache_ws")
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), "fp16").cpu().numpy()
    assert ndgi.ndgi_workspace_check(model, "fp16") == (0, 0)
    ref = oracle.decode_points(m, q, precision="fp16")
    rng = float(np.ptp(oracle.decode_points(m, synth.random_queries(100, 1 << 14), precision="fp16")))
    assert rel_err(got, ref, rng) <= 2e-3
