"""GPU parity of the gather and the FP32 point decode against the FP64 oracle.

BC values: the palette numerators P35 the kernel used must equal the
oracle's exactly (integer work).  RGB: max |err| / HDR range <= 1e-5 for the
FP32 path (range = max - min over all channels of the oracle output of the
evaluated set).
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import edge_queries, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def test_p35_exhaustive_endpoint_pairs(ndgi):
    # Every (r0, r1) pair x every index: 65536 (block, plane) pairs, texel p holds index p % 8.
    bits = 0
    for p in range(16):
        bits |= (p % 8) << (3 * p)
    idx = np.frombuffer(bits.to_bytes(6, "little"), np.uint8)
    pairs = np.arange(65536)
    blocks = np.zeros((65536, 8), np.uint8)
    blocks[:, 0] = pairs & 255
    blocks[:, 1] = pairs >> 8
    blocks[:, 2:] = idx
    bc4 = blocks.reshape(128, 128, 4, 8)            # 512x512 texels, 4 planes
    m = synth.model(1, 512, 512, 512, 512, 4, 4, 4, 16)
    m["bc4"] = bc4
    ix, iy = np.meshgrid(np.arange(512), np.arange(512))
    q = np.stack([(ix.ravel() + 0.5) / 512, (iy.ravel() + 0.5) / 512, np.zeros(ix.size)], 1).astype(np.float32)
    x, p35 = ndgi.ndgi_debug_features(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda())
    _, p35_ref = oracle.features(m, q)
    assert np.array_equal(p35.cpu().numpy()[:, 0, :], p35_ref[:, 0, :])
    # the decoded value is fl32(P35) * fl32(1/8925): at texel centres v_s is that value exactly
    vals = np.float32(p35_ref[:, 0, :]) * (np.float32(1) / np.float32(8925))
    assert np.array_equal(x.cpu().numpy()[:, :4], vals.astype(np.float32))


@pytest.mark.parametrize("shape", [(8, 8, 32, "f32"), (16, 8, 64, "f16"), (16, 16, 64, "f32")])
def test_gather_bit_exact_random(ndgi, shape):
    cs, ct, H, tdt = shape
    m = synth.model(11, 1000, 700, 256, 128, cs, 24, ct, H, temporal_dtype=tdt)
    q = edge_queries(20000, 12)
    x, p35 = ndgi.ndgi_debug_features(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda())
    xr, pr = oracle.features(m, q)
    assert np.array_equal(p35.cpu().numpy(), pr)
    assert np.max(np.abs(x.cpu().numpy() - xr)) < 2e-6 * max(1.0, np.abs(xr).max())


def test_keyframes_exact(ndgi):
    m = synth.model(3, 64, 64, 16, 16, 4, 8, 4, 16)
    q = np.zeros((8, 3), np.float32)
    q[:, 2] = np.arange(8) / 8
    x, _ = ndgi.ndgi_debug_features(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda())
    assert np.array_equal(x.cpu().numpy()[:, 4:], m["temporal"])


def test_mirror_mode_out_of_range(ndgi):
    m = synth.model(4, 64, 64, 32, 32, 4, 8, 4, 16, address_mode=1)
    q = np.random.default_rng(5).uniform(-2.0, 3.0, (5000, 3)).astype(np.float32)
    x, p35 = ndgi.ndgi_debug_features(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda())
    xr, pr = oracle.features(m, q)
    assert np.array_equal(p35.cpu().numpy(), pr)
    assert np.max(np.abs(x.cpu().numpy() - xr)) < 2e-5


def test_fp32_small_points_config(ndgi):
    m, q = synth.small_points_config(1)        # 256^2 lightmap, 64^2x8 BC4, T=8, 16->32->32->3, 4 times
    got = ndgi.ndgi_decode_points(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    ref = oracle.decode_points(m, q)
    assert rel_err(got, ref) <= FP32_TOL


def test_fp32_2048_atlas_edges_and_ragged(ndgi):
    m = synth.points_model_2048(2)
    model = ndgi.Model.from_arrays(m)
    q = edge_queries(100_003, 7)               # not a multiple of any tile
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    ref = oracle.decode_points(m, q)
    assert rel_err(got, ref) <= FP32_TOL
    # n = 1 and n = 0
    one = ndgi.ndgi_decode_points(model, torch.from_numpy(q[:1]).cuda(), "fp32").cpu().numpy()
    assert rel_err(one, ref[:1], rng=ref.max() - ref.min()) <= FP32_TOL
    empty = ndgi.ndgi_decode_points(model, torch.zeros((0, 3), dtype=torch.float32, device="cuda"), "fp32")
    assert empty.shape == (0, 3)


def test_fp32_full_size_sampled(ndgi):
    # 2^24 random queries at the benchmark's size; the oracle checks a seeded sample.
    m = synth.points_model_2048(2)
    model = ndgi.Model.from_arrays(m)
    q = synth.random_queries(2, 1 << 24)
    out = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    idx = np.random.default_rng(0).choice(q.shape[0], 1 << 15, replace=False)
    ref = oracle.decode_points(m, q[idx])
    assert rel_err(out[idx], ref) <= FP32_TOL
    assert np.all(np.isfinite(out))


def test_fp32_deterministic(ndgi):
    m = synth.points_model_2048(2)
    model = ndgi.Model.from_arrays(m)
    q = torch.from_numpy(synth.random_queries(9, 50000)).cuda()
    a = ndgi.ndgi_decode_points(model, q, "fp32")
    b = ndgi.ndgi_decode_points(model, q, "fp32")
    assert torch.equal(a, b)


def test_unsupported_shape_rejected(ndgi):
    m = synth.model(4, 64, 64, 32, 32, 4, 8, 4, 24)
    with pytest.raises(ndgi.NdgiError) as e:
        ndgi.ndgi_decode_points(ndgi.Model.from_arrays(m), torch.zeros((4, 3), device="cuda"), "fp32")
    assert e.value.status == 2


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_non_finite_and_out_of_range_queries(ndgi, prec):
    # Coordinates outside [0, 1) sample the clamped edge texels (the default
    # address mode); NaN, +-inf and huge values give in-bounds taps and finite
    # results without any error, and the queries around them decode as usual.
    m = synth.model(33, 256, 256, 128, 128, 16, 24, 8, 64, temporal_dtype="f16")
    model = ndgi.Model.from_arrays(m)
    q = synth.random_queries(34, 4000)
    q[:1000, :2] = q[:1000, :2] * 3.0 - 1.0                 # u, v in [-1, 2): clamped taps
    bad = np.array([np.nan, np.inf, -np.inf, 1e30, -1e30], np.float32)
    rows = []
    for i, b in enumerate(bad):
        for axis in range(3):
            r = 1000 + 3 * i + axis
            q[r, axis] = b
            rows.append(r)
    q[1100, :] = np.nan
    rows.append(1100)
    got = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), prec).cpu().numpy()
    ndgi.ndgi_check()
    assert np.all(np.isfinite(got))
    ok = np.ones(len(q), bool)
    ok[rows] = False
    ref = oracle.decode_points(m, q[ok], precision=prec if prec != "fp32" else "fp32")
    assert rel_err(got[ok], ref) <= (FP32_TOL if prec == "fp32" else 2e-3)
