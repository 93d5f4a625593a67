"""GPU parity of the tensor-core (tcgen05) decode against the FP64 oracle.

The oracle is evaluated on the parameters the decode stores (MLP weights and
biases rounded once to FP16 or BF16).  FP16 is gated at max |err| / range <=
2e-3; BF16 (8-bit significand, about 4e-3 per rounding) is reported and only
sanity-gated at 2e-2.  Features are gathered exactly as in the FP32 path.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import edge_queries, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = {"fp16": 2e-3, "bf16": 2e-2}


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def decode(ndgi, m, q, prec):
    model = ndgi.Model.from_arrays(m)
    out = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), prec).cpu().numpy()
    ndgi.ndgi_check()
    return out


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_small_points_config(ndgi, prec):
    m, q = synth.small_points_config(1)
    got = decode(ndgi, m, q, prec)
    ref = oracle.decode_points(m, q, precision=prec)
    err = rel_err(got, ref)
    print(f"{prec} small config max|err|/range = {err:.3e}")
    assert err <= GATE[prec]


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_2048_atlas_ragged(ndgi, prec):
    m = synth.points_model_2048(2)
    q = edge_queries(70_001, 21)
    got = decode(ndgi, m, q, prec)
    ref = oracle.decode_points(m, q, precision=prec)
    err = rel_err(got, ref)
    ref32 = oracle.decode_points(m, q, precision="fp32")
    print(f"{prec}: vs stored weights {err:.3e}, vs FP32 master {rel_err(got, ref32):.3e}")
    assert err <= GATE[prec]


@pytest.mark.parametrize("shape", [(8, 8, 32), (16, 8, 16), (16, 16, 64), (4, 4, 16), (8, 8, 16), (16, 8, 32)])
def test_tc_shapes(ndgi, shape):
    cs, ct, H = shape
    m = synth.model(31, 512, 512, 128, 128, cs, 12, ct, H, temporal_dtype="f32")
    q = edge_queries(5000, 22)
    got = decode(ndgi, m, q, "fp16")
    assert rel_err(got, oracle.decode_points(m, q, precision="fp16")) <= GATE["fp16"]


def test_tc_tiny_and_tail(ndgi):
    m = synth.points_model_2048(2)
    # a handful of queries has no meaningful range of its own: take the model's HDR range from 2^14 queries
    rng = float(np.ptp(oracle.decode_points(m, synth.random_queries(39, 1 << 14), precision="fp16")))
    for n in (1, 127, 129, 1000):
        q = synth.random_queries(40 + n, n)
        got = decode(ndgi, m, q, "fp16")
        ref = oracle.decode_points(m, q, precision="fp16")
        assert rel_err(got, ref, rng) <= GATE["fp16"]


def test_tc_full_size_sampled(ndgi):
    m = synth.points_model_2048(2)
    q = synth.random_queries(2, 1 << 24)
    got = decode(ndgi, m, q, "fp16")
    idx = np.random.default_rng(1).choice(q.shape[0], 1 << 15, replace=False)
    ref = oracle.decode_points(m, q[idx], precision="fp16")
    assert rel_err(got[idx], ref) <= GATE["fp16"]
    assert np.all(np.isfinite(got))


def test_tc_deterministic(ndgi):
    m = synth.points_model_2048(2)
    q = synth.random_queries(5, 100_000)
    assert np.array_equal(decode(ndgi, m, q, "fp16"), decode(ndgi, m, q, "fp16"))


SIZES = (256, 256, 512, 1024)


def page_err(phys, ref, reqs):
    worst = 0.0
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = phys[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        worst = max(worst, float(np.abs(a - b).max() / max(b.max() - b.min(), 1e-6)))
    return worst


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_pages_ragged_and_zipf(ndgi, prec):
    maps = synth.page_models(41, sizes=SIZES, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.full((1024, 1024, 4), float("nan"), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, prec, 4096, phys)
    for reqs in (synth.ragged_page_requests(5, SIZES, 40, slots_x=8, slot=128),
                 synth.zipf_page_requests(6, SIZES, 64, page=128, slots_x=8)):
        phys.fill_(float("nan"))
        r, n = ndgi.page_requests_to_device(reqs)
        plan.decode(r, n)
        st, err = plan.check()
        assert st == 0 and err == 0
        ndgi.ndgi_check()
        ref = oracle.decode_pages(maps, reqs, 1024, 1024, precision=prec)
        got = phys.cpu().numpy()
        assert page_err(got, ref, reqs) <= GATE[prec]
        assert np.all(np.isnan(got[..., 0][np.isnan(ref[..., 0])]))
    plan.close()


# (lanes, slots) of the warp-specialised page kernel: four MMA lanes, each with
# a producer warpgroup that writes the layer-1 rows of its next tile.
WS_SHAPES = ((8, 1),)


@pytest.mark.parametrize("prec", ["fp16", "bf16"])
def test_tc_pages_warp_specialised(ndgi, prec):
    # The warp-specialised kernel runs the same arithmetic as the 4 x 1 kernel
    # (same ring values, blend, MMAs and epilogue conversions), so its texels
    # equal that kernel's bit for bit; both are checked against the oracle.
    maps = synth.page_models(43, sizes=SIZES, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.full((1024, 1024, 4), float("nan"), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, prec, 4096, phys)
    for reqs in (synth.ragged_page_requests(15, SIZES, 40, slots_x=8, slot=128),
                 synth.zipf_page_requests(16, SIZES, 64, page=128, slots_x=8),
                 synth.zipf_page_requests(17, SIZES, 1, page=128, slots_x=8)):
        r, n = ndgi.page_requests_to_device(reqs)
        out = {}
        for shape in ((1, 4, 1), (1, 8, 1)):
            plan.set_shape(*shape)
            phys.fill_(float("nan"))
            plan.decode(r, n)
            st, err = plan.check()
            assert st == 0 and err == 0
            ndgi.ndgi_check()
            out[shape] = phys.cpu().numpy()
        a, b = out[(1, 4, 1)], out[(1, 8, 1)]
        assert np.array_equal(np.isnan(a), np.isnan(b))
        assert np.array_equal(np.nan_to_num(a), np.nan_to_num(b))
        ref = oracle.decode_pages(maps, reqs, 1024, 1024, precision=prec)
        assert page_err(b, ref, reqs) <= GATE[prec]
    # an empty frame leaves the texture untouched
    phys.fill_(float("nan"))
    r, n = ndgi.page_requests_to_device(synth.zipf_page_requests(18, SIZES, 4, page=128, slots_x=8))
    n.zero_()
    plan.decode(r, n)
    ndgi.ndgi_check()
    assert torch.isnan(phys).all()
    plan.close()


def test_tc_pages_full_resolution_features(ndgi):
    # features at the lightmap's own resolution: the per-texel gather path
    maps = [synth.model(60 + i, s, s, s, s, 16, 24, 8, 64, temporal_dtype="f16") for i, s in enumerate((256, 512))]
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.full((512, 512, 4), float("nan"), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    reqs = synth.ragged_page_requests(9, (256, 512), 12, slots_x=4, slot=128)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    ndgi.ndgi_check()
    ref = oracle.decode_pages(maps, reqs, 512, 512, precision="fp16")
    assert page_err(phys.cpu().numpy(), ref, reqs) <= GATE["fp16"]
    plan.close()


def test_tc_pages_autotune_and_rgba16f(ndgi):
    maps = synth.page_models(42, sizes=SIZES, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.zeros((1024, 1024, 4), dtype=torch.float16, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    reqs = synth.zipf_page_requests(7, SIZES, 64, page=128, slots_x=8)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.autotune(r, n, len(reqs))
    prec, cps, lanes, slots = plan.info()
    assert prec == 1 and cps == 1 and (lanes, slots) in WS_SHAPES + ((4, 1), (2, 2))
    with pytest.raises(ndgi.NdgiError):
        plan.set_shape(1, 3, 3)
    with pytest.raises(ndgi.NdgiError):
        plan.set_shape(2, 4, 1)
    # the same decode into an RGBA32F texture: gated against the oracle; the RGBA16F texture must then be
    # exactly its FP16 rounding (the kernels convert their FP32 result once, round to nearest even)
    phys32 = torch.zeros((1024, 1024, 4), dtype=torch.float32, device="cuda")
    plan32 = ndgi.PagesPlan(models, "fp16", 64, phys32)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024, precision="fp16")
    for shape in ((1, 2, 2), (1, 4, 1), (1, 8, 1), (1, lanes, slots)):   # every built shape decodes the same texels
        plan.set_shape(*shape)
        plan32.set_shape(*shape)
        assert plan.info()[1:] == shape
        phys.zero_()
        phys32.zero_()
        plan.decode(r, n)
        plan32.decode(r, n)
        ndgi.ndgi_check()
        assert page_err(phys32.cpu().numpy(), ref, reqs) <= GATE["fp16"]
        assert torch.equal(phys, phys32.to(torch.float16))
    plan.close()
    plan32.close()


def test_tc_gather_exhaustive_endpoint_pairs(ndgi):
    # Every (r0, r1) pair x every index through the texel-sliced copy ndgi_prepare builds: at texel
    # centres the tensor-core gather returns fl32(P35) * fl32(1/8925) exactly, like the FP32 gather.
    bits = 0
    for p in range(16):
        bits |= (p % 8) << (3 * p)
    idx = np.frombuffer(bits.to_bytes(6, "little"), np.uint8)
    pairs = np.arange(65536)
    blocks = np.zeros((65536, 8), np.uint8)
    blocks[:, 0] = pairs & 255
    blocks[:, 1] = pairs >> 8
    blocks[:, 2:] = idx
    m = synth.model(1, 512, 512, 512, 512, 4, 4, 4, 16)
    m["bc4"] = blocks.reshape(128, 128, 4, 8)
    ix, iy = np.meshgrid(np.arange(512), np.arange(512))
    q = np.stack([(ix.ravel() + 0.5) / 512, (iy.ravel() + 0.5) / 512, np.zeros(ix.size)], 1).astype(np.float32)
    x = ndgi.ndgi_debug_features_tc(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda()).cpu().numpy()
    _, p35_ref = oracle.features(m, q)
    vals = np.float32(p35_ref[:, 0, :]) * (np.float32(1) / np.float32(8925))
    assert np.array_equal(x[:, :4], vals.astype(np.float32))


@pytest.mark.parametrize("shape", [(16, 8, 64, "f16", 0), (16, 16, 64, "f32", 0), (8, 8, 32, "f32", 1),
                                   (4, 4, 16, "f32", 0), (16, 8, 32, "f16", 1)])
def test_tc_gather_matches_fp32_gather(ndgi, shape):
    cs, ct, H, tdt, mode = shape
    m = synth.model(13, 1000, 700, 256, 128, cs, 24, ct, H, temporal_dtype=tdt, address_mode=mode)
    q = edge_queries(30000, 14)
    if mode == 1:
        q[:5000, :2] = np.random.default_rng(15).uniform(-2.0, 3.0, (5000, 2)).astype(np.float32)
    model = ndgi.Model.from_arrays(m)
    qt = torch.from_numpy(q).cuda()
    x_tc = ndgi.ndgi_debug_features_tc(model, qt).cpu().numpy()
    x32, _ = ndgi.ndgi_debug_features(model, qt)
    x32 = x32.cpu().numpy()
    xr, _ = oracle.features(m, q)
    assert np.max(np.abs(x_tc - x32)) <= 2e-6 * max(1.0, np.abs(x32).max())
    assert np.max(np.abs(x_tc - xr)) <= 4e-6 * max(1.0, np.abs(xr).max())


@pytest.mark.parametrize("shape", [(1, 4, 1), (1, 8, 1)])
def test_tc_pages_mirror_address_mode(ndgi, shape):
    # The page kernels with mirrored-repeat addressing (mode 1).  A page texel's
    # taps overhang the map by at most one feature texel, which the mirror maps
    # back to the edge texel (as clamping does), so this checks the mode-1 path
    # of the ring's column range and the taps, including full pages at the corners.
    sizes = (256, 512)
    maps = [synth.model(50 + i, s, s, s // 2, s // 2, 16, 24, 8, 64, temporal_dtype="f16", address_mode=1)
            for i, s in enumerate(sizes)]
    models = [ndgi.Model.from_arrays(mm) for mm in maps]
    phys = torch.full((512, 512, 4), float("nan"), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    plan.set_shape(*shape)
    reqs = synth.ragged_page_requests(51, sizes, 12, slots_x=4, slot=128)
    corners = np.zeros(4, dtype=synth.PAGE_REQ_DTYPE)   # full pages at the corners of both maps
    for i, (mi, cx, cy) in enumerate(((0, 0, 0), (0, 1, 1), (1, 0, 1), (1, 1, 0))):
        sz = sizes[mi]
        corners[i] = (mi, cx * (sz - 128), cy * (sz - 128), 128, 128, np.float32(0.3 + 0.1 * i),
                      ((12 + i) % 4) * 128, ((12 + i) // 4) * 128)
    reqs = np.concatenate([reqs, corners])
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    assert plan.check() == (0, 0)
    ndgi.ndgi_check()
    ref = oracle.decode_pages(maps, reqs, 512, 512, precision="fp16")
    assert page_err(phys.cpu().numpy(), ref, reqs) <= GATE["fp16"]
    plan.close()


@pytest.mark.parametrize("hidden", [32, 16])
def test_tc_pages_other_hidden_widths(ndgi, hidden):
    # the page kernels at the other built hidden widths: the warp-specialised kernel equals the 4 x 1 kernel
    # bit for bit, and both meet the FP16 gate against the oracle
    sizes = (256, 512)
    maps = synth.page_models(47, sizes=sizes, hidden=hidden, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.zeros((512, 512, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    reqs = synth.ragged_page_requests(48, sizes, 16, slots_x=4, slot=128)
    r, n = ndgi.page_requests_to_device(reqs)
    out = {}
    for shape in ((1, 4, 1), (1, 8, 1)):
        plan.set_shape(*shape)
        phys.zero_()
        plan.decode(r, n)
        assert plan.check() == (0, 0)
        out[shape] = phys.cpu().numpy()
    assert np.array_equal(out[(1, 4, 1)], out[(1, 8, 1)])
    ref = oracle.decode_pages(maps, reqs, 512, 512, precision="fp16", fill=0.0)
    assert page_err(out[(1, 8, 1)], ref, reqs) <= GATE["fp16"]
    plan.close()
