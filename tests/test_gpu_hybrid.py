"""GPU parity of the hybrid feature map decoder (the paper's full decoder,
Sec. 3.3 Eq. 4-5, Sec. 4) against the FP64 oracle.

- FP32 CUDA-core decode: within 1e-5 of the oracle's range (FP32 feature
  arithmetic, CUDA's erff and sincospif).
- FP16 / BF16 tensor-core decode, against the oracle on the stored FP16 /
  BF16 weights: 2e-3 of range for FP16 (features and hidden activations
  rounded to FP16 once each, FP32 accumulation), 2e-2 for BF16 (8-bit
  significand).
- Hidden widths 16, 32 and 64 (the paper's profiles use 16 and 64), clamp
  and mirror addressing, ragged query counts, and the page decode over tables
  of per-tile models with ragged requests, both output formats, a rejected
  request and untouched texels.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import edge_queries, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = {"fp32": 1e-5, "fp16": 2e-3, "bf16": 2e-2}


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def model(seed, hidden, mode=0):
    return synth.hybrid_model(seed, 128, 128, 128, 128, 32, 32, 12, 64, 24, 64, 24, hidden, address_mode=mode)


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("hidden", [16, 32, 64])
@pytest.mark.parametrize("mode", [0, 1])
def test_points_match_oracle(ndgi, prec, hidden, mode):
    m = model(40 + hidden + mode, hidden, mode)
    hm = ndgi.HybridModel.from_arrays(m)
    q = edge_queries(20_000, 41)
    if mode == 1:
        q[:2000, :2] = np.random.default_rng(42).uniform(-1.5, 2.5, (2000, 2)).astype(np.float32)
    got = ndgi.ndgi_hybrid_decode_points(hm, torch.from_numpy(q).cuda(), prec).cpu().numpy()
    ref = oracle.hybrid_decode_points(m, q, precision=prec if prec != "fp32" else "fp32")
    err = rel_err(got, ref)
    print(f"hybrid points {prec} H={hidden} mode {mode}: max|err|/range = {err:.3e}")
    assert err <= GATE[prec]
    if prec != "fp32":
        assert ndgi.ndgi_hybrid_workspace_check(hm, prec) == (0, 0)


@pytest.mark.parametrize("n", [1, 127, 129, 513, 70_001])
def test_points_ragged_counts(ndgi, n):
    m = model(50, 64)
    hm = ndgi.HybridModel.from_arrays(m)
    q = synth.random_queries(51, n)
    ref = oracle.hybrid_decode_points(m, q, precision="fp16")
    rng = float(np.ptp(oracle.hybrid_decode_points(m, synth.random_queries(52, 4096), precision="fp16")))
    out = torch.full((n + 5, 3), 7.0, device="cuda")
    ndgi.ndgi_hybrid_decode_points(hm, torch.from_numpy(q).cuda(), "fp16", out=out[:n])
    o = out.cpu().numpy()
    assert rel_err(o[:n], ref, rng) <= GATE["fp16"]
    assert np.all(o[n:] == 7.0)                                   # nothing written past n


def test_points_empty_and_bad_arguments(ndgi):
    from paper_2604_12625_gb300 import _abi as A
    import ctypes as C
    hm = ndgi.HybridModel.from_arrays(model(53, 16))
    L = A.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.ndgi_hybrid_decode_points(C.byref(hm.desc), A.NDGI_FP32, None, None, 0, None, s) == A.NDGI_OK
    assert L.ndgi_hybrid_decode_points(C.byref(hm.desc), A.NDGI_FP16, None, C.c_void_p(16), 4, C.c_void_p(16),
                                       s) == A.NDGI_ERR_INVALID_ARG     # FP16 without a workspace
    assert L.ndgi_hybrid_decode_points(C.byref(hm.desc), A.NDGI_FP8_E4M3, None, C.c_void_p(16), 4,
                                       C.c_void_p(16), s) == A.NDGI_ERR_UNSUPPORTED
    bad = A.HybridDesc.from_buffer_copy(hm.desc)
    bad.hidden = 48
    assert L.ndgi_hybrid_decode_points(C.byref(bad), A.NDGI_FP32, None, C.c_void_p(16), 4, C.c_void_p(16),
                                       s) == A.NDGI_ERR_UNSUPPORTED
    bad = A.HybridDesc.from_buffer_copy(hm.desc)
    bad.uv_w = 130
    assert L.ndgi_hybrid_decode_points(C.byref(bad), A.NDGI_FP32, None, C.c_void_p(16), 4, C.c_void_p(16),
                                       s) == A.NDGI_ERR_INVALID_ARG


def ragged_requests(seed, n_models, n, slots_x):
    rng = np.random.default_rng(seed)
    reqs = np.zeros(n, dtype=synth.PAGE_REQ_DTYPE)
    for i in range(n):
        w = 128 if i == 0 else (1 if i == 1 else int(rng.integers(1, 129)))
        h = 128 if i == 0 else (1 if i == 1 else int(rng.integers(1, 129)))
        reqs[i] = (int(rng.integers(0, n_models)), int(rng.integers(0, 128 - w + 1)), int(rng.integers(0, 128 - h + 1)),
                   w, h, np.float32(rng.random()), (i % slots_x) * 128, (i // slots_x) * 128)
    return reqs


def page_err(phys, ref, reqs):
    worst = 0.0
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = phys[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        worst = max(worst, float(np.abs(a - b).max() / max(b.max() - b.min(), 1e-3)))
    return worst


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("hidden", [16, 64])
def test_pages_match_oracle(ndgi, prec, hidden):
    s = synth.hybrid_tile_set(60 + hidden, 6, "M.64" if hidden == 64 else "M")
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, prec)
    table = ndgi.HybridTable(models, prec)
    slots_x = 4
    reqs = ragged_requests(61, 6, 14, slots_x)
    phys_h = 4 * 128
    phys = torch.full((phys_h, slots_x * 128, 4), -3.0, dtype=torch.float32, device="cuda")
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    got = phys.cpu().numpy()
    maps = [synth.hybrid_tile_of(s, i) for i in range(6)]
    ref = oracle.hybrid_decode_pages(maps, reqs, slots_x * 128, phys_h, precision=prec, fill=-3.0)
    err = page_err(got, ref, reqs)
    print(f"hybrid pages {prec} H={hidden}: max|err|/page range = {err:.3e}")
    assert err <= GATE[prec]
    assert np.array_equal(got[..., 3], ref[..., 3])              # A = 1 inside requests, untouched elsewhere
    assert np.array_equal(got[ref[..., 3] == -3.0], ref[ref[..., 3] == -3.0])
    table.close()


def test_pages_rgba16f_and_rejected_request(ndgi):
    s = synth.hybrid_tile_set(70, 3, "M.64")
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, "fp16")
    table = ndgi.HybridTable(models, "fp16")
    reqs = ragged_requests(71, 3, 6, 3)
    reqs[3]["model"] = 7                                          # out of range: rejected, others decoded
    phys = torch.zeros((2 * 128, 3 * 128, 4), dtype=torch.float16, device="cuda")
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    st, word = table.check()
    assert word == 1 and st != 0
    assert table.check() == (0, 0)                                # the word was cleared
    got = phys.float().cpu().numpy()
    good = np.delete(reqs, 3)
    maps = [synth.hybrid_tile_of(s, i) for i in range(3)]
    ref = oracle.hybrid_decode_pages(maps, good, 3 * 128, 2 * 128, precision="fp16", fill=0.0)
    # the FP16 decode's gate plus one FP16 storage rounding of each output (2^-11 relative)
    for rr in good:
        sl = (slice(rr["dst_y"], rr["dst_y"] + rr["h"]), slice(rr["dst_x"], rr["dst_x"] + rr["w"]))
        a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        bound = GATE["fp16"] * max(b.max() - b.min(), 1e-3) + np.abs(b) * 2.0 ** -11
        assert np.all(np.abs(a - b) <= bound)
    r3 = reqs[3]
    assert np.all(got[r3["dst_y"]:r3["dst_y"] + r3["h"], r3["dst_x"]:r3["dst_x"] + r3["w"]] == 0)
    table.close()


def test_timeout_injection_points_and_pages(ndgi):
    from paper_2604_12625_gb300 import _abi as A
    m = model(80, 64)
    hm = ndgi.HybridModel.from_arrays(m)
    q = torch.from_numpy(synth.random_queries(81, 5000)).cuda()
    ndgi.ndgi_hybrid_debug_inject(hm, "fp16", flags=1)
    ndgi.ndgi_hybrid_decode_points(hm, q, "fp16")
    st, word = ndgi.ndgi_hybrid_workspace_check(hm, "fp16")
    assert st == A.NDGI_ERR_TIMEOUT and word & 16
    ndgi.ndgi_hybrid_debug_inject(hm, "fp16", flags=0)
    got = ndgi.ndgi_hybrid_decode_points(hm, q, "fp16").cpu().numpy()
    assert ndgi.ndgi_hybrid_workspace_check(hm, "fp16") == (0, 0)
    assert rel_err(got, oracle.hybrid_decode_points(m, q.cpu().numpy(), precision="fp16")) <= GATE["fp16"]
    s = synth.hybrid_tile_set(82, 2, "M.64")
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, "fp16")
    table = ndgi.HybridTable(models, "fp16")
    reqs = ragged_requests(83, 2, 4, 2)
    r, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.zeros((2 * 128, 2 * 128, 4), dtype=torch.float32, device="cuda")
    ndgi.ndgi_hybrid_debug_inject(None, "fp16", table=table, flags=1)
    table.decode(r, len(reqs), phys)
    st, word = table.check()
    assert st == A.NDGI_ERR_TIMEOUT and word & 16
    ndgi.ndgi_hybrid_debug_inject(None, "fp16", table=table, flags=0)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    maps = [synth.hybrid_tile_of(s, i) for i in range(2)]
    ref = oracle.hybrid_decode_pages(maps, reqs, 2 * 128, 2 * 128, precision="fp16", fill=0.0)
    assert page_err(phys.cpu().numpy(), ref, reqs) <= GATE["fp16"]
    table.close()


def test_full_frame_sampled(ndgi):
    # the benchmark frame: 4096 M.64 tile models, 4096 whole-tile requests at their own t, RGBA16F
    s = synth.hybrid_tile_set(90, 4096, "M.64")
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, "fp16")
    table = ndgi.HybridTable(models, "fp16")
    slots_x = 64
    reqs = synth.hybrid_tile_requests(91, 4096, 4096, slots_x=slots_x)
    r, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.zeros((64 * 128, slots_x * 128, 4), dtype=torch.float32, device="cuda")
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    pick = np.random.default_rng(92).choice(len(reqs), 6, replace=False)
    pick = np.concatenate([pick, [0, len(reqs) - 1]])
    used = sorted(set(int(reqs[i]["model"]) for i in pick))
    remap = {mi: k for k, mi in enumerate(used)}
    sub = reqs[pick].copy()
    sub["model"] = [remap[int(mi)] for mi in sub["model"]]
    maps = [synth.hybrid_tile_of(s, mi) for mi in used]
    ref = oracle.hybrid_decode_pages(maps, sub, slots_x * 128, 64 * 128, precision="fp16", fill=0.0)
    err = page_err(phys.cpu().numpy(), ref, sub)
    print(f"hybrid full frame, {len(sub)} sampled pages: max|err|/page range = {err:.3e}")
    assert err <= GATE["fp16"]
    table.close()


@pytest.mark.parametrize("fast", [0, 1, 2, 3])
def test_gelu_on_device_against_oracle(ndgi, fast):
    # exact form (erff) within a few FP32 ulps; the A&S 7.1.28 forms within 2e-6 (1 + |x|); the epilogues'
    # polynomial form within 4.5e-5 + 4e-6 |x| (beyond the clamp at 4.5 the error grows as
    # |x| erfc(4.5 / sqrt 2) / 2 = 3.4e-6 |x|): far below FP16's rounding of the result, |x| 2^-12
    x = np.concatenate([np.linspace(-12, 12, 200_001), [0.0, -0.0, 1e-30, -1e-30, 30.0, -30.0, 1e4, -1e4]])
    x = x.astype(np.float32)
    y = ndgi.ndgi_debug_gelu(torch.from_numpy(x).cuda(), fast=fast).cpu().numpy().astype(np.float64)
    ref = oracle.gelu(x.astype(np.float64))
    bound = {0: 4e-7 * (1 + np.abs(x)), 1: 2e-6 * (1 + np.abs(x)), 2: 2e-6 * (1 + np.abs(x)),
             3: 4.5e-5 + 4e-6 * np.abs(x)}[fast]
    err = np.abs(y - ref)
    print(f"gelu fast={fast}: max |err| / (1 + |x|) = {np.max(err / (1 + np.abs(x))):.3e}")
    assert np.all(err <= bound)
    if fast == 2:   # the packed form rounds exactly as the scalar form
        y1 = ndgi.ndgi_debug_gelu(torch.from_numpy(x).cuda(), fast=1).cpu().numpy()
        assert np.array_equal(y.astype(np.float32), y1)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_pages_unstaged_volume_and_fractional_uv(ndgi, prec):
    # F3D 256^2 (a page's footprint exceeds the 48^2 staging: the per-texel gather runs) and F_uv at half the
    # lightmap's resolution (non-zero fractions at texel centres: the full bilinear sample runs)
    maps = [synth.hybrid_model(100 + i, 128, 128, 64, 64, 256, 256, 12, 64, 24, 64, 24, 64, address_mode=i)
            for i in range(2)]
    models = [ndgi.HybridModel.from_arrays(m) for m in maps]
    table = ndgi.HybridTable(models, prec)
    reqs = ragged_requests(101, 2, 6, 3)
    phys = torch.zeros((2 * 128, 3 * 128, 4), dtype=torch.float32, device="cuda")
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    ref = oracle.hybrid_decode_pages(maps, reqs, 3 * 128, 2 * 128, precision=prec, fill=0.0)
    err = page_err(phys.cpu().numpy(), ref, reqs)
    print(f"hybrid pages unstaged {prec}: max|err|/page range = {err:.3e}")
    assert err <= GATE[prec]
    table.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_pages_with_mirrored_border(ndgi, prec):
    # a 4-texel mirrored border per edge (supplement S3): (w + 8) x (h + 8) texels per request
    s = synth.hybrid_tile_set(130, 3, "M.64")
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, prec)
    table = ndgi.HybridTable(models, prec)
    table.set_border(4)
    reqs = ragged_requests(131, 3, 6, 3)
    reqs["w"] = np.maximum(reqs["w"], 4)
    reqs["h"] = np.maximum(reqs["h"], 4)
    reqs["x0"] = np.minimum(reqs["x0"], 128 - reqs["w"])
    reqs["y0"] = np.minimum(reqs["y0"], 128 - reqs["h"])
    reqs["dst_x"] = (np.arange(6) % 3) * 144 + 4
    reqs["dst_y"] = (np.arange(6) // 3) * 144 + 4
    phys = torch.zeros((2 * 144, 3 * 144, 4), dtype=torch.float32, device="cuda")
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    maps = [synth.hybrid_tile_of(s, i) for i in range(3)]
    ref = oracle.hybrid_decode_pages(maps, reqs, 3 * 144, 2 * 144, precision=prec, fill=0.0, border=4)
    got = phys.cpu().numpy()
    padded = reqs.copy()
    padded["dst_x"] -= 4
    padded["dst_y"] -= 4
    padded["w"] += 8
    padded["h"] += 8
    err = page_err(got, ref, padded)
    print(f"hybrid pages with border {prec}: max|err|/page range = {err:.3e}")
    assert err <= GATE[prec]
    assert np.array_equal(got[..., 3], ref[..., 3])
    # a request narrower than the border is rejected, the others decode
    reqs[2]["w"] = 3
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    assert table.check()[1] == 1
    table.close()
