"""GPU parity of the FP8 (E4M3) page decode against the oracle's FP8 decode.

Bit-exact: the stored FP8 image (scales, weight codes, three-term biases) and
the decode of a model on which every quantisation is exact.  Elsewhere the
decode quantises activations that the two sides compute in different
arithmetic (FP16 ring features and FP32 accumulation here, FP64 there), so an
activation near an E4M3 rounding boundary may round to the neighbouring
value: the gate is on the error distribution, and the error against the FP32
master weights is reported beside it.  The calibration maxima are passed to
both sides (rounded to FP32 first), so both derive the same scales.
"""
import numpy as np
import pytest

import oracle
import synth
from _models import fp8_exact_model

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("shape", [(16, 8, 64), (16, 16, 64), (16, 8, 32)])
def test_fp8_image_matches_oracle(ndgi, shape):
    cs, ct, H = shape
    m = synth.model(70 + H + ct, 256, 256, 128, 128, cs, 24, ct, H, temporal_dtype="f16")
    am = f32(oracle.fp8_calibrate(m, synth.random_queries(71, 1 << 12)))
    model = ndgi.Model.from_arrays(m)
    ndgi.ndgi_prepare_fp8(model, am)
    got = ndgi.ndgi_fp8_unpack(model)
    sc = oracle.fp8_scales(m, am)
    for k in ("a1", "a2", "a3", "out", "s1", "s2", "s3"):
        assert got["scales"][k] == sc[k], k
    assert got["scales"]["status"] == 0
    wq = oracle.fp8_weights(m, am)
    for k in ("w1", "w2", "w3"):
        assert np.array_equal(got[k].astype(np.float64), wq[k]), k
    _, v2, b2 = oracle.fp8_bias(np.asarray(m["b2"], np.float64), sc["a3"])
    _, v3, b3 = oracle.fp8_bias(np.asarray(m["b3"], np.float64), sc["out"])
    assert got["scales"]["v2"] == v2 and got["scales"]["v3"] == v3
    assert np.array_equal(got["b2"].astype(np.float64), b2)
    assert np.array_equal(got["b3"].astype(np.float64), b3)


def test_fp8_calibration_matches_oracle(ndgi):
    m = synth.model(72, 256, 256, 128, 128, 16, 24, 8, 64, temporal_dtype="f16")
    q = synth.random_queries(73, 1 << 14)
    got = ndgi.ndgi_calibrate_fp8(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda()).cpu().numpy()
    ref = oracle.fp8_calibrate(m, q)
    assert np.all(np.abs(got - ref) <= 1e-5 * ref)


def test_fp8_exact_model_is_bit_exact(ndgi):
    m = fp8_exact_model()
    model = ndgi.Model.from_arrays(m)
    am = np.array([1.0, 3.5, 1.875])
    ndgi.ndgi_prepare_fp8(model, am)
    phys = torch.zeros((16, 48, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan([model], "fp8", 8, phys)
    reqs = np.zeros(3, dtype=synth.PAGE_REQ_DTYPE)
    for i, (t, x0) in enumerate(((0.0, 0), (0.375, 8), (0.875, 16))):
        reqs[i] = (0, x0, 4, 16, 12, np.float32(t), 16 * i, 0)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    assert plan.check() == (0, 0)
    ndgi.ndgi_check()
    ref = oracle.decode_pages([m], reqs, 48, 16, precision="fp8", act_max=am[None], fill=0.0)
    assert np.array_equal(phys.cpu().numpy().astype(np.float64), ref)
    assert np.array_equal(ref, oracle.decode_pages([m], reqs, 48, 16, precision="fp32", fill=0.0))
    plan.close()


TIGHT = (1e-2, 2e-2, 5e-2)


def page_errors(got, ref, reqs):
    """Per request: (max, rms, then the share of values above each TIGHT bound) of |got - ref| over RGB,
    relative to the page's range."""
    out = []
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        rng = max(b.max() - b.min(), 1e-6)
        d = np.abs(a - b) / rng
        out.append((d.max(), np.sqrt((d ** 2).mean()), *[(d > x).mean() for x in TIGHT]))
    return np.array(out)


@pytest.mark.parametrize("ct", [8, 16])
def test_fp8_pages_error_distribution(ndgi, ct):
    sizes = (256, 256, 512, 1024)
    maps = [synth.model(80 + i, s, s, s // 2, s // 2, 16, 24, ct, 64, temporal_dtype="f16")
            for i, s in enumerate(sizes)]
    am = np.stack([f32(oracle.fp8_calibrate(mm, synth.random_queries(90 + i, 1 << 14))) for i, mm in enumerate(maps)])
    models = [ndgi.Model.from_arrays(mm) for mm in maps]
    for mod, a in zip(models, am):
        ndgi.ndgi_prepare_fp8(mod, a)
    phys = torch.zeros((1024, 1024, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp8", 256, phys)
    reqs = synth.ragged_page_requests(95, sizes, 40, slots_x=8, slot=128)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    assert plan.check() == (0, 0)
    ndgi.ndgi_check()
    got = phys.cpu().numpy()
    # the warp-specialised kernel (four MMA lanes, each with a producer warpgroup)
    # runs the same arithmetic: identical texels
    plan.set_shape(1, 8, 1)
    phys.zero_()
    plan.decode(r, n)
    assert plan.check() == (0, 0)
    ndgi.ndgi_check()
    assert np.array_equal(phys.cpu().numpy(), got)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024, precision="fp8", act_max=am, fill=0.0)
    e = page_errors(got, ref, reqs)
    e32 = page_errors(got, oracle.decode_pages(maps, reqs, 1024, 1024, precision="fp32", fill=0.0), reqs)
    share = [float(np.average(e[:, 2 + i], weights=reqs["w"] * reqs["h"])) for i in range(len(TIGHT))]
    print(f"ct={ct}: vs oracle FP8 max {e[:, 0].max():.3e} rms {e[:, 1].mean():.3e} share above "
          + ", ".join(f"{x:g}: {v:.2e}" for x, v in zip(TIGHT, share))
          + f"; vs FP32 master max {e32[:, 0].max():.3e} rms {e32[:, 1].mean():.3e}")
    # rounding flips of single activations (one E4M3 step, 6-12% of the value) give errors around 1e-2 of the
    # range; the bulk agrees closely and large errors are rare.  test_fp8_rounding_accounting shows layer by
    # layer that every flip is a value within the kernel's pre-rounding error of a rounding boundary; the
    # largest page error measured from such flips is 0.13 of the page range
    assert share[0] <= 0.06 and share[2] <= 0.01
    assert e[:, 1].mean() <= 0.01 and e[:, 0].max() <= 0.15
    assert e32[:, 1].mean() <= 0.08


def test_fp8_refusals(ndgi):
    m = synth.model(74, 64, 64, 32, 32, 16, 8, 8, 16, temporal_dtype="f32")
    model = ndgi.Model.from_arrays(m)
    with pytest.raises(ndgi.NdgiError):          # hidden 16: no FP8 image
        ndgi.ndgi_prepare_fp8(model, [1.0, 1.0, 1.0])
    m = synth.model(75, 64, 64, 32, 32, 16, 8, 8, 64, temporal_dtype="f32")
    model = ndgi.Model.from_arrays(m)
    with pytest.raises(ndgi.NdgiError):          # FP8 needs ndgi_prepare_fp8
        ndgi.ndgi_prepare(model, "fp8")
    with pytest.raises(ndgi.NdgiError):          # negative maximum
        ndgi.ndgi_prepare_fp8(model, [1.0, -1.0, 1.0])
    ndgi.ndgi_prepare_fp8(model, [1.0, 4.0, 4.0])
    q = torch.from_numpy(synth.random_queries(76, 100)).cuda()
    with pytest.raises(ndgi.NdgiError):          # points: FP8 is built for pages
        ndgi.ndgi_decode_points(model, q, "fp8")


def code_value(c):
    """E4M3 code -> value, from the format (sign, 4-bit exponent with bias 7, 3-bit mantissa; subnormals)."""
    c = np.asarray(c, np.int64)
    e, mnt = (c >> 3) & 15, c & 7
    v = np.where(e == 0, mnt / 8.0 * 2.0 ** -6, (1 + mnt / 8.0) * 2.0 ** (e.astype(np.float64) - 7))
    return np.where(c & 0x80, -v, v)


def test_code_value_matches_the_oracle_rounding():
    codes = np.array([c for c in range(256) if c not in (0x7F, 0xFF)])   # the two NaN codes
    v, back = oracle.e4m3(code_value(codes))
    assert np.array_equal(v, code_value(codes))
    assert np.array_equal(back[codes != 0x80], codes[codes != 0x80])    # -0 rounds to +0's code


def adjacent_flip_ok(exact, code_kernel, code_ref, tol):
    """Every mismatch is a one-step flip of a value within tol of the rounding boundary between the two codes."""
    bad = code_kernel != code_ref
    if not bad.any():
        return True, 0
    a, b = code_value(code_kernel[bad]), code_value(code_ref[bad])
    mid = 0.5 * (a + b)
    grid = np.unique(code_value(np.arange(256)[(np.arange(256) != 0x7F) & (np.arange(256) != 0xFF)]))
    ia, ib = np.searchsorted(grid, a), np.searchsorted(grid, b)
    ok = (np.abs(ia - ib) == 1) & (np.abs(exact[bad] - mid) <= tol[bad])
    return bool(ok.all()), int(bad.sum())


def h16(x):
    return np.asarray(x, np.float64).astype(np.float16).astype(np.float64)


@pytest.mark.parametrize("item", [0, 2])
def test_fp8_rounding_accounting(ndgi, item):
    # Operands and accumulators of one 128-texel tile, dumped by the 4x1 kernel, checked layer by layer:
    # each layer's input codes are the exact rounding of what produced them (A1: the kernel's FP16 blend,
    # emulated bit for bit; A2, A3: the dumped FP32 accumulators), and each accumulator is within FP32
    # accumulation error of the exact sum of products of the dumped codes and the stored weights.  So every
    # code that differs from the oracle's FP64 decode is a one-step flip of a value inside the kernel's
    # documented pre-rounding error of an E4M3 rounding boundary.
    cs, ct, H = 16, 8, 64
    m = synth.model(110, 256, 256, 128, 128, cs, 24, ct, H, temporal_dtype="f16")
    am = f32(oracle.fp8_calibrate(m, synth.random_queries(111, 1 << 14)))
    model = ndgi.Model.from_arrays(m)
    ndgi.ndgi_prepare_fp8(model, am)
    phys = torch.zeros((128, 3 * 128, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan([model], "fp8", 8, phys)
    plan.set_shape(1, 4, 1)
    reqs = np.zeros(3, dtype=synth.PAGE_REQ_DTYPE)
    for i, (x0, y0, t) in enumerate(((0, 0, 0.3), (96, 40, 0.71), (128, 128, 0.05))):
        reqs[i] = (0, x0, y0, 128, 128, np.float32(t), 128 * i, 0)
    dump = torch.zeros(plan.fp8_dump_size(), dtype=torch.uint8, device="cuda")
    plan.set_fp8_dump(item, dump)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    assert plan.check() == (0, 0)
    plan.set_fp8_dump(-1, None)
    words = dump.cpu().numpy().view(np.uint32)
    Q = (H + 32) // 4
    R = 8 + 2 * H + 2 * Q + 4
    rows, tail = words[:128 * R].reshape(128, R), words[128 * R:]
    A1 = rows[:, :8].copy().view(np.uint8).astype(np.int64)
    D1 = rows[:, 8:8 + H].copy().view(np.float32).astype(np.float64)
    A2 = rows[:, 8 + H:8 + H + Q].copy().view(np.uint8).astype(np.int64)
    D2 = rows[:, 8 + H + Q:8 + 2 * H + Q].copy().view(np.float32).astype(np.float64)
    A3 = rows[:, 8 + 2 * H + Q:8 + 2 * H + 2 * Q].copy().view(np.uint8).astype(np.int64)
    D3 = rows[:, 8 + 2 * H + 2 * Q:R].copy().view(np.float32).astype(np.float64)
    vt_k = tail[:ct].copy().view(np.float32).astype(np.float64)
    b1t = tail[ct:ct + H].copy().view(np.uint8).reshape(H, 4).astype(np.int64)
    sc = oracle.fp8_scales(m, am)
    wq = oracle.fp8_weights(m, am)
    rq = reqs[item]
    tt = np.arange(128)
    ix, iy = rq["x0"] + (tt % 64), rq["y0"] + tt // 64
    q = np.stack([(ix + 0.5) / 256, (iy + 0.5) / 256, np.full(128, rq["t"])], 1).astype(np.float32)
    x64, p35 = oracle.features(m, q)
    a1, inv_a1 = sc["a1"], 1.0 / sc["a1"]
    # ---- layer-1 spatial inputs: the kernel's FP16 blend, emulated ----
    fx = (q[:, 0].astype(np.float64) * 128 - 0.5) % 1.0
    fy = (q[:, 1].astype(np.float64) * 128 - 0.5) % 1.0
    f = h16(np.float32(p35.astype(np.float32) * np.float32(1.0 / 8925.0)))       # [n][4][cs] ring values
    wx0, wx1 = h16((1 - fx) * inv_a1)[:, None], h16(fx * inv_a1)[:, None]
    wy0, wy1 = h16(1 - fy)[:, None], h16(fy)[:, None]
    w = [h16(wx0 * wy0), h16(wx1 * wy0), h16(wx0 * wy1), h16(wx1 * wy1)]
    v = h16(w[0] * f[:, 0])
    for k in (1, 2, 3):
        v = h16(w[k] * f[:, k] + v)
    _, emu_codes = oracle.e4m3(v.reshape(-1))
    assert np.array_equal(A1[:, :cs], emu_codes.reshape(128, cs))
    exact = x64[:, :cs] * inv_a1
    assert np.all(np.abs(v - exact) <= 8 * 2.0 ** -11 * np.abs(exact) + 2.0 ** -24 * inv_a1)
    _, ref_codes = oracle.e4m3(exact.reshape(-1))
    ok, flips1 = adjacent_flip_ok(exact.reshape(-1), A1[:, :cs].reshape(-1), ref_codes,
                                  (8 * 2.0 ** -11 * np.abs(exact) + 2.0 ** -24 * inv_a1).reshape(-1))
    assert ok
    # ---- the request's temporal inputs (folded into b1') ----
    vt64 = x64[0, cs:]
    _, vt_ref = oracle.e4m3(vt64 * inv_a1)
    _, vt_ker = oracle.e4m3(vt_k * inv_a1)
    assert np.array_equal(code_value(vt_ker) * a1, vt_k)                         # the kernel's values are codes
    ok, flips_t = adjacent_flip_ok(vt64 * inv_a1, vt_ker, vt_ref, 4 * 2.0 ** -24 * inv_a1 * (1 + np.abs(vt64)))
    assert ok
    # ---- layer 1: accumulator vs the exact sum of the dumped codes times the stored weights ----
    v1 = code_value(A1[:, cs:cs + 3])
    assert np.all(v1 == v1[0, 0]) and np.all(A1[:, cs + 3:] == 0)
    terms1 = code_value(b1t[:, :3])                                               # [H][3]
    prod1 = code_value(A1[:, :cs])[:, :, None] * (wq["w1"][:cs] / sc["s1"])[None]
    y1 = prod1.sum(1) + v1[:, :1] * terms1.sum(1)[None]
    mag1 = np.abs(prod1).sum(1) + (abs(v1[0, 0]) * np.abs(terms1).sum(1))[None]
    acc1 = np.abs(D1 - y1) / np.maximum(mag1, 1e-30)
    # the kernel's folded bias against the unfused definition (stored b1 + stored W1_t times q(v_t)), in units a2
    b1_ker = v1[0, 0] * terms1.sum(1)
    _, vb1, b1_stored = oracle.fp8_bias(np.asarray(m["b1"], np.float64), sc["a2"])
    b1_def = (b1_stored + code_value(vt_ker) * a1 @ wq["w1"][cs:]) / sc["a2"]
    fold = np.abs(b1_ker - b1_def)
    beta = np.abs(b1_def)
    # ---- layers 2 and 3 ----
    _, A2_from_D1 = oracle.e4m3(np.maximum(D1, 0).reshape(-1))
    assert np.array_equal(A2[:, :H].reshape(-1), A2_from_D1)
    terms2, v2, _ = oracle.fp8_bias(np.asarray(m["b2"], np.float64), sc["a3"])
    assert np.all(code_value(A2[:, H:H + 3]) == v2) and np.all(A2[:, H + 3:] == 0)
    prod2 = code_value(A2[:, :H])[:, :, None] * (wq["w2"] / sc["s2"])[None]
    y2 = prod2.sum(1) + v2 * terms2.sum(1)[None]
    acc2 = np.abs(D2 - y2) / np.maximum(np.abs(prod2).sum(1) + np.abs(v2 * terms2).sum(1)[None], 1e-30)
    _, A3_from_D2 = oracle.e4m3(np.maximum(D2, 0).reshape(-1))
    assert np.array_equal(A3[:, :H].reshape(-1), A3_from_D2)
    terms3, v3, _ = oracle.fp8_bias(np.asarray(m["b3"], np.float64), sc["out"])
    assert np.all(code_value(A3[:, H:H + 3]) == v3)
    prod3 = code_value(A3[:, :H])[:, :, None] * (wq["w3"] / sc["s3"])[None]
    y3 = prod3.sum(1) + v3 * terms3.sum(1)[None]
    acc3 = np.abs(D3[:, :3] - y3) / np.maximum(np.abs(prod3).sum(1) + np.abs(v3 * terms3).sum(1)[None], 1e-30)
    # ---- the stored RGB is the layer-3 accumulator times the output scale ----
    got = phys.cpu().numpy()[iy - rq["y0"], 128 * item + (ix - rq["x0"])][:, :3].astype(np.float64)
    assert np.array_equal(got, (D3[:, :3].astype(np.float32) * np.float32(sc["out"])).astype(np.float64))
    print(f"item {item}: layer-1 input flips vs FP64 {flips1} of {128 * cs}, temporal {flips_t}; accumulation "
          f"error / sum|terms|: {acc1.max():.2e} {acc2.max():.2e} {acc3.max():.2e}; fold |b1' - def| max "
          f"{fold.max():.2e} (|b1'| max {beta.max():.2e})")
    # FP32 accumulation of at most 96 exact products (measured: 0, 0 and 3.7e-8 of sum|terms|), with margin
    assert max(acc1.max(), acc2.max(), acc3.max()) <= 2.0 ** -20
    # the fold's three E4M3 terms (residual after three terms: max(2^-12 |beta|, v1 2^-10)), the stored b1's own
    # three terms likewise (its ones value vb1), and FP32 sums
    b1a = np.abs(np.asarray(m["b1"], np.float64)) / sc["a2"]
    bound = (np.maximum(2.0 ** -12 * beta, v1[0, 0] * 2.0 ** -10) + np.maximum(2.0 ** -12 * b1a, vb1 * 2.0 ** -10)
             + 2.0 ** -20 * (1 + beta))
    assert np.all(fold <= bound)
    plan.close()
