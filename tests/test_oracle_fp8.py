"""Pins of the oracle's FP8 (E4M3) decode: the format, the rounding, the scale
reading and a model on which FP8 quantisation is exact.

E4M3 is fixed by its definition (1 sign, 4 exponent bits with bias 7,
3 mantissa bits, no infinities, largest finite 448, code S.1111.111 = NaN);
the table below is written from that definition, and torch's own
float8_e4m3fn conversion is an independent implementation of the same
rounding (nearest, ties to even) for magnitudes below 448.
"""
import numpy as np
import pytest

import oracle
import synth
from _models import fp8_exact_model as exact_model


def e4m3_table():
    """(code, value) of every finite E4M3 code, from the format definition."""
    out = []
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue   # NaN
        mag = (m / 8.0) * 2.0 ** -6 if e == 0 else (1.0 + m / 8.0) * 2.0 ** (e - 7)
        out.append((code, -mag if s else mag))
    return out


def test_every_code_is_a_fixed_point_with_its_code():
    table = e4m3_table()
    assert len(table) == 254
    vals = np.array([v for _, v in table])
    y, codes = oracle.e4m3(vals)
    assert np.array_equal(y, vals)
    assert [c for c, _ in table] == codes.tolist()
    assert max(vals) == 448.0 and min(v for v in vals if v > 0) == 2.0 ** -9


def test_ties_to_even_and_nearest():
    mags = sorted({abs(v) for _, v in e4m3_table()})
    codes = {abs(v): c & 0x7F for c, v in e4m3_table()}
    for lo, hi in zip(mags[:-1], mags[1:]):
        mid = 0.5 * (lo + hi)
        want = lo if codes[lo] % 2 == 0 else hi
        got, _ = oracle.e4m3([mid, -mid, np.nextafter(mid, 0), np.nextafter(mid, 1e9)])
        assert got[0] == want and got[1] == -want
        assert got[2] == lo and got[3] == hi


def test_saturation_and_subnormals():
    y, c = oracle.e4m3([448.0, 449.0, 464.0, 500.0, 1e30, -1e30, 2.0 ** -10, 3 * 2.0 ** -10, 2.0 ** -9,
                        2.0 ** -6, 2.0 ** -6 * 15 / 16])
    assert y.tolist() == [448.0, 448.0, 448.0, 448.0, 448.0, -448.0, 0.0, 2.0 ** -8, 2.0 ** -9, 2.0 ** -6,
                          2.0 ** -6]
    assert c[0] == 0x7E and c[5] == 0xFE and c[7] == 2 and c[8] == 1 and c[9] == 8


def test_matches_torch_float8_below_448():
    torch = pytest.importorskip("torch")
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("torch without float8")
    rng = np.random.default_rng(3)
    x = (rng.choice([-1, 1], 200_000) * np.exp2(rng.uniform(-12, 8.8, 200_000))).astype(np.float32)
    x = x[np.abs(x) < 448]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got, _ = oracle.e4m3(x.astype(np.float64))
    assert np.array_equal(got, ref)


def test_p2_is_the_smallest_power_of_two():
    rng = np.random.default_rng(4)
    for y in np.concatenate([np.exp2(rng.uniform(-30, 30, 2000)), 448.0 * np.exp2(np.arange(-20, 20))]):
        P = oracle.p2(y)
        assert np.log2(P) == round(np.log2(P))
        assert y <= 448.0 * P and y > 448.0 * P / 2


def test_scale_chain_and_bounds():
    m = synth.model(7, 128, 128, 64, 64, 16, 8, 8, 64, temporal_dtype="f32")
    q = synth.random_queries(8, 4096)
    am = oracle.fp8_calibrate(m, q)
    sc = oracle.fp8_scales(m, am)
    assert sc["a2"] == sc["a1"] * sc["s1"] and sc["a3"] == sc["a2"] * sc["s2"] and sc["out"] == sc["a3"] * sc["s3"]
    assert am[0] <= 448 * sc["a1"] < 2 * am[0] * (1 + 1e-12)
    for layer, (s, a_in, m_next) in enumerate(((sc["s1"], sc["a1"], am[1]), (sc["s2"], sc["a2"], am[2])), 1):
        wmax = np.abs(np.asarray(m[f"w{layer}"], np.float64)).max()
        assert wmax <= 448 * s and m_next / a_in <= 448 * s
        assert max(wmax, m_next / a_in) > 224 * s           # smallest such power of two
    assert np.abs(np.asarray(m["w3"], np.float64)).max() <= 448 * sc["s3"]
    wq = oracle.fp8_weights(m, am)
    for k, s in (("w1", sc["s1"]), ("w2", sc["s2"]), ("w3", sc["s3"])):
        ratio = wq[k] / s
        assert np.array_equal(oracle.e4m3(ratio)[0], ratio.reshape(-1))   # every stored weight is s * E4M3
        w = np.asarray(m[k], np.float64)
        big = np.abs(w) >= s * 2.0 ** -6                                  # normal range: 2^-4 relative
        assert np.all(np.abs(wq[k] - w)[big] <= np.abs(w)[big] * 2.0 ** -4)


def test_three_term_bias_split():
    rng = np.random.default_rng(5)
    b = rng.normal(0, 1, 500) * np.exp2(rng.uniform(-6, 6, 500))
    for u in (2.0 ** -10, 2.0 ** -4, 1.0):
        terms, v, stored = oracle.fp8_bias(b, u)
        assert np.array_equal(oracle.e4m3(terms)[0], terms.reshape(-1))   # each term is an E4M3 value
        assert v >= 1 and np.abs(b / u).max() <= 448 * v
        beta = b / u / v
        # each rounding leaves max(2^-4 |r|, 2^-10) (4 significant bits, or half the subnormal spacing
        # 2^-9), so after three terms |residual| <= max(2^-12 |beta/v|, 2^-10), in units u v
        bound = u * v * np.maximum(2.0 ** -12 * np.abs(beta), 2.0 ** -10)
        assert np.all(np.abs(stored - b) <= bound)
        assert np.abs(stored - b).max() > 0            # not trivially exact


def test_fp8_pages_exact_when_every_value_is_representable():
    m = exact_model()
    reqs = np.zeros(3, dtype=synth.PAGE_REQ_DTYPE)
    for i, (t, x0) in enumerate(((0.0, 0), (0.375, 8), (0.875, 16))):
        reqs[i] = (0, x0, 4, 16, 12, np.float32(t), 16 * i, 0)
    am = np.array([1.0, 3.5, 1.875])                     # max |x|, max relu(z1), max relu(z2)
    ref = oracle.decode_pages([m], reqs, 48, 16, precision="fp32", fill=0.0)
    got = oracle.decode_pages([m], reqs, 48, 16, precision="fp8", act_max=am[None], fill=0.0)
    assert np.array_equal(got, ref)
    sc = oracle.fp8_scales(m, am)
    assert 3.5 / sc["a2"] == 448.0                        # the 3.5 unit lands exactly on E4M3's largest value


def test_fp8_pages_error_is_quantisation_sized():
    m = synth.model(12, 256, 256, 128, 128, 16, 8, 8, 64, temporal_dtype="f32")
    am = oracle.fp8_calibrate(m, synth.random_queries(13, 1 << 14))
    reqs = synth.ragged_page_requests(14, (256,), 4, slots_x=2, slot=128)
    ref = oracle.decode_pages([m], reqs, 256, 256, precision="fp32", fill=0.0)
    got = oracle.decode_pages([m], reqs, 256, 256, precision="fp8", act_max=am[None], fill=0.0)
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = got[sl][..., :3], ref[sl][..., :3]
        rng_ = b.max() - b.min()
        mx, rms = np.abs(a - b).max() / rng_, np.sqrt(((a - b) ** 2).mean()) / rng_
        # E4M3 keeps 4 significant bits: errors of a few percent of the range (measured: rms 2-6%,
        # max 6-11% on this random model), never zero and never a gross scale error
        assert 1e-4 < rms < 0.08 and mx < 0.25
