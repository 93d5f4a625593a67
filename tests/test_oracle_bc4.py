"""Pins for the oracle's BC4 decode, bilinear gather and temporal lerp.

Each check is fixed by something other than the oracle's own code: the BC4
palette closed forms of the format definition (endpoint pair plus 6 or 4
interpolants, Eq. 7 / supplement S2 with w on a 1/7 or 1/5 grid), single-bit
index probes for the bit layout, exact linear reproduction by the bilinear
filter, partition of unity, and keyframe rows of the temporal line.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle


def block(r0, r1, idx):
    """BC4 block bytes from endpoints and 16 3-bit indices (texel p at bit 3p of the index field)."""
    bits = 0
    for p, k in enumerate(idx):
        bits |= (k & 7) << (3 * p)
    return bytes([r0, r1]) + bits.to_bytes(6, "little")


def test_eight_value_mode_closed_form():
    # r0 > r1: the palette is r0, r1 and six interpolants (8-k)/7 r0 + (k-1)/7 r1, k = 2..7.
    for (r0, r1) in [(255, 0), (200, 17), (1, 0), (254, 253)]:
        for k in range(8):
            b = block(r0, r1, [k] * 16)
            got = Fraction(oracle.bc4_p35(b, 5), 8925)
            if k == 0:
                want = Fraction(r0, 255)
            elif k == 1:
                want = Fraction(r1, 255)
            else:
                want = (Fraction(8 - k, 7) * r0 + Fraction(k - 1, 7) * r1) / 255
            assert got == want, (r0, r1, k)


def test_eight_value_mode_255_0():
    # (r0, r1) = (255, 0) with index k >= 2 gives P35 = 5*255*(8-k).
    for k in range(2, 8):
        assert oracle.bc4_p35(block(255, 0, [k] * 16), 0) == 5 * 255 * (8 - k)


def test_six_value_mode_closed_form_and_literals():
    # r0 <= r1: r0, r1, four interpolants (6-k)/5 r0 + (k-1)/5 r1, then 0 and 1.
    for (r0, r1) in [(0, 255), (17, 200), (100, 101)]:
        for k in range(8):
            got = Fraction(oracle.bc4_p35(block(r0, r1, [k] * 16), 9), 8925)
            if k == 0:
                want = Fraction(r0, 255)
            elif k == 1:
                want = Fraction(r1, 255)
            elif k <= 5:
                want = (Fraction(6 - k, 5) * r0 + Fraction(k - 1, 5) * r1) / 255
            elif k == 6:
                want = Fraction(0)
            else:
                want = Fraction(1)
            assert got == want, (r0, r1, k)
    assert oracle.bc4_p35(block(0, 255, [6] * 16), 3) == 0
    assert oracle.bc4_p35(block(0, 255, [7] * 16), 3) == 8925


def test_equal_endpoints():
    # r0 == r1 is six-value mode: every interpolant equals the endpoint; 6, 7 stay literals.
    for a in (0, 77, 255):
        for k in range(6):
            assert oracle.bc4_p35(block(a, a, [k] * 16), 0) == 35 * a
        assert oracle.bc4_p35(block(a, a, [6] * 16), 0) == 0
        assert oracle.bc4_p35(block(a, a, [7] * 16), 0) == 8925


def test_palette_is_eq7_interpolation():
    # Eq. 7: f_p = (1 - w_p) e1 + w_p e2 with e1 = r0/255, e2 = r1/255 and w on the 1/7 grid
    # (eight-value mode): index order 0, 2, 3, 4, 5, 6, 7, 1 has w = 0, 1/7, ..., 1.
    r0, r1 = 230, 12
    order = [0, 2, 3, 4, 5, 6, 7, 1]
    for step, k in enumerate(order):
        w = Fraction(step, 7)
        want = (1 - w) * Fraction(r0, 255) + w * Fraction(r1, 255)
        assert Fraction(oracle.bc4_p35(block(r0, r1, [k] * 16), 0), 8925) == want


def test_single_bit_index_probes():
    # Index bit layout: texel p = 4*row + col owns bits 16+3p .. 18+3p of the 64-bit block.
    for p in range(16):
        for bit in range(3):
            raw = bytearray(8)
            raw[0], raw[1] = 255, 0
            pos = 16 + 3 * p + bit
            raw[pos // 8] |= 1 << (pos % 8)
            for q in range(16):
                got = oracle.bc4_p35(bytes(raw), q)
                want_k = (1 << bit) if q == p else 0
                assert got == oracle.bc4_p35(block(255, 0, [want_k] * 16), 0), (p, bit, q)


def test_value_is_single_fp32_rounding():
    inv = np.float32(1.0) / np.float32(8925.0)
    for p35 in [0, 1, 35, 4462, 8924, 8925, 1234, 5 * 255 * 3]:
        want = np.float32(np.float32(p35) * inv)
        assert oracle.p35_value(p35) == float(want)
        assert abs(float(want) - p35 / 8925) <= 2 ** -24


def _model(feat_w, feat_h, cs, bc4, temporal, lm=None, mode=0):
    lm = lm or (feat_w, feat_h)
    H = 4
    z = np.zeros
    return dict(lm_w=lm[0], lm_h=lm[1], feat_w=feat_w, feat_h=feat_h, cs=cs, t_count=temporal.shape[0],
                ct=temporal.shape[1], hidden=H, bc4=bc4, temporal=temporal, address_mode=mode,
                w1=z((cs + temporal.shape[1], H), np.float32), b1=z(H, np.float32), w2=z((H, H), np.float32),
                b2=z(H, np.float32), w3=z((H, 3), np.float32), b3=z(3, np.float32))


def test_partition_of_unity_constant_planes():
    # Constant planes (r0 == r1 == a, all indices 0) give v_s = a/255 for any (u, v).
    cs = 3
    bc4 = np.zeros((4, 4, cs, 8), np.uint8)
    vals = [0, 128, 255]
    for c in range(cs):
        bc4[:, :, c, 0] = vals[c]
        bc4[:, :, c, 1] = vals[c]
    m = _model(16, 16, cs, bc4, np.zeros((2, 1), np.float32))
    q = np.random.default_rng(0).random((500, 3), dtype=np.float32)
    x, _ = oracle.features(m, q)
    for c in range(cs):
        assert np.all(np.abs(x[:, c] - vals[c] / 255) <= 1e-7)


def test_bilinear_reproduces_linear_ramp():
    # An 8-texel ramp f(ix) = (7 - ix)/7 along x (blocks (255,0) with indices giving
    # 7/7..4/7 and 3/7..0/7) is reproduced exactly by the bilinear filter at every
    # interior sample point x = u*8 - 0.5 in [0, 7].
    order = [0, 2, 3, 4, 5, 6, 7, 1]      # index whose value is (7 - step)/7
    bc4 = np.zeros((1, 2, 1, 8), np.uint8)
    for bx in range(2):
        idx = [order[4 * bx + (p % 4)] for p in range(16)]
        bc4[0, bx, 0] = np.frombuffer(block(255, 0, idx), np.uint8)
    m = _model(8, 4, 1, bc4, np.zeros((1, 1), np.float32))
    u = np.linspace(0.5 / 8, 7.5 / 8, 97).astype(np.float32)
    q = np.stack([u, np.full_like(u, 0.3), np.zeros_like(u)], 1)
    x, _ = oracle.features(m, q)
    xs = u.astype(np.float64) * 8 - 0.5
    want = (7 - xs) / 7
    assert np.max(np.abs(x[:, 0] - want)) < 1e-7


def test_texel_centre_returns_texel():
    rng = np.random.default_rng(3)
    bc4 = rng.integers(0, 256, (4, 4, 2, 8), dtype=np.uint8)
    m = _model(16, 16, 2, bc4, np.zeros((1, 1), np.float32))
    ix, iy = np.meshgrid(np.arange(16), np.arange(16))
    u = ((ix.ravel() + 0.5) / 16).astype(np.float32)
    v = ((iy.ravel() + 0.5) / 16).astype(np.float32)
    q = np.stack([u, v, np.zeros_like(u)], 1)
    x, p35 = oracle.features(m, q)
    for n in range(q.shape[0]):
        tx, ty = ix.ravel()[n], iy.ravel()[n]
        for c in range(2):
            blk = bytes(bc4[ty // 4, tx // 4, c])
            want = oracle.p35_value(oracle.bc4_p35(blk, (ty % 4) * 4 + tx % 4))
            assert x[n, c] == want
            assert p35[n, 0, c] == oracle.bc4_p35(blk, (ty % 4) * 4 + tx % 4)


def test_edge_clamp_and_mirror():
    rng = np.random.default_rng(4)
    bc4 = rng.integers(0, 256, (2, 2, 1, 8), dtype=np.uint8)
    # Inside [0,1) clamp and mirrored repeat agree (taps -1 and W map to 0 and W-1).
    q = rng.random((300, 3), dtype=np.float32)
    a, _ = oracle.features(_model(8, 8, 1, bc4, np.zeros((1, 1), np.float32), mode=0), q)
    b, _ = oracle.features(_model(8, 8, 1, bc4, np.zeros((1, 1), np.float32), mode=1), q)
    assert np.array_equal(a, b)
    # Outside [0,1): clamp holds the edge texel, mirror reflects: u and -u give the same sample.
    qo = q.copy()
    qo[:, 0] = -q[:, 0]
    mm = _model(8, 8, 1, bc4, np.zeros((1, 1), np.float32), mode=1)
    ra, _ = oracle.features(mm, q)
    rb, _ = oracle.features(mm, qo)
    assert np.max(np.abs(ra - rb)) < 1e-12
    qc = q.copy()
    qc[:, 0] = 1.5
    qe = q.copy()
    qe[:, 0] = 0.99999
    mc = _model(8, 8, 1, bc4, np.zeros((1, 1), np.float32), mode=0)
    assert np.array_equal(oracle.features(mc, qc)[1][:, 0], oracle.features(mc, qe)[1][:, 1])


def test_keyframes_and_periodic_lerp():
    rng = np.random.default_rng(5)
    T, ct = 8, 5
    K = rng.normal(size=(T, ct)).astype(np.float32)
    m = _model(4, 4, 1, np.zeros((1, 1, 1, 8), np.uint8), K)
    # t = j/T with T a power of two: v_t equals keyframe row j exactly.
    q = np.zeros((T, 3), np.float32)
    q[:, 2] = np.arange(T, dtype=np.float32) / T
    x, _ = oracle.features(m, q)
    assert np.array_equal(x[:, 1:], K.astype(np.float64))
    # Midpoints are the average of neighbouring rows; the last segment wraps to row 0.
    q[:, 2] = (np.arange(T, dtype=np.float32) + 0.5) / T
    x, _ = oracle.features(m, q)
    want = 0.5 * (K.astype(np.float64) + np.roll(K, -1, axis=0).astype(np.float64))
    assert np.max(np.abs(x[:, 1:] - want)) < 1e-15
    # Periodic in t: t and t + 1 and t - 1 agree (t on a 2^-10 grid so t +- 1 is exact).
    tq = (rng.integers(0, 1024, 50) / 1024).astype(np.float32)
    for shift in (1.0, -1.0):
        a = np.zeros((50, 3), np.float32)
        a[:, 2] = tq
        b = a.copy()
        b[:, 2] = tq + np.float32(shift)
        xa, _ = oracle.features(m, a)
        xb, _ = oracle.features(m, b)
        assert np.array_equal(xa, xb)


def test_temporal_lerp_non_power_of_two_within_bound():
    rng = np.random.default_rng(6)
    T, ct = 24, 3
    K = rng.normal(size=(T, ct)).astype(np.float32)
    m = _model(4, 4, 1, np.zeros((1, 1, 1, 8), np.uint8), K)
    q = np.zeros((T, 3), np.float32)
    q[:, 2] = (np.arange(T) / T).astype(np.float32)
    x, _ = oracle.features(m, q)
    # fl32(j/24) differs from j/24 by at most half an ulp; |dv_t| <= ulp * 24 * |dK|.
    bound = 2 ** -24 * 24 * np.max(np.abs(np.diff(np.vstack([K, K[:1]]), axis=0)))
    assert np.max(np.abs(x[:, 1:] - K)) <= bound + 1e-15
