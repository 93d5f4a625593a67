"""Pins of the oracle's hybrid-decoder fit (Sec. 3.4's BC simulation, Eq. 6-7,
applied to the decoder of Sec. 3.3):

- the straight-through forward equals the pinned hybrid decode of the same
  model with F_uv and every F3D slice packed to BC4 (decode of pack = the
  forward), on F_ut / F_vt values that UNORM8 stores exactly;
- the analytic gradient matches FP64 central finite differences of the
  continuous relaxation (GELU is smooth, so no kink handling), norm-wise per
  tensor and elementwise with a 1e-6 floor.
"""
import numpy as np
import pytest

import oracle
import synth

KEYS = oracle.HFIT_KEYS


def problem(seed=0, hidden=16):
    p = synth.hybrid_fit_init(seed, 32, 32, 32, 32, 8, 8, 6, 16, 5, 16, 5, hidden)
    rng = np.random.default_rng(seed + 1)
    q = synth.random_queries(seed + 2, 300)
    q[:10, :2] = rng.uniform(-0.3, 1.3, (10, 2)).astype(np.float32)
    tgt = rng.normal(size=(300, 3))
    return p, q, tgt


def test_forward_equals_decode_of_packed_model():
    p, q, _ = problem(1)
    p["ut"] = (np.round(p["ut"] * 255) / 255).astype(np.float32)
    p["vt"] = (np.round(p["vt"] * 255) / 255).astype(np.float32)
    vt_, vh, vw = p["vol_shape"]
    m = dict(kind="hybrid", lm_w=32, lm_h=32, uv_w=32, uv_h=32, vol_shape=p["vol_shape"], hidden=p["hidden"],
             address_mode=0,
             uv_bc4=oracle.bc_pack(p["uv_ea"], p["uv_eb"], p["uv_wt"]),
             vol_bc4=np.stack([oracle.bc_pack(p["vol_ea"][k], p["vol_eb"][k], p["vol_wt"][k]) for k in range(vt_)]),
             ut=np.round(p["ut"] * 255).astype(np.uint8), vt=np.round(p["vt"] * 255).astype(np.uint8),
             **{k: p[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")})
    y_fit = oracle.hfit_forward(p, q)
    y_dec = oracle.hybrid_decode_points(m, q)
    # equal up to the FP32 storage of the 8-bit values k/255 in the fit (a few 1e-8)
    assert np.allclose(y_fit, y_dec, rtol=0, atol=1e-6)
    assert not np.allclose(y_fit, oracle.hfit_forward(p, q, relaxed=True), atol=1e-6)   # the quantisers act


def test_backward_matches_finite_differences_relaxed():
    p, q, tgt = problem(3)
    loss, g = oracle.hfit_backward(p, q, tgt, relaxed=True)
    rng = np.random.default_rng(4)
    h = 1e-3

    def loss_at(k, i, val):
        pp = dict(p)
        arr = p[k].copy().reshape(-1)
        arr[i] = val
        pp[k] = arr.reshape(p[k].shape)
        return np.mean((oracle.hfit_forward(pp, q, relaxed=True) - tgt) ** 2), float(arr[i])

    for k in KEYS:
        flat = p[k].reshape(-1)
        idx = rng.choice(flat.size, min(flat.size, 12), replace=False)
        fd = np.zeros(idx.size)
        for j, i in enumerate(idx):
            lp, vp = loss_at(k, i, np.float32(float(flat[i]) + h))
            lm, vm = loss_at(k, i, np.float32(float(flat[i]) - h))
            fd[j] = (lp - lm) / (vp - vm)                       # the realised FP32 step
        an = g[k].reshape(-1)[idx]
        assert np.linalg.norm(an - fd) <= 2e-3 * max(np.linalg.norm(an), 1e-9), k
        assert np.all(np.abs(an - fd) <= 2e-3 * np.abs(an) + 1e-6), k


# --------------------------------------------------------------------------
# Eq. 7 with one weight per texel shared by the channels (the BC7 simulation)
# --------------------------------------------------------------------------

def shared_problem(seed=0, hidden=16):
    p = synth.hybrid_fit_init(seed, 32, 32, 32, 32, 8, 8, 6, 16, 5, 16, 5, hidden, shared_w=True)
    rng = np.random.default_rng(seed + 1)
    q = synth.random_queries(seed + 2, 300)
    q[:10, :2] = rng.uniform(-0.3, 1.3, (10, 2)).astype(np.float32)
    return p, q, rng.normal(size=(300, 3))


def mode6_blocks(ea, eb, w):
    """BC7 mode-6 blocks [..][16] of 8-bit even endpoints 255 ea, 255 eb (codes / 2, p-bits 0) and 4-bit
    indices 15 w, written field by field (the anchor texel's index kept below 8 by swapping the endpoints)."""
    from test_oracle_bc7 import write_block
    lead = ea.shape[:-1]
    out = np.zeros(lead + (16,), np.uint8)
    for i in np.ndindex(*lead):
        A = np.rint(ea[i] * 255).astype(int)
        B = np.rint(eb[i] * 255).astype(int)
        k = np.rint(w[i] * 15).astype(int)
        if k[0] >= 8:
            A, B, k = B, A, 15 - k
        out[i] = write_block(6, 0, 0, 0, [[[int(v) for v in A // 2], [int(v) for v in B // 2]]], [[0, 0]],
                             [int(v) for v in k], [0] * 16)
    return out


def test_shared_weight_forward_equals_bc7_decode():
    p, q, _ = shared_problem(5)
    rng = np.random.default_rng(6)
    for key in ("uv", "vol"):
        ea, eb, w = p[f"{key}_ea"], p[f"{key}_eb"], p[f"{key}_wt"]
        p[f"{key}_ea"] = (2 * rng.integers(0, 128, ea.shape) / 255).astype(np.float32)
        p[f"{key}_eb"] = (2 * rng.integers(0, 128, eb.shape) / 255).astype(np.float32)
        p[f"{key}_wt"] = (rng.integers(0, 16, w.shape) / 15).astype(np.float32)
    p["ut"] = (np.round(p["ut"] * 255) / 255).astype(np.float32)
    p["vt"] = (np.round(p["vt"] * 255) / 255).astype(np.float32)
    m = dict(kind="hybrid", lm_w=32, lm_h=32, uv_w=32, uv_h=32, vol_shape=p["vol_shape"], hidden=p["hidden"],
             address_mode=0, feat_format=1,
             uv_bc7=mode6_blocks(p["uv_ea"], p["uv_eb"], p["uv_wt"]),
             vol_bc7=mode6_blocks(p["vol_ea"], p["vol_eb"], p["vol_wt"]),
             ut=np.round(p["ut"] * 255).astype(np.uint8), vt=np.round(p["vt"] * 255).astype(np.uint8),
             **{k: p[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")})
    y_fit = oracle.hfit_forward(p, q)
    y_dec = oracle.hybrid_decode_points(m, q)
    assert np.allclose(y_fit, y_dec, rtol=0, atol=1e-6)
    assert not np.allclose(y_fit, oracle.hfit_forward(p, q, relaxed=True), atol=1e-6)


def test_shared_weight_backward_matches_finite_differences():
    p, q, tgt = shared_problem(7)
    loss, g = oracle.hfit_backward(p, q, tgt, relaxed=True)
    rng = np.random.default_rng(8)
    h = 1e-3
    for k in ("uv_ea", "uv_eb", "uv_wt", "vol_ea", "vol_eb", "vol_wt", "w1"):
        flat = p[k].reshape(-1)
        assert g[k].shape == p[k].shape
        idx = rng.choice(flat.size, 12, replace=False)
        fd = np.zeros(idx.size)
        for j, i in enumerate(idx):
            vals = []
            for s in (+1, -1):
                pp = dict(p)
                arr = flat.copy()
                arr[i] = np.float32(float(flat[i]) + s * h)
                pp[k] = arr.reshape(p[k].shape)
                vals.append((np.mean((oracle.hfit_forward(pp, q, relaxed=True) - tgt) ** 2), float(arr[i])))
            fd[j] = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        an = g[k].reshape(-1)[idx]
        assert np.linalg.norm(an - fd) <= 2e-3 * max(np.linalg.norm(an), 1e-9), k
        assert np.all(np.abs(an - fd) <= 2e-3 * np.abs(an) + 1e-6), k


# --------------------------------------------------------------------------
# Training-time quantisation noise on the sampled vectors (Sec. 3.4)
# --------------------------------------------------------------------------

def test_noise_draws_are_uniform_and_deterministic():
    a = 1.0 / 256
    nz = oracle.fit_noise(5, 3, 20_000, a)
    assert nz.shape == (20_000, 12)
    assert np.all(nz >= -a / 2) and np.all(nz < a / 2)
    assert np.array_equal(nz, oracle.fit_noise(5, 3, 20_000, a))
    assert np.array_equal(nz[100:200], oracle.fit_noise(5, 3, 100, a, first=100))
    assert not np.array_equal(nz, oracle.fit_noise(5, 4, 20_000, a))
    stats = pytest.importorskip("scipy.stats")
    for k in (0, 5, 11):
        assert stats.kstest(nz[:, k] / a + 0.5, "uniform").pvalue > 1e-3
    assert abs(np.corrcoef(nz[:, 0], nz[:, 1])[0, 1]) < 0.05


def test_noise_is_an_additive_input_shift():
    """A constant noise c on input k is a shift of the first layer's bias by c W1[k] (a linear layer)."""
    p, q, tgt = problem(9)
    c, k = 0.01, 5
    nz = np.zeros((q.shape[0], 12))
    nz[:, k] = c
    pb = dict(p)
    pb["b1"] = (p["b1"].astype(np.float64) + c * p["w1"][k].astype(np.float64)).astype(np.float32)
    y_n = oracle.hfit_forward(p, q, noise=nz)
    assert np.allclose(y_n, oracle.hfit_forward(pb, q), rtol=0, atol=1e-6)   # b1 stored in FP32
    assert not np.allclose(y_n, oracle.hfit_forward(p, q), atol=1e-6)
    # the gradient with a random noise array matches finite differences of the same noisy loss
    nz = oracle.fit_noise(2, 0, q.shape[0], 1.0 / 256)
    _, g = oracle.hfit_backward(p, q, tgt, relaxed=True, noise=nz)
    flat = p["uv_ea"].reshape(-1)
    for i in (0, 7, 33):
        vals = []
        for s in (+1, -1):
            arr = flat.copy()
            arr[i] = np.float32(float(flat[i]) + s * 1e-3)
            pp = dict(p, uv_ea=arr.reshape(p["uv_ea"].shape))
            vals.append((np.mean((oracle.hfit_forward(pp, q, relaxed=True, noise=nz) - tgt) ** 2), float(arr[i])))
        fd = (vals[0][0] - vals[1][0]) / (vals[0][1] - vals[1][1])
        assert abs(g["uv_ea"].reshape(-1)[i] - fd) <= 2e-3 * abs(fd) + 1e-6


def test_shared_weight_maps_are_exact_mode6_blocks():
    """The shared-weight simulation's texels are exactly the BC7 decode of its mode-6 pack, on random
    parameters, and the fit's forward equals the hybrid decode of the packed model."""
    p, q, _ = shared_problem(11)
    for key in ("uv", "vol"):
        ea, eb, w = p[f"{key}_ea"], p[f"{key}_eb"], p[f"{key}_wt"]
        blocks = oracle.bc7_pack_sim(ea, eb, w)
        assert blocks.shape == ea.shape[:-1] + (16,)
        assert np.all((blocks[..., 0] & 0x7F) == 64)                     # mode 6 everywhere
        bh, bw = ea.shape[-3], ea.shape[-2]
        dec = oracle.bc7_decode(blocks.reshape(-1, bw, 16), 4 * bw, blocks.size // (16 * bw) * 4)
        assert np.array_equal(dec, oracle.bc_sim7_rgba8(ea, eb, w))
    p["ut"] = (np.round(p["ut"] * 255) / 255).astype(np.float32)
    p["vt"] = (np.round(p["vt"] * 255) / 255).astype(np.float32)
    m = dict(kind="hybrid", lm_w=32, lm_h=32, uv_w=32, uv_h=32, vol_shape=p["vol_shape"], hidden=p["hidden"],
             address_mode=0, feat_format=1,
             uv_bc7=oracle.bc7_pack_sim(p["uv_ea"], p["uv_eb"], p["uv_wt"]),
             vol_bc7=oracle.bc7_pack_sim(p["vol_ea"], p["vol_eb"], p["vol_wt"]),
             ut=np.round(p["ut"] * 255).astype(np.uint8), vt=np.round(p["vt"] * 255).astype(np.uint8),
             **{k: p[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")})
    assert np.allclose(oracle.hfit_forward(p, q), oracle.hybrid_decode_points(m, q), rtol=0, atol=1e-6)


def test_mode6_endpoint_parity_rule():
    """An endpoint keeps the 8-bit values of its majority parity exactly and moves the others by one level."""
    p, _, _ = shared_problem(12)
    ea = p["uv_ea"][:1, :1].copy()
    ea[0, 0] = np.float32([10, 12, 14, 15]) / 255              # three even: p = 0, the odd 15 -> 14
    eb = p["uv_eb"][:1, :1].copy()
    eb[0, 0] = np.float32([11, 13, 200, 0]) / 255              # 2-2 tie: p = 0; 11 -> 10, 13 -> 12
    w = np.zeros((1, 1, 16), np.float32)
    w[0, 0, 1] = 1.0                                           # texel 1 at index 15 (endpoint 1)
    rgba = oracle.bc_sim7_rgba8(ea, eb, w)
    assert list(rgba[0, 0]) == [10, 12, 14, 14]
    assert list(rgba[0, 1]) == [10, 12, 200, 0]
