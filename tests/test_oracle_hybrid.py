"""Pins of the oracle's hybrid-feature-map decoder (the paper's full decoder:
Sec. 3.3 Eq. 4-5, Sec. 4), each against something other than the oracle's
own formula:

- gamma(t) of Eq. 4 at times where sin and cos are known in closed form;
- GELU against the standard normal CDF's tabulated values and SciPy's ndtr,
  and its odd-part identity GELU(x) - GELU(-x) = x;
- V_uv against the simple model's spatial sampler (pinned by the BC4 tests)
  on the same BC4 planes;
- V_uvt at t-slice centres against that sampler on the slice's planes,
  linear in t between centres and clamped outside them;
- V_ut / V_vt on planes holding an affine ramp in (x, t), which bilinear
  interpolation reproduces exactly away from the clamped edges;
- the MLP's layer order, transposition and bias placement through weights
  that keep every hidden pre-activation far above zero (GELU = identity to
  FP64 precision, so the network is a plain matrix product), and its
  activation through hidden units whose pre-activation is exactly +-1;
- the page decode against the point decode at texel centres, and its
  mirrored tile border against NumPy's symmetric padding of the interior.
"""
import numpy as np
import pytest

import oracle
import synth


def small_model(seed=11, mode=0, hidden=16):
    return synth.hybrid_model(seed, 48, 40, 32, 24, 16, 12, 6, 20, 9, 28, 7, hidden, address_mode=mode)


def simple_on_planes(bc4, w, h, mode):
    """A simple model over the given four BC4 planes (its temporal part unused)."""
    m = synth.model(5, 64, 64, w, h, 4, 4, 2, 16, temporal_dtype="f32", address_mode=mode)
    m["bc4"] = np.ascontiguousarray(bc4)
    return m


def test_gamma_closed_form():
    r2, r3 = np.sqrt(0.5), np.sqrt(3.0) / 2
    cases = {0.0: [0, 1, 0, 1], 0.5: [1, 0, 0, -1], 0.25: [r2, r2, 1, 0], 1.0 / 6: [0.5, r3, r3, 0.5],
             0.75: [r2, -r2, -1, 0], 1.0: [0, -1, 0, 1]}
    for t, want in cases.items():
        assert np.allclose(oracle.hybrid_gamma(t), want, rtol=0, atol=1e-15), t


def test_gelu_normal_cdf():
    # Phi(1) = 0.841344746068543, Phi(2) = 0.977249868051821 (standard normal table)
    assert oracle.gelu(0.0) == 0.0
    assert abs(oracle.gelu(1.0) - 0.841344746068543) < 1e-15
    assert abs(oracle.gelu(-1.0) + 0.158655253931457) < 1e-15
    assert abs(oracle.gelu(2.0) - 2 * 0.977249868051821) < 1e-14
    x = np.linspace(-6, 6, 97)
    assert np.allclose(oracle.gelu(x) - oracle.gelu(-x), x, rtol=0, atol=1e-14)
    special = pytest.importorskip("scipy.special")
    assert np.allclose(oracle.gelu(x), x * special.ndtr(x), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("mode", [0, 1])
def test_uv_plane_matches_the_simple_sampler(mode):
    m = small_model(12, mode)
    q = synth.random_queries(13, 3000)
    q[:500, :2] = np.random.default_rng(14).uniform(-1.2, 2.2, (500, 2)).astype(np.float32)
    _, x = oracle.hybrid_decode_points(m, q, features=True)
    xs, _ = oracle.features(simple_on_planes(m["uv_bc4"], m["uv_w"], m["uv_h"], mode), q)
    assert np.array_equal(x[:, 4:8], xs[:, :4])


def test_volume_slices_trilinear_in_t():
    # 8 slices, so the float32 times (k + 0.5) / 8 and (k + 0.75) / 8 are exact
    m = synth.hybrid_model(15, 48, 40, 32, 24, 16, 12, 8, 20, 9, 28, 7, 16)
    vol_t, vol_h, vol_w = m["vol_shape"]
    q = synth.random_queries(16, 800)
    per_slice = []
    for k in range(vol_t):
        xs, _ = oracle.features(simple_on_planes(m["vol_bc4"][k], vol_w, vol_h, 0), q)
        per_slice.append(xs[:, :4])
    for k in range(vol_t):                                    # slice centres: that slice alone
        qk = q.copy()
        qk[:, 2] = (k + 0.5) / vol_t
        _, x = oracle.hybrid_decode_points(m, qk, features=True)
        assert np.allclose(x[:, :4], per_slice[k], rtol=0, atol=1e-15)
    for k in range(vol_t - 1):                                # a quarter of the way between centres
        qk = q.copy()
        qk[:, 2] = (k + 0.75) / vol_t
        _, x = oracle.hybrid_decode_points(m, qk, features=True)
        assert np.allclose(x[:, :4], 0.75 * per_slice[k] + 0.25 * per_slice[k + 1], rtol=0, atol=1e-12)
    for t, k in ((0.0, 0), (0.2 / vol_t, 0), (1.0, vol_t - 1), ((vol_t - 0.1) / vol_t, vol_t - 1)):
        qk = q.copy()
        qk[:, 2] = t                                          # outside the centres: clamped to the edge slice
        _, x = oracle.hybrid_decode_points(m, qk, features=True)
        assert np.allclose(x[:, :4], per_slice[k], rtol=0, atol=1e-15)


def ramp_plane(nx, nt, a, b, c):
    """Bytes a*x + b*y + c*ch + 3 of a [nt][nx][2] plane."""
    y, x, ch = np.meshgrid(np.arange(nt), np.arange(nx), np.arange(2), indexing="ij")
    v = a * x + b * y + c * ch + 3
    assert v.max() < 256
    return v.astype(np.uint8)


@pytest.mark.parametrize("mode", [0, 1])
def test_time_planes_reproduce_affine_ramps(mode):
    m = small_model(17, mode)
    ut_t, ut_w, _ = m["ut"].shape
    vt_t, vt_h, _ = m["vt"].shape
    m["ut"] = ramp_plane(ut_w, ut_t, 5, 9, 11)
    m["vt"] = ramp_plane(vt_h, vt_t, 3, 13, 7)
    rng = np.random.default_rng(18)
    n = 2000
    q = np.empty((n, 3), np.float32)
    # interior of every axis: between the first and last texel centres
    q[:, 0] = rng.uniform(0.5 / ut_w, (ut_w - 0.5) / ut_w, n)
    q[:, 1] = rng.uniform(0.5 / vt_h, (vt_h - 0.5) / vt_h, n)
    q[:, 2] = rng.uniform(0.5 / min(ut_t, vt_t), 1 - 0.5 / min(ut_t, vt_t), n)
    _, x = oracle.hybrid_decode_points(m, q, features=True)
    u, v, t = (q[:, k].astype(np.float64) for k in range(3))
    xu, tu = u * ut_w - 0.5, t * ut_t - 0.5
    xv, tv = v * vt_h - 0.5, t * vt_t - 0.5
    for ch in range(2):
        assert np.allclose(x[:, 8 + ch], (5 * xu + 9 * tu + 11 * ch + 3) / 255, rtol=0, atol=1e-12)
        assert np.allclose(x[:, 10 + ch], (3 * xv + 13 * tv + 7 * ch + 3) / 255, rtol=0, atol=1e-12)
    # clamped corners: below the first centres every term is the edge texel
    q2 = np.array([[0.1 / ut_w, 0.1 / vt_h, 0.0]], np.float32)
    _, x2 = oracle.hybrid_decode_points(m, q2, features=True)
    if mode == 0:
        assert np.allclose(x2[0, 8:12], np.array([3, 14, 3, 10]) / 255, rtol=0, atol=1e-15)


def test_gamma_is_the_last_four_inputs():
    m = small_model(19)
    q = synth.random_queries(20, 50)
    _, x = oracle.hybrid_decode_points(m, q, features=True)
    for i in range(50):
        assert np.allclose(x[i, 12:], oracle.hybrid_gamma(float(q[i, 2])), rtol=0, atol=1e-15)


def test_mlp_layers_through_the_linear_regime():
    # pre-activations >= 20: GELU(z) = z Phi(z) = z to FP64 precision, so the
    # network is x W1 + b1 -> (.) W2 + b2 -> (.) W3 + b3 as plain matrix products
    H = 16
    m = small_model(21, hidden=H)
    rng = np.random.default_rng(22)
    m["w1"] = rng.uniform(0, 1, (16, H)).astype(np.float32)
    m["b1"] = np.full(H, 20.0, np.float32)
    m["w2"] = rng.uniform(0, 0.5, (H, H)).astype(np.float32)
    m["b2"] = np.full(H, 20.0, np.float32)
    m["w3"] = rng.uniform(-1, 1, (H, 3)).astype(np.float32)
    m["b3"] = rng.uniform(-1, 1, 3).astype(np.float32)
    q = synth.random_queries(23, 300)
    y, x = oracle.hybrid_decode_points(m, q, features=True)
    w = {k: m[k].astype(np.float64) for k in ("w1", "b1", "w2", "b2", "w3", "b3")}
    h1 = x @ w["w1"] + w["b1"]
    assert h1.min() > 10
    h2 = h1 @ w["w2"] + w["b2"]
    want = h2 @ w["w3"] + w["b3"]
    assert np.allclose(y, want, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("z,phi", [(1.0, 0.841344746068543), (-1.0, 0.158655253931457)])
def test_mlp_activation_at_unit_preactivation(z, phi):
    # W1 = W2 = 0: every hidden unit of layer 1 sees b1 = z, of layer 2 b2 = z
    H = 16
    m = small_model(24, hidden=H)
    m["w1"] = np.zeros((16, H), np.float32)
    m["b1"] = np.full(H, z, np.float32)
    m["w2"] = np.zeros((H, H), np.float32)
    m["b2"] = np.full(H, z, np.float32)
    m["w3"] = np.random.default_rng(25).uniform(-1, 1, (H, 3)).astype(np.float32)
    m["b3"] = np.float32([0.5, -0.25, 0.125])
    y = oracle.hybrid_decode_points(m, synth.random_queries(26, 4))
    want = m["b3"].astype(np.float64) + z * phi * m["w3"].astype(np.float64).sum(axis=0)
    assert np.allclose(y, want[None, :], rtol=0, atol=1e-14)


def test_pages_equal_points_at_texel_centres():
    # power-of-two lightmaps, so the float32 texel-centre queries are exact
    models = [synth.hybrid_model(27, 64, 32, 32, 24, 16, 12, 6, 20, 9, 28, 7, 16),
              synth.hybrid_model(28, 64, 32, 64, 32, 8, 8, 4, 16, 5, 8, 5, 32, 1)]
    spec = [(0, 0, 0, 7, 3, 0.0), (0, 64 - 5, 32 - 9, 5, 9, 0.999), (1, 0, 32 - 16, 16, 16, 0.5),
            (1, 64 - 33, 0, 33, 2, 0.123), (1, 40, 10, 1, 1, 0.75)]
    reqs = np.zeros(len(spec), dtype=synth.PAGE_REQ_DTYPE)
    dx = 0
    for i, (mi, x0, y0, w, h, t) in enumerate(spec):
        reqs[i] = (mi, x0, y0, w, h, np.float32(t), dx + 1, 2 + i % 2)
        dx += w + 2
    phys_w, phys_h = dx + 2, 20
    got = oracle.hybrid_decode_pages(models, reqs, phys_w, phys_h)
    covered = np.zeros((phys_h, phys_w), bool)
    for r in reqs:
        m = models[r["model"]]
        jj, ii = np.meshgrid(np.arange(r["h"]), np.arange(r["w"]), indexing="ij")
        u = ((r["x0"] + ii + 0.5) / m["lm_w"]).astype(np.float32)
        v = ((r["y0"] + jj + 0.5) / m["lm_h"]).astype(np.float32)
        q = np.stack([u.ravel(), v.ravel(), np.full(u.size, r["t"], np.float32)], 1)
        want = oracle.hybrid_decode_points(m, q).reshape(r["h"], r["w"], 3)
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        assert np.array_equal(got[sl][..., :3], want)
        assert np.all(got[sl][..., 3] == 1.0)
        covered[sl] = True
    assert np.all(np.isnan(got[~covered]))


@pytest.mark.parametrize("b", [1, 4])
def test_page_border_is_symmetric_padding(b):
    models = [synth.hybrid_model(29, 64, 64, 64, 64, 16, 16, 6, 20, 9, 28, 7, 16)]
    reqs = np.zeros(2, dtype=synth.PAGE_REQ_DTYPE)
    reqs[0] = (0, 3, 7, 20, 13, np.float32(0.4), b, b)
    reqs[1] = (0, 40, 50, 24, 14, np.float32(0.8), 40 + b, b)
    W, H = 80, 24
    plain = oracle.hybrid_decode_pages(models, reqs, W, H, fill=0.0)
    padded = oracle.hybrid_decode_pages(models, reqs, W, H, fill=0.0, border=b)
    for r in reqs:
        inner = plain[r["dst_y"]:r["dst_y"] + r["h"], r["dst_x"]:r["dst_x"] + r["w"]]
        want = np.pad(inner, ((b, b), (b, b), (0, 0)), mode="symmetric")
        got = padded[r["dst_y"] - b:r["dst_y"] + r["h"] + b, r["dst_x"] - b:r["dst_x"] + r["w"] + b]
        assert np.array_equal(got, want)
