"""Pins for the oracle's fit: analytic FP64 gradient vs central finite
differences on the continuous relaxation (norm-wise per tensor and
elementwise), vs an independent PyTorch FP64 autograd of the straight-through
forward, the split of the temporal gradient between the two keyframes around
t (Eq. 2), plus Adam and the sampler.  Samples are queries (u, v, t) with
most t between keyframes.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
from _fit_ref import tiny_problem, torch_forward  # noqa: E402


def _flat_loss(p, s, tgt, lm, relaxed):
    y, signs = oracle.fit_forward(p, s, lm, lm, relaxed=relaxed, want_signs=True)
    return oracle.fit_loss(y, tgt), signs


@pytest.mark.parametrize("seed", [0, 1])
def test_backward_matches_finite_differences_relaxed(seed):
    lm = 16
    p, s, tgt = tiny_problem(seed)
    loss, g = oracle.fit_backward(p, s, tgt, lm, lm, relaxed=True)
    base_loss, base_signs = _flat_loss(p, s, tgt, lm, True)
    assert abs(loss - base_loss) < 1e-12
    h = 1e-6
    for key in oracle.FIT_KEYS:
        arr = p[key]
        fd = np.zeros(arr.shape)
        keep = np.ones(arr.shape, bool)
        flat = arr.reshape(-1)
        for i in range(flat.size):
            # perturb in FP64 through a float32 parameter: use h on the float32 grid
            orig = flat[i]
            up, dn = np.float32(orig + h), np.float32(orig - h)
            flat[i] = up
            lu, su = _flat_loss(p, s, tgt, lm, True)
            flat[i] = dn
            ld, sd = _flat_loss(p, s, tgt, lm, True)
            flat[i] = orig
            if not (np.array_equal(su, base_signs) and np.array_equal(sd, base_signs)):
                keep.reshape(-1)[i] = False
                continue
            fd.reshape(-1)[i] = (lu - ld) / (float(up) - float(dn))
        ga = g[key]
        err = np.linalg.norm((ga - fd)[keep])
        ref = max(np.linalg.norm(fd[keep]), 1e-6)
        assert err / ref < 1e-3, (key, err, ref)
        # elementwise too, relative to each element with an absolute floor of 1e-6
        elem = np.abs(ga - fd)[keep] / np.maximum(np.abs(fd[keep]), 1e-6)
        assert elem.max() < 1e-3, (key, elem.max())
        assert keep.mean() > 0.5


def test_backward_matches_torch_autograd_ste():
    lm, T = 16, 3
    p, s, tgt = tiny_problem(3, T=T)
    y_t, t = torch_forward(p, s, lm, T)
    y_o = oracle.fit_forward(p, s, lm, lm, relaxed=False)
    assert np.max(np.abs(y_t.detach().numpy() - y_o)) < 1e-6
    loss = ((y_t - torch.tensor(tgt)) ** 2).mean()
    loss.backward()
    lo, g = oracle.fit_backward(p, s, tgt, lm, lm, relaxed=False)
    assert abs(lo - loss.item()) < 1e-6
    for k in oracle.FIT_KEYS:
        ref = t[k].grad.numpy()
        err = np.linalg.norm(g[k] - ref) / max(np.linalg.norm(ref), 1e-12)
        assert err < 1e-6, (k, err)


def test_adam_first_step_closed_form():
    # First Adam step with bias correction moves each parameter by lr * g/(|g| + eps).
    p = np.array([0.5, 0.5, 0.2], np.float32)
    g = np.array([0.3, -2.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(p, g, m, v, 1, 1e-2)
    want = np.array([0.5, 0.5, 0.2]) - 1e-2 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(p - want)) < 1e-7
    q = np.array([0.001, 0.999], np.float32)
    oracle.adam(q, np.array([1.0, -1.0]), np.zeros(2), np.zeros(2), 1, 1e-2, project=True)
    assert q[0] == 0.0 and q[1] == 1.0


def test_splitmix64_reference_output():
    # The generator's first output from state 0 is the published 0xE220A8397B1DCDAF.
    assert oracle.lib().om_splitmix64_next(0) == 0xE220A8397B1DCDAF


def test_fit_draw_ranges_and_uniformity():
    tx, s = oracle.fit_draw(123, 7, 200000, 1024, 512)
    assert tx[:, 0].min() >= 0 and tx[:, 0].max() < 1024 and tx[:, 1].max() < 512
    assert np.array_equal(s[:, 0], ((tx[:, 0] + 0.5) / 1024).astype(np.float32))
    assert np.array_equal(s[:, 1], ((tx[:, 1] + 0.5) / 512).astype(np.float32))
    t = s[:, 2].astype(np.float64)
    assert t.min() >= 0.0 and t.max() < 1.0
    assert np.array_equal(t * 2.0 ** 24, np.floor(t * 2.0 ** 24))       # 24-bit fractions
    hist = np.histogram(t, bins=24, range=(0, 1))[0] / len(t)
    assert np.max(np.abs(hist - 1 / 24)) < 0.003
    ta, a = oracle.fit_draw(123, 7, 10, 1024, 512, first=5)
    assert np.array_equal(a, s[5:15]) and np.array_equal(ta, tx[5:15])


def test_temporal_gradient_splits_between_the_two_keyframes():
    # v_t = (1 - alpha) K[j0] + alpha K[j1] (Eq. 2): at a fractional t the gradient of K lands on rows j0 and
    # j1 in the ratio (1 - alpha) : alpha; at a keyframe time t = j/T it lands on row j alone.  T = 8 keeps
    # every t*T below exact in FP32, so alpha is exactly 1/2, 3/4 or 0.
    lm, T = 16, 8
    p, s, tgt = tiny_problem(4, T=T, n=1)
    for t, rows in ((0.5625, {4: 0.5, 5: 0.5}), (0.96875, {7: 0.25, 0: 0.75}), (0.375, {3: 1.0})):
        s[0, 2] = np.float32(t)
        _, g = oracle.fit_backward(p, s, tgt, lm, lm, relaxed=True)
        gk = g["temporal"]
        total = gk.sum(axis=0)
        assert np.abs(total).max() > 0
        for j in range(T):
            assert np.allclose(gk[j], rows.get(j, 0.0) * total, rtol=1e-12, atol=0.0), (t, j)


def test_keyframe_time_forward_equals_keyframe_row():
    # at t = j/T the temporal feature is row j exactly, and the forward equals the decode of that row
    lm, T = 16, 4
    p, s, tgt = tiny_problem(5, T=T, n=30)
    s[:, 2] = (np.arange(30) % T / T).astype(np.float32)
    y = oracle.fit_forward(p, s, lm, lm, relaxed=True)
    p2 = {k: v.copy() for k, v in p.items()}
    for j in range(T):                                   # make every other row irrelevant: same result
        others = [r for r in range(T) if r != j]
        p2["temporal"][others] = 1e3
        sel = np.flatnonzero(np.arange(30) % T == j)
        y2 = oracle.fit_forward(p2, s[sel], lm, lm, relaxed=True)
        assert np.array_equal(y2, y[sel])
        p2["temporal"][:] = p["temporal"]
