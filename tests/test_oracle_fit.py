"""Pins for the oracle's fit: analytic FP64 gradient vs central finite
differences on the continuous relaxation, vs an independent PyTorch FP64
autograd of the straight-through forward, plus Adam and the sampler.
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
    s = oracle.fit_draw(123, 7, 200000, 1024, 1024, 24)
    assert s[:, 0].min() >= 0 and s[:, 0].max() < 1024
    assert s[:, 2].min() >= 0 and s[:, 2].max() < 24
    hist = np.bincount(s[:, 2], minlength=24) / len(s)
    assert np.max(np.abs(hist - 1 / 24)) < 0.003
    a = oracle.fit_draw(123, 7, 10, 1024, 1024, 24, first=5)
    assert np.array_equal(a, s[5:15])
