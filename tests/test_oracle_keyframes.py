"""Pins of non-uniform keyframe times (Sec. 3.1: the t_i may be non-uniform,
denser around light-switch events), for the decode's temporal features and
the fit's temporal gradient:

- keyframe times j/T reproduce the uniform path;
- at t = t_j the temporal feature is row j exactly, at a segment's midpoint
  the average of its two rows, including the wrap segment from t_(T-1) to
  t_0 + 1;
- the fit's temporal gradient splits between the segment's two rows in the
  ratio (1 - alpha) : alpha with alpha from the non-uniform segment.
"""
import numpy as np

import oracle
import synth
from _fit_ref import tiny_problem

KEYS = np.float32([0.0, 0.125, 0.25, 0.375, 0.5, 0.625, 0.75, 0.875])
SWITCH = np.float32([0.03125, 0.25, 0.5, 0.6875, 0.71875, 0.75, 0.9375])   # denser around 0.72


def model_with(key_t, T):
    m = synth.model(21, 64, 64, 32, 32, 8, T, 8, 16, temporal_dtype="f32")
    if key_t is not None:
        m["key_t"] = key_t
    return m


def test_uniform_times_reproduce_the_uniform_path():
    q = synth.random_queries(22, 4000)
    a, _ = oracle.features(model_with(None, 8), q)
    b, _ = oracle.features(model_with(KEYS, 8), q)
    assert np.allclose(a, b, rtol=0, atol=1e-14)


def test_rows_at_keyframes_and_midpoints():
    T = len(SWITCH)
    m = model_with(SWITCH, T)
    K = np.asarray(m["temporal"], np.float64)
    q = np.zeros((2 * T, 3), np.float32)
    q[:, :2] = 0.3
    k = SWITCH.astype(np.float64)
    q[:T, 2] = SWITCH
    mids = [(k[j] + k[j + 1]) / 2 for j in range(T - 1)] + [((k[-1] + k[0] + 1) / 2) % 1.0]
    q[T:, 2] = np.float32(mids)
    x, _ = oracle.features(m, q)
    for j in range(T):
        assert np.array_equal(x[j, 8:], K[j])
    for j in range(T):
        tq = float(q[T + j, 2])
        start, end = k[j], (k[j + 1] if j + 1 < T else k[0] + 1)
        tt = tq if tq >= start else tq + 1
        a = (tt - start) / (end - start)                          # ~1/2 up to the FP32 rounding of the midpoint
        assert abs(a - 0.5) < 1e-6
        assert np.allclose(x[T + j, 8:], (1 - a) * K[j] + a * K[(j + 1) % T], rtol=0, atol=1e-12)
    # the wrap segment from either side of t = 0, and times outside [0, 1) (periodic)
    for t, (j0, j1) in ((0.99, (T - 1, 0)), (0.01, (T - 1, 0)), (1.3, (1, 2)), (-0.3, (3, 4))):
        a0, a1, al = oracle.temporal_weights(t, T, SWITCH)
        assert (a0, a1) == (j0, j1) and 0 <= al < 1


def test_fit_temporal_gradient_split_nonuniform():
    lm, T = 16, len(SWITCH)
    p, s, tgt = tiny_problem(6, T=T, n=1)
    p["key_t"] = SWITCH
    k = SWITCH.astype(np.float64)
    for t in (0.70703125, 0.96875, 0.25):
        s[0, 2] = np.float32(t)
        j0, j1, al = oracle.temporal_weights(t, T, SWITCH)
        start, end = k[j0], (k[j1] if j1 > j0 else k[0] + 1)
        tt = t if t >= start else t + 1
        assert abs(al - (tt - start) / (end - start)) < 1e-15
        _, g = oracle.fit_backward(p, s, tgt, lm, lm, relaxed=True)
        gk = g["temporal"]
        total = gk.sum(axis=0)
        for j in range(T):
            w = (1 - al if j == j0 else 0.0) + (al if j == j1 else 0.0)
            assert np.allclose(gk[j], w * total, rtol=1e-12, atol=1e-300), (t, j)
