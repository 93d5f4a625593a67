"""The tensor-core epilogues' GELU polynomial (Sec. 4: GELU on the hidden layers)
pinned on the CPU against the exact definition x Phi(x) = x/2 (1 + erf(x/sqrt 2))
with scipy's erf: the coefficients compiled into hybrid.cu are the generator's,
and the kernel's FP32 steps (clamp, Horner on the halved coefficients in
t^2, Phi = 1/2 + t P / 2, x Phi) stay within the documented bound
4.5e-5 + 4e-6 |x| everywhere, including far beyond the clamp."""
import importlib.util
import os
import re

import numpy as np
import pytest

scipy_special = pytest.importorskip("scipy.special")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_12625_gb300", "csrc")


def kernel_coefficients():
    src = open(os.path.join(CSRC, "hybrid.cu")).read()
    body = src[src.index("float2 gelu_poly2("):]
    body = body[:body.index("\n}\n")]
    found = dict(re.findall(r"\b(c\d)\s*=\s*([-+0-9.eE]+)f", body))
    return np.array([float(found[f"c{k}"]) for k in range(9)], dtype=np.float32)


def generator():
    spec = importlib.util.spec_from_file_location("gelu_poly_fit", os.path.join(CSRC, "gelu_poly_fit.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def kernel_steps(x, c):
    """The FP32 operations of gelu_poly2, one rounding per step."""
    f = np.float32
    x = x.astype(f)
    t = np.minimum(np.maximum(x, f(-4.5)), f(4.5))
    s = (t * t).astype(f)
    h = (f(0.5) * c).astype(f)
    p = (h[8] * s + h[7]).astype(f)
    for k in range(6, -1, -1):
        p = (p * s + h[k]).astype(f)
    phi = (t * p + f(0.5)).astype(f)
    return (x * phi).astype(f)


def exact(x):
    x = x.astype(np.float64)
    return 0.5 * x * (1.0 + scipy_special.erf(x / np.sqrt(2.0)))


def test_coefficients_are_the_generators():
    c = kernel_coefficients()
    g = generator().fit()
    np.testing.assert_allclose(c, g, rtol=1e-5, atol=0)


def test_error_bound_on_a_dense_grid():
    c = kernel_coefficients()
    x = np.linspace(-40.0, 40.0, 2_000_001).astype(np.float32)
    err = np.abs(kernel_steps(x, c).astype(np.float64) - exact(x))
    bound = 4.5e-5 + 4e-6 * np.abs(x.astype(np.float64))
    worst = np.argmax(err - bound)
    assert np.all(err <= bound), f"x = {x[worst]}: error {err[worst]:.3e} > {bound[worst]:.3e}"
    # the bound is not loose by orders of magnitude: the polynomial's own error inside the clamp
    assert err[np.abs(x) <= 4.5].max() > 1e-5


def test_special_values():
    c = kernel_coefficients()
    x = np.array([0.0, -0.0, 1e-30, -1e-30, 4.5, -4.5, 1e6, -1e6], dtype=np.float32)
    y = kernel_steps(x, c)
    assert y[0] == 0.0 and y[1] == 0.0
    assert abs(y[2]) < 1e-29 and abs(y[3]) < 1e-29
    # at and beyond the clamp: Phi is held at its value at +-4.5 (within 1.5e-6 of 1 or 0, either side)
    err = np.abs(y[4:].astype(np.float64) - exact(x[4:]))
    assert np.all(err <= 4.5e-5 + 4e-6 * np.abs(x[4:].astype(np.float64)))


def test_error_bound_far_out():
    c = kernel_coefficients()
    m = np.logspace(np.log10(4.5), 30, 20001)
    x = np.concatenate([m, -m]).astype(np.float32)
    err = np.abs(kernel_steps(x, c).astype(np.float64) - exact(x))
    assert np.all(err <= 4.5e-5 + 4e-6 * np.abs(x.astype(np.float64)))
