"""Shared helpers for the GPU parity tests."""
import numpy as np


def rel_err(got, ref, rng=None):
    """max |got - ref| / range(ref) (the HDR range of the evaluated set)."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if rng is None:
        rng = float(ref.max() - ref.min())
    return float(np.max(np.abs(got - ref))) / rng


def edge_queries(n_rand, seed):
    """Random queries plus the edges of the domain: u, v, t at 0, at keyframe-like
    values, and just below 1."""
    rng = np.random.default_rng(seed)
    q = rng.random((n_rand, 3), dtype=np.float32)
    below1 = np.nextafter(np.float32(1), np.float32(0))
    edges = np.array([0.0, 0.5, 0.25, below1, 1e-7, 0.999], np.float32)
    e = np.array(np.meshgrid(edges, edges, edges)).reshape(3, -1).T.astype(np.float32)
    return np.concatenate([q, e], 0)
