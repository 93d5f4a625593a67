"""GPU parity with non-uniform keyframe times (Sec. 3.1: the t_i may be
non-uniform, denser around a light-switch event): the decodes' temporal lerp
(FP32 points, FP16 tensor-core points on both gather paths, FP16 pages) and
the fit's forward and backward, against the oracle pinned by
test_oracle_keyframes."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import edge_queries, rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


KEYS = synth.switch_key_times()


def model(seed, feat=128, lm=256, cs=16, ct=8, H=64):
    m = synth.model(seed, lm, lm, feat, feat, cs, len(KEYS), ct, H, temporal_dtype="f16")
    m["key_t"] = KEYS
    return m


def queries(n, seed):
    q = edge_queries(n, seed)
    rng = np.random.default_rng(seed + 1)
    k = rng.integers(0, len(KEYS), 2000)
    q[:2000, 2] = KEYS[k]                                         # exactly at keyframes
    q[2000:2400, 2] = np.float32(rng.uniform(KEYS[-1], 1.0, 400))  # the wrap segment
    q[2400:2800, 2] = np.float32(rng.uniform(0.0, KEYS[0] + 1e-3, 400))
    i = int(np.searchsorted(KEYS, 0.73))
    q[2800:3200, 2] = np.float32(rng.uniform(KEYS[i - 1] - 0.02, KEYS[i] + 0.02, 400))   # around the switch
    return q


@pytest.mark.parametrize("prec,n,feat", [("fp32", 20_000, 128), ("fp16", 20_000, 128), ("fp16", 300_000, 128),
                                         ("fp16", 20_000, 1024)])
def test_points_with_switch_keyframes(ndgi, prec, n, feat):
    # feat 1024 with 20,000 queries takes the direct tensor-core gather, the others the decoded-texel cache
    m = model(120, feat=feat, lm=2 * feat)
    mod = ndgi.Model.from_arrays(m)
    q = queries(n, 121)
    got = ndgi.ndgi_decode_points(mod, torch.from_numpy(q).cuda(), prec).cpu().numpy()
    ref = oracle.decode_points(m, q, precision=prec)
    err = rel_err(got, ref)
    print(f"switch keyframes points {prec} n={n} ({ndgi.ndgi_decode_points_path(mod, prec, n)}): {err:.3e}")
    assert err <= (1e-5 if prec == "fp32" else 2e-3)


def test_pages_with_switch_keyframes(ndgi):
    maps = [model(122 + i) for i in range(2)]
    models = [ndgi.Model.from_arrays(m) for m in maps]
    reqs = synth.ragged_page_requests(123, (256, 256), 12, slots_x=4, slot=128)
    i = int(np.searchsorted(KEYS, 0.73))
    reqs["t"][:4] = KEYS[[0, i - 1, i, len(KEYS) - 1]]
    reqs["t"][4] = np.float32(0.995)
    phys = torch.zeros((3 * 128, 4 * 128, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    r, n = ndgi.page_requests_to_device(reqs)
    for shape in ((1, 4, 1), (1, 8, 1)):
        plan.set_shape(*shape)
        plan.decode(r, n)
        assert plan.check() == (0, 0)
        got = phys.cpu().numpy()
        ref = oracle.decode_pages(maps, reqs, 4 * 128, 3 * 128, precision="fp16", fill=0.0)
        for q in reqs:
            sl = (slice(q["dst_y"], q["dst_y"] + q["h"]), slice(q["dst_x"], q["dst_x"] + q["w"]))
            a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
            assert np.abs(a - b).max() <= 2e-3 * max(b.max() - b.min(), 1e-6)
    plan.close()


def norm_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_fit_forward_backward_with_switch_keyframes(ndgi):
    feat, lm, T = 32, 64, len(KEYS)
    p = synth.fit_init(124, feat, feat, 16, T, 8, 64)
    p["key_t"] = KEYS
    s = synth.fit_samples(125, 4000, lm, lm, T)
    s[:500, 2] = np.float32(np.random.default_rng(126).uniform(KEYS[-1], 1.0, 500))
    tgt = np.random.default_rng(127).normal(size=(len(s), 3))
    st = ndgi.FitState.from_arrays(p, lm, lm)
    y = ndgi.ndgi_fit_forward(st, torch.from_numpy(s).cuda())
    assert rel_err(y.cpu().numpy(), oracle.fit_forward(p, s, lm, lm)) <= 1e-5
    dy = (2.0 * (y.double() - torch.from_numpy(tgt).cuda()) / (3 * len(s))).float()
    g = ndgi.ndgi_fit_backward(st, torch.from_numpy(s).cuda(), dy.contiguous())
    _, gr = oracle.fit_backward(p, s, tgt, lm, lm)
    for k in oracle.FIT_KEYS:
        assert norm_err(g[k].cpu().numpy(), gr[k]) <= 1e-3, k
