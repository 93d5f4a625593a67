"""GPU parity of the batched per-tile fit (Sec. 3.5: one model per VT tile;
Sec. 4: many models fitted side by side): ndgi_encode_fit_batch against the
oracle's loop run model by model (model m draws with seed + m), against
separate single-model fits, and on a batch of a few hundred tile models."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("ea", "eb", "w", "temporal", "w1", "b1", "w2", "b2", "w3", "b3")


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def problem(M, seed, cs=4, ct=4, H=16, feat=16, lm=32, T=4):
    ps = [synth.fit_init(seed + m, feat, feat, cs, T, ct, H) for m in range(M)]
    tg = np.stack([synth.fit_targets(seed + 100 + m, lm, lm, T, n_gauss=5) for m in range(M)])
    return ps, tg


def test_batch_matches_oracle_loop_per_model(ndgi):
    M, lm, batch, seed = 5, 32, 2048, 91
    ps, tg = problem(M, 30)
    fb = ndgi.FitBatch.from_arrays(ps, lm, lm)
    cfg = ndgi.fit_config(steps=3, batch=batch, lr=1e-2, loss_every=1, seed=seed)
    _, log = ndgi.ndgi_encode_fit_batch(fb, torch.from_numpy(tg).cuda(), cfg)
    torch.cuda.synchronize()
    losses = np.zeros(3)
    for m in range(M):
        q = {k: ps[m][k].copy() for k in KEYS}
        mom = {k: (np.zeros(q[k].size), np.zeros(q[k].size)) for k in KEYS}
        for step in range(3):
            texel, s = oracle.fit_draw(seed + m, step, batch, lm, lm)
            loss, g = oracle.fit_backward(q, s, oracle.fit_targets_at(tg[m], texel, s), lm, lm)
            losses[step] += loss / M
            for i, k in enumerate(KEYS):
                oracle.adam(q[k].reshape(-1), g[k].reshape(-1), mom[k][0], mom[k][1], step + 1, 1e-2, project=i < 3)
        got = fb.model(m)
        for k in KEYS:
            a = got[k].cpu().numpy()
            close = np.mean(np.abs(a - q[k]) <= 1e-4 + 1e-3 * np.abs(q[k]))
            assert close > 0.99, (m, k, close)
    assert np.allclose(log.cpu().numpy(), losses, rtol=1e-4)


def test_batch_equals_separate_fits(ndgi):
    M, lm, seed = 3, 32, 5
    ps, tg = problem(M, 40, cs=16, ct=8, H=64)
    fb = ndgi.FitBatch.from_arrays(ps, lm, lm)
    cfg = ndgi.fit_config(steps=20, batch=4096, lr=1e-2, seed=seed)
    ndgi.ndgi_encode_fit_batch(fb, torch.from_numpy(tg).cuda(), cfg)
    for m in range(M):
        st = ndgi.FitState.from_arrays(ps[m], lm, lm)
        ndgi.ndgi_encode_fit(st, torch.from_numpy(tg[m]).cuda(), ndgi.fit_config(steps=20, batch=4096, lr=1e-2,
                                                                                   seed=seed + m))
        for k in KEYS:
            a, b = fb.model(m)[k].cpu().numpy(), st.t[k].cpu().numpy()
            close = np.mean(np.abs(a - b) <= 1e-4 + 1e-3 * np.abs(b))
            assert close > 0.99, (m, k, close)


def test_many_tile_models_reduce_their_loss(ndgi):
    M, lm = 256, 32
    ps, tg = problem(M, 50, cs=16, ct=8, H=64)
    fb = ndgi.FitBatch.from_arrays(ps, lm, lm)
    cfg = ndgi.fit_config(steps=150, batch=1 << 12, lr=1e-2, loss_every=10, freeze_steps=15, seed=6)
    _, log = ndgi.ndgi_encode_fit_batch(fb, torch.from_numpy(tg).cuda(), cfg)
    log = log.cpu().numpy()
    assert log[-1] < 0.25 * log[0]
    for k in ("ea", "eb", "w"):
        assert float(fb.t[k].min()) >= 0.0 and float(fb.t[k].max()) <= 1.0
