"""GPU parity of the hybrid decoder's fit (Sec. 3.4's BC simulation applied to
the decoder of Sec. 3.3) against the FP64 oracle (pinned against finite
differences and the packed-model decode):

- forward, straight-through and relaxed: <= 1e-5 of range;
- backward: norm-wise relative error per tensor <= 1e-3, and elementwise
  within 1e-3 of the tensor's largest gradient;
- three Adam steps of the device loop against the oracle's loop on the same
  sample stream and interpolated targets; a longer fit reduces the loss and
  keeps the feature maps in [0, 1];
- the decode of the trained model packed to BC4 / UNORM8 equals the fit's
  straight-through forward.
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = oracle.HFIT_KEYS


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def params(seed, hidden=64, shared=False):
    return synth.hybrid_fit_init(seed, 64, 64, 64, 64, 16, 16, 6, 32, 8, 32, 8, hidden, shared_w=shared)


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("relaxed", [False, True])
@pytest.mark.parametrize("hidden", [16, 64])
def test_forward_matches_oracle(ndgi, relaxed, hidden, shared):
    p = params(1, hidden, shared)
    q = synth.random_queries(2, 20_000)
    q[:2000, :2] = np.random.default_rng(3).uniform(-0.5, 1.5, (2000, 2)).astype(np.float32)
    st = ndgi.HybridFitState.from_arrays(p)
    y = ndgi.ndgi_hybrid_fit_forward(st, torch.from_numpy(q).cuda(), relaxed=relaxed).cpu().numpy()
    assert rel_err(y, oracle.hfit_forward(p, q, relaxed=relaxed)) <= 1e-5


@pytest.mark.parametrize("shared", [False, True])
@pytest.mark.parametrize("relaxed", [False, True])
@pytest.mark.parametrize("hidden", [16, 32, 64])
def test_backward_matches_oracle(ndgi, relaxed, hidden, shared):
    p = params(4, hidden, shared)
    n = 3000
    q = synth.random_queries(5, n)
    tgt = np.random.default_rng(6).normal(size=(n, 3))
    st = ndgi.HybridFitState.from_arrays(p)
    y = ndgi.ndgi_hybrid_fit_forward(st, torch.from_numpy(q).cuda(), relaxed=relaxed)
    dy = (2.0 * (y.double() - torch.from_numpy(tgt).cuda()) / (3 * n)).float().contiguous()
    g = ndgi.ndgi_hybrid_fit_backward(st, torch.from_numpy(q).cuda(), dy, relaxed=relaxed)
    _, gr = oracle.hfit_backward(p, q, tgt, relaxed=relaxed)
    for k in KEYS:
        a = g[k].cpu().numpy().astype(np.float64)
        assert np.linalg.norm(a - gr[k]) <= 1e-3 * max(np.linalg.norm(gr[k]), 1e-30), k
        assert np.abs(a - gr[k]).max() <= 1e-3 * max(np.abs(gr[k]).max(), 1e-30), k


@pytest.mark.parametrize("shared,noise", [(False, 0.0), (True, 0.0), (True, 1.0 / 256)])
def test_encode_fit_matches_oracle_loop(ndgi, shared, noise):
    p = params(7, 16, shared)
    lm, T, batch, seed = 64, 4, 2048, 55
    targets = synth.fit_targets(8, lm, lm, T, n_gauss=6)
    st = ndgi.HybridFitState.from_arrays(p)
    cfg = ndgi.fit_config(steps=3, batch=batch, lr=1e-2, loss_every=1, seed=seed, noise_alpha=noise)
    _, log = ndgi.ndgi_hybrid_encode_fit(st, torch.from_numpy(targets).cuda(), cfg)
    torch.cuda.synchronize()
    q = {k: np.asarray(p[k], np.float32).copy() for k in KEYS}
    qd = dict(p)
    mom = {k: (np.zeros(q[k].size), np.zeros(q[k].size)) for k in KEYS}
    losses = []
    for step in range(3):
        texel, s = oracle.fit_draw(seed, step, batch, lm, lm)
        tg = oracle.fit_targets_at(targets, texel, s)
        qd.update(q)
        nz = oracle.fit_noise(seed, step, batch, noise) if noise else None
        loss, g = oracle.hfit_backward(qd, s, tg, noise=nz)
        losses.append(loss)
        for i, k in enumerate(KEYS):
            oracle.adam(q[k].reshape(-1), g[k].reshape(-1), mom[k][0], mom[k][1], step + 1, 1e-2, project=i < 8)
    assert np.allclose(log.cpu().numpy(), losses, rtol=1e-4)
    for k in KEYS:
        a = st.t[k].cpu().numpy()
        close = np.mean(np.abs(a - q[k]) <= 1e-4 + 1e-3 * np.abs(q[k]))
        assert close > 0.99, (k, close)


def test_fit_reduces_loss_and_packs_to_its_forward(ndgi):
    p = params(9, 64)
    lm, T = 64, 8
    keys = np.float32([0.0, 0.1, 0.25, 0.4, 0.5, 0.7, 0.8, 0.95])
    targets = synth.fit_targets_at_times(10, lm, lm, keys, n_gauss=6, t_on=0.4, t_off=0.8)
    st = ndgi.HybridFitState.from_arrays(p)
    key_dev = torch.from_numpy(keys).cuda()
    cfg = ndgi.fit_config(steps=300, batch=1 << 13, lr=1e-2, loss_every=30, freeze_steps=30, seed=11)
    _, log = ndgi.ndgi_hybrid_encode_fit(st, torch.from_numpy(targets).cuda(), cfg, key_t=key_dev)
    log = log.cpu().numpy()
    assert log[-1] < 0.3 * log[0]
    for k in ("uv_ea", "uv_eb", "uv_wt", "vol_ea", "vol_eb", "vol_wt", "ut", "vt"):
        assert float(st.t[k].min()) >= 0.0 and float(st.t[k].max()) <= 1.0, k
    # pack the trained maps (BC4 per map and per F3D slice, UNORM8 planes) and decode them
    t = st.t
    uv = ndgi.ndgi_bc_pack(t["uv_ea"], t["uv_eb"], t["uv_wt"])
    vol = torch.stack([ndgi.ndgi_bc_pack(t["vol_ea"][k].contiguous(), t["vol_eb"][k].contiguous(),
                                         t["vol_wt"][k].contiguous()) for k in range(t["vol_ea"].shape[0])])
    ut = torch.round(t["ut"] * 255).to(torch.uint8)
    vt = torch.round(t["vt"] * 255).to(torch.uint8)
    hm = ndgi.HybridModel(lm, lm, uv, vol.contiguous(), ut, vt, *[t[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
    qq = torch.from_numpy(synth.random_queries(12, 20_000)).cuda()
    dec = ndgi.ndgi_hybrid_decode_points(hm, qq, "fp32").cpu().numpy()
    # the forward with F_ut / F_vt at their stored UNORM8 values
    t["ut"].copy_(ut.float() / 255)
    t["vt"].copy_(vt.float() / 255)
    fwd = ndgi.ndgi_hybrid_fit_forward(st, qq).cpu().numpy()
    assert rel_err(dec, fwd) <= 1e-5


def test_shared_weight_export_matches_oracle(ndgi):
    p = params(12, 16, shared=True)
    t = {k: torch.from_numpy(np.ascontiguousarray(p[k])).cuda() for k in ("uv_ea", "uv_eb", "uv_wt", "vol_ea",
                                                                           "vol_eb", "vol_wt")}
    uv = ndgi.ndgi_bc_sim7_to_rgba8(t["uv_ea"], t["uv_eb"], t["uv_wt"]).cpu().numpy()
    assert np.array_equal(uv, oracle.bc_sim7_rgba8(p["uv_ea"], p["uv_eb"], p["uv_wt"]))
    vol = ndgi.ndgi_bc_sim7_to_rgba8(t["vol_ea"], t["vol_eb"], t["vol_wt"]).cpu().numpy()
    assert vol.shape == (6 * 16, 16, 4)
    assert np.array_equal(vol, oracle.bc_sim7_rgba8(p["vol_ea"], p["vol_eb"], p["vol_wt"]))
    for key, img in (("uv", uv), ("vol", vol)):
        blk = ndgi.ndgi_bc7_pack_sim(t[f"{key}_ea"], t[f"{key}_eb"], t[f"{key}_wt"])
        assert np.array_equal(blk.cpu().numpy(), oracle.bc7_pack_sim(p[f"{key}_ea"], p[f"{key}_eb"], p[f"{key}_wt"]))
        bw = blk.shape[-2]
        dec = ndgi.ndgi_bc7_decode(blk.reshape(-1, bw, 16)).cpu().numpy()
        assert np.array_equal(dec, img)                       # the pack is exact


def test_shared_weight_fit_packs_exactly_to_bc7(ndgi):
    p = params(13, 64, shared=True)
    lm, T = 64, 8
    targets = synth.fit_targets(14, lm, lm, T, n_gauss=6)
    st = ndgi.HybridFitState.from_arrays(p)
    cfg = ndgi.fit_config(steps=200, batch=1 << 13, lr=1e-2, loss_every=50, seed=15, noise_alpha=1.0 / 256)
    _, log = ndgi.ndgi_hybrid_encode_fit(st, torch.from_numpy(targets).cuda(), cfg)
    assert log[-1] < 0.5 * log[0]
    t = st.t
    uv = ndgi.ndgi_bc7_pack_sim(t["uv_ea"], t["uv_eb"], t["uv_wt"])
    vol = ndgi.ndgi_bc7_pack_sim(t["vol_ea"], t["vol_eb"], t["vol_wt"])
    ut = torch.round(t["ut"] * 255).to(torch.uint8)
    vt = torch.round(t["vt"] * 255).to(torch.uint8)
    hm = ndgi.HybridModel(lm, lm, uv, vol, ut, vt, *[t[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")])
    qq = torch.from_numpy(synth.random_queries(16, 20_000)).cuda()
    dec = ndgi.ndgi_hybrid_decode_points(hm, qq, "fp32").cpu().numpy()
    t["ut"].copy_(ut.float() / 255)
    t["vt"].copy_(vt.float() / 255)
    fwd = ndgi.ndgi_hybrid_fit_forward(st, qq).cpu().numpy()
    assert rel_err(dec, fwd) <= 1e-5


@pytest.mark.parametrize("shared,noise", [(False, 0.0), (True, 1.0 / 256)])
def test_batched_fit_matches_oracle_loops(ndgi, shared, noise):
    """Three stacked models, two steps: each model follows the oracle's loop with its own stream (seed + m)."""
    n_models, lm, T, batch, seed = 3, 64, 4, 1024, 70
    ps = [params(71 + m, 16, shared) for m in range(n_models)]
    targets = np.stack([synth.fit_targets(80 + m, lm, lm, T, n_gauss=6) for m in range(n_models)])
    fb = ndgi.HybridFitBatch.from_arrays(ps)
    cfg = ndgi.fit_config(steps=2, batch=batch, lr=1e-2, loss_every=1, seed=seed, noise_alpha=noise)
    _, log = ndgi.ndgi_hybrid_encode_fit_batch(fb, torch.from_numpy(targets).cuda(), cfg)
    torch.cuda.synchronize()
    losses = np.zeros(2)
    for m in range(n_models):
        q = {k: np.asarray(ps[m][k], np.float32).copy() for k in KEYS}
        qd = dict(ps[m])
        mom = {k: (np.zeros(q[k].size), np.zeros(q[k].size)) for k in KEYS}
        for step in range(2):
            texel, s = oracle.fit_draw(seed + m, step, batch, lm, lm)
            tg = oracle.fit_targets_at(targets[m], texel, s)
            qd.update(q)
            nz = oracle.fit_noise(seed + m, step, batch, noise) if noise else None
            loss, g = oracle.hfit_backward(qd, s, tg, noise=nz)
            losses[step] += loss / n_models
            for i, k in enumerate(KEYS):
                oracle.adam(q[k].reshape(-1), g[k].reshape(-1), mom[k][0], mom[k][1], step + 1, 1e-2,
                            project=i < 8)
        got = fb.model(m)
        for k in KEYS:
            a = got[k].cpu().numpy()
            close = np.mean(np.abs(a - q[k]) <= 1e-4 + 1e-3 * np.abs(q[k]))
            assert close > 0.99, (m, k, close)
    assert np.allclose(log.cpu().numpy(), losses, rtol=1e-4)


def test_batched_fit_equals_separate_fits(ndgi):
    n_models, lm, T, batch, seed = 2, 64, 4, 4096, 90
    ps = [params(91 + m, 64, True) for m in range(n_models)]
    targets = np.stack([synth.fit_targets(95 + m, lm, lm, T, n_gauss=6) for m in range(n_models)])
    cfg = ndgi.fit_config(steps=20, batch=batch, lr=1e-2, loss_every=20, seed=seed)
    fb = ndgi.HybridFitBatch.from_arrays(ps)
    ndgi.ndgi_hybrid_encode_fit_batch(fb, torch.from_numpy(targets).cuda(), cfg)
    for m in range(n_models):
        st = ndgi.HybridFitState.from_arrays(ps[m])
        cfg_m = ndgi.fit_config(steps=20, batch=batch, lr=1e-2, loss_every=20, seed=seed + m)
        ndgi.ndgi_hybrid_encode_fit(st, torch.from_numpy(targets[m]).cuda(), cfg_m)
        got = fb.model(m)
        for k in KEYS:
            a, b = got[k].cpu().numpy(), st.t[k].cpu().numpy()
            close = np.mean(np.abs(a - b) <= 1e-4 + 1e-3 * np.abs(b))   # FP32 atomics order only
            assert close > 0.99, (m, k, close)


def test_fit_resumes_from_its_workspace(ndgi):
    """Two calls of 3 steps (the second with step_offset = 3 and the first call's workspace, which holds the Adam
    moments) follow the same trajectory as one call of 6 steps: same samples, same bias corrections."""
    p = params(17, 16, shared=True)
    lm, T = 64, 4
    targets = torch.from_numpy(synth.fit_targets(18, lm, lm, T, n_gauss=6)).cuda()
    one = ndgi.HybridFitState.from_arrays(p)
    _, log1 = ndgi.ndgi_hybrid_encode_fit(one, targets, ndgi.fit_config(steps=6, batch=2048, loss_every=1, seed=19))
    two = ndgi.HybridFitState.from_arrays(p)
    ws, log_a = ndgi.ndgi_hybrid_encode_fit(two, targets, ndgi.fit_config(steps=3, batch=2048, loss_every=1,
                                                                          seed=19))
    _, log_b = ndgi.ndgi_hybrid_encode_fit(two, targets, ndgi.fit_config(steps=3, batch=2048, loss_every=1, seed=19),
                                           step_offset=3, ws=ws)
    assert np.allclose(np.concatenate([log_a.cpu().numpy(), log_b.cpu().numpy()]), log1.cpu().numpy(), rtol=1e-5)
    for k in KEYS:
        a, b = one.t[k].cpu().numpy(), two.t[k].cpu().numpy()
        assert np.mean(np.abs(a - b) <= 1e-5 + 1e-4 * np.abs(b)) > 0.99, k
