"""GPU parity of the BC pack and the differentiable fit against the FP64 oracle.

Pack: bit-exact blocks; decode(pack(E, W)) gives exactly the straight-through
features of the fit forward.  Fit samples are queries (u, v, t) with most t
between keyframes, so the temporal interpolation (Eq. 2) and its gradient
split between two keyframe rows are exercised.  Fit forward: <= 1e-5 of
range.  Backward: norm-wise relative error per tensor <= 1e-3 against the
oracle's analytic FP64 gradient (STE) and against FP64 central finite
differences of the continuous relaxation, the latter also elementwise with
an absolute floor of 1e-6 (parameters whose +-h step flips a ReLU are
dropped).
"""
import numpy as np
import pytest

import oracle
import synth
from _gpu import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

KEYS = ("ea", "eb", "w", "temporal", "w1", "b1", "w2", "b2", "w3", "b3")


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def test_bc_pack_bit_exact(ndgi):
    rng = np.random.default_rng(1)
    bh, bw, cs = 64, 48, 16
    ea = rng.random((bh, bw, cs), dtype=np.float32)
    eb = rng.random((bh, bw, cs), dtype=np.float32)
    w = rng.random((bh, bw, cs, 16), dtype=np.float32)
    eb[::7] = ea[::7]                                   # equal endpoints
    ea[0, 0, :4] = [0.0, 1.0, -0.5, 2.0]                # clamped values
    w[1, 1, 0, :] = np.array([0, 1 / 7, 0.5 / 7, 1.5 / 7, 1, 0.9999, 6.5 / 7, 0.5] * 2, np.float32)
    got = ndgi.ndgi_bc_pack(*[torch.from_numpy(a).cuda() for a in (ea, eb, w)]).cpu().numpy()
    assert np.array_equal(got, oracle.bc_pack(ea, eb, w))


def test_decode_of_pack_equals_fit_features(ndgi):
    p = synth.fit_init(5, 64, 64, 8, 8, 8, 32)
    blocks = ndgi.ndgi_bc_pack(*[torch.from_numpy(p[k]).cuda() for k in ("ea", "eb", "w")])
    m = dict(lm_w=128, lm_h=128, feat_w=64, feat_h=64, cs=8, t_count=8, ct=8, hidden=32,
             bc4=blocks.cpu().numpy(), temporal=p["temporal"], address_mode=0,
             **{k: p[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")})
    s = synth.fit_samples(6, 4096, 128, 128, 8)
    q = s
    x, _ = ndgi.ndgi_debug_features(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda())
    y_dec = ndgi.ndgi_decode_points(ndgi.Model.from_arrays(m), torch.from_numpy(q).cuda(), "fp32").cpu().numpy()
    y_fit = ndgi.ndgi_fit_forward(ndgi.FitState.from_arrays(p, 128, 128), torch.from_numpy(s).cuda()).cpu().numpy()
    y_ref = oracle.fit_forward(p, s, 128, 128)
    assert rel_err(y_fit, y_ref) <= 1e-5
    assert rel_err(y_dec, y_ref) <= 1e-5
    # the gather of the packed blocks reproduces the oracle's STE features
    xo, _ = oracle.features(m, q)
    assert np.max(np.abs(x.cpu().numpy() - xo)) < 1e-6


@pytest.mark.parametrize("relaxed", [False, True])
def test_fit_forward(ndgi, relaxed):
    p = synth.fit_init(7, 128, 64, 16, 24, 8, 64)
    s = synth.fit_samples(8, 30001, 256, 128, 24)
    y = ndgi.ndgi_fit_forward(ndgi.FitState.from_arrays(p, 256, 128), torch.from_numpy(s).cuda(),
                              relaxed=relaxed).cpu().numpy()
    yr = oracle.fit_forward(p, s, 256, 128, relaxed=relaxed)
    assert rel_err(y, yr) <= 1e-5


def norm_err(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


@pytest.mark.parametrize("shape", [(4, 4, 16, 64), (16, 8, 64, 3000)])
def test_fit_backward_vs_oracle_ste(ndgi, shape):
    cs, ct, H, n = shape
    feat, lm, T = 32, 64, 6
    p = synth.fit_init(9, feat, feat, cs, T, ct, H)
    s = synth.fit_samples(10, n, lm, lm, T)
    tgt = np.random.default_rng(11).normal(size=(n, 3))
    st = ndgi.FitState.from_arrays(p, lm, lm)
    y = ndgi.ndgi_fit_forward(st, torch.from_numpy(s).cuda())
    dy = (2.0 * (y.double() - torch.from_numpy(tgt).cuda()) / (3 * n)).float()
    g = ndgi.ndgi_fit_backward(st, torch.from_numpy(s).cuda(), dy.contiguous())
    _, gr = oracle.fit_backward(p, s, tgt, lm, lm)
    for k in KEYS:
        assert norm_err(g[k].cpu().numpy(), gr[k]) <= 1e-3, k


def test_fit_backward_vs_finite_differences(ndgi):
    # continuous relaxation: GPU backward against FP64 central differences
    cs, ct, H, lm, feat, T, n = 4, 4, 16, 16, 8, 3, 48
    p = synth.fit_init(12, feat, feat, cs, T, ct, H)
    p["b1"] = p["b1"] + 0.3
    s = synth.fit_samples(13, n, lm, lm, T)
    tgt = np.random.default_rng(14).normal(size=(n, 3))
    st = ndgi.FitState.from_arrays(p, lm, lm)
    y = ndgi.ndgi_fit_forward(st, torch.from_numpy(s).cuda(), relaxed=True)
    dy = (2.0 * (y.double() - torch.from_numpy(tgt).cuda()) / (3 * n)).float()
    g = ndgi.ndgi_fit_backward(st, torch.from_numpy(s).cuda(), dy.contiguous(), relaxed=True)
    base, base_signs = oracle.fit_forward(p, s, lm, lm, relaxed=True, want_signs=True)
    h = 1e-6
    for k in KEYS:
        flat = p[k].reshape(-1)
        fd = np.zeros(flat.size)
        keep = np.ones(flat.size, bool)
        for i in range(flat.size):
            o = flat[i]
            up, dn = np.float32(o + h), np.float32(o - h)
            flat[i] = up
            yu, su = oracle.fit_forward(p, s, lm, lm, relaxed=True, want_signs=True)
            flat[i] = dn
            yd, sd = oracle.fit_forward(p, s, lm, lm, relaxed=True, want_signs=True)
            flat[i] = o
            if not (np.array_equal(su, base_signs) and np.array_equal(sd, base_signs)):
                keep[i] = False
                continue
            fd[i] = (oracle.fit_loss(yu, tgt) - oracle.fit_loss(yd, tgt)) / (float(up) - float(dn))
        gk = g[k].cpu().numpy().reshape(-1)
        assert norm_err(gk[keep], fd[keep]) <= 1e-3, k
        elem = np.abs(gk[keep] - fd[keep]) / np.maximum(np.abs(fd[keep]), 1e-6)
        assert elem.max() <= 1e-3, (k, float(elem.max()))


def test_encode_fit_matches_oracle_loop(ndgi):
    # three Adam steps of the device fit loop against the oracle's loop on the same sample stream
    cs, ct, H, feat, lm, T, batch = 4, 4, 16, 16, 32, 4, 2048
    p = synth.fit_init(15, feat, feat, cs, T, ct, H)
    targets = synth.fit_targets(16, lm, lm, T, n_gauss=6)
    st = ndgi.FitState.from_arrays(p, lm, lm)
    cfg = ndgi.fit_config(steps=3, batch=batch, lr=1e-2, loss_every=1, seed=77)
    _, log = ndgi.ndgi_encode_fit(st, torch.from_numpy(targets).cuda(), cfg)
    torch.cuda.synchronize()
    q = {k: p[k].copy() for k in KEYS}
    mom = {k: (np.zeros(q[k].size), np.zeros(q[k].size)) for k in KEYS}
    losses = []
    for step in range(3):
        texel, s = oracle.fit_draw(77, step, batch, lm, lm)
        tg = oracle.fit_targets_at(targets, texel, s)        # keyframe targets interpolated at each t
        loss, g = oracle.fit_backward(q, s, tg, lm, lm)
        losses.append(loss)
        for i, k in enumerate(KEYS):
            flat = q[k].reshape(-1)
            oracle.adam(flat, g[k].reshape(-1), mom[k][0], mom[k][1], step + 1, 1e-2, project=i < 3)
    assert np.allclose(log.cpu().numpy(), losses, rtol=1e-4)
    for k in KEYS:
        a = st.t[k].cpu().numpy()
        # straight-through rounding decisions can flip for parameters sitting on a bin edge
        frac_close = np.mean(np.abs(a - q[k]) <= 1e-4 + 1e-3 * np.abs(q[k]))
        assert frac_close > 0.99, (k, frac_close)


def test_encode_fit_reduces_loss(ndgi):
    cs, ct, H, feat, lm, T = 16, 8, 64, 64, 128, 8
    p = synth.fit_init(17, feat, feat, cs, T, ct, H)
    targets = synth.fit_targets(18, lm, lm, T, n_gauss=8)
    st = ndgi.FitState.from_arrays(p, lm, lm)
    cfg = ndgi.fit_config(steps=200, batch=1 << 14, lr=1e-2, loss_every=10, freeze_steps=20, seed=3)
    _, log = ndgi.ndgi_encode_fit(st, torch.from_numpy(targets).cuda(), cfg)
    log = log.cpu().numpy()
    assert log[-1] < 0.2 * log[0]
    for k in ("ea", "eb", "w"):
        v = st.t[k]
        assert float(v.min()) >= 0.0 and float(v.max()) <= 1.0


@pytest.mark.parametrize("relaxed", [False, True])
def test_autograd_function_matches_torch_reference(ndgi, relaxed):
    # loss.backward() through ndgi.NdgiDecodeFunction (hand-written CUDA backward)
    # against PyTorch FP64 autograd of an independent statement of the STE forward
    from _fit_ref import tiny_problem, torch_forward
    lm, T = 64, 6
    p, s, tgt = tiny_problem(21, feat=32, lm=lm, cs=4, T=T, ct=4, H=16, n=700)
    params = {k: torch.from_numpy(np.ascontiguousarray(p[k], np.float32)).cuda().requires_grad_()
              for k in KEYS}
    y = ndgi.ndgi_decode_fit(params, torch.from_numpy(s).cuda(), lm, lm, relaxed=relaxed)
    loss = ((y.double() - torch.from_numpy(tgt).cuda()) ** 2).mean()
    loss.backward()
    if relaxed:   # the continuous relaxation: the oracle's analytic FP64 gradient
        yr = oracle.fit_forward(p, s, lm, lm, relaxed=True)
        _, gr = oracle.fit_backward(p, s, tgt, lm, lm, relaxed=True)
        ref_y, ref_g = yr, gr
    else:
        y_t, t = torch_forward(p, s, lm, T)
        ((y_t - torch.from_numpy(tgt)) ** 2).mean().backward()
        ref_y, ref_g = y_t.detach().numpy(), {k: t[k].grad.numpy() for k in KEYS}
    assert rel_err(y.detach().cpu().numpy(), ref_y) <= 1e-5
    for k in KEYS:
        assert norm_err(params[k].grad.cpu().numpy(), ref_g[k]) <= 1e-3, k
