"""Shared references for the fit tests: a tiny seeded fit problem and an
independent PyTorch FP64 statement of the straight-through fit forward
(autograd then gives the reference gradient)."""
import numpy as np
import torch

import oracle
import synth


def tiny_problem(seed=0, feat=8, lm=16, cs=2, T=3, ct=2, H=6, n=40):
    p = synth.fit_init(seed, feat, feat, cs, T, ct, H)
    p["b1"] = p["b1"] + 0.3  # keep most units active so FD sees a smooth function
    s = synth.fit_samples(seed + 1, n, lm, lm, T)
    tgt = np.random.default_rng(seed + 2).normal(size=(n, 3))
    return p, s, tgt


def torch_forward(p, s, lm, T):
    """Independent PyTorch FP64 statement of the straight-through fit forward at queries s [n][3] = (u, v, t)."""
    t = {k: torch.tensor(np.asarray(v, np.float64), requires_grad=True) for k, v in p.items()
         if k in oracle.FIT_KEYS}
    bh, bw, cs = p["ea"].shape
    fw, fh = bw * 4, bh * 4

    def ste(x, scale):
        xs = torch.tensor(np.asarray(x.detach().numpy(), np.float32))
        q = torch.floor(torch.clamp(xs * scale + 0.5, 0, scale)).double() / scale
        return x + (q - x).detach()

    qa, qb, qw = ste(t["ea"], 255.0), ste(t["eb"], 255.0), ste(t["w"], 7.0)
    # full-resolution feature planes F[c][ty][tx] from blocks (Eq. 7)
    f = (1 - qw) * qa[..., None] + qw * qb[..., None]               # [bh][bw][cs][16]
    f = f.reshape(bh, bw, cs, 4, 4).permute(2, 0, 3, 1, 4).reshape(cs, fh, fw)
    u = torch.tensor(s[:, 0], dtype=torch.float64)
    v = torch.tensor(s[:, 1], dtype=torch.float64)
    x = u * fw - 0.5
    y = v * fh - 0.5
    x0, y0 = torch.floor(x), torch.floor(y)
    fx, fy = x - x0, y - y0
    cx0 = x0.long().clamp(0, fw - 1)
    cx1 = (x0.long() + 1).clamp(0, fw - 1)
    cy0 = y0.long().clamp(0, fh - 1)
    cy1 = (y0.long() + 1).clamp(0, fh - 1)
    vs = ((1 - fy) * ((1 - fx) * f[:, cy0, cx0] + fx * f[:, cy0, cx1])
          + fy * ((1 - fx) * f[:, cy1, cx0] + fx * f[:, cy1, cx1])).T
    # temporal feature: linear interpolation between the keyframes j/T around t (periodic)
    st = torch.tensor(s[:, 2], dtype=torch.float64) * T
    j0 = torch.floor(st)
    al = (st - j0)[:, None]
    j0 = j0.long() % T
    vt = (1 - al) * t["temporal"][j0] + al * t["temporal"][(j0 + 1) % T]
    xin = torch.cat([vs, vt], 1)
    h1 = torch.relu(xin @ t["w1"] + t["b1"])
    h2 = torch.relu(h1 @ t["w2"] + t["b2"])
    return h2 @ t["w3"] + t["b3"], t
