"""Seeded synthetic inputs for the NDGI decode and fit paths.

This module only *draws* inputs: random BC4 block bytes, temporal feature lines,
Xavier-initialised MLP weights, query coordinates, page requests and procedural
HDR targets.  It holds none of the decode arithmetic (no BC4 palette, no
interpolation, no MLP evaluation), so both the FP64 oracle and the CUDA path
can consume the same arrays without sharing any of the method's code.

The paper's lightmap datasets (FarmLand, Room, City, Yard; supplement S4) are
not public, so every workload is a seeded stand-in with the shapes of the
paper's representation (Sec. 3.3-3.4): 4x4 BC blocks of 8-bit endpoints and
3-bit indices, a small temporal feature axis, and a two-hidden-layer MLP.
"""
from __future__ import annotations

import numpy as np

# Page request record, 32 bytes, matching `ndgi_page_req` in include/ndgi.h.
PAGE_REQ_DTYPE = np.dtype(
    [("model", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("w", "<i4"), ("h", "<i4"),
     ("t", "<f4"), ("dst_x", "<i4"), ("dst_y", "<i4")])

# Fit sample record: a query (u, v, t), like a point decode's.
SAMPLE_DTYPE = np.float32


def _rng(seed):
    return np.random.default_rng(np.random.SeedSequence(int(seed)))


def bc4_planes(rng, feat_w, feat_h, cs):
    """Uniform random BC4 blocks: endpoints and 3-bit indices all uniform.

    Layout [feat_h/4][feat_w/4][cs][8] bytes (block-major, channel-minor).
    """
    assert feat_w % 4 == 0 and feat_h % 4 == 0
    nbytes = (feat_h // 4) * (feat_w // 4) * cs * 8
    raw = np.frombuffer(rng.bytes(nbytes), dtype=np.uint8).copy()
    return raw.reshape(feat_h // 4, feat_w // 4, cs, 8)


def xavier_mlp(rng, cin, hidden, cout=3):
    """Xavier-uniform weights stored [in][out], biases U(-0.1, 0.1)."""
    def lin(fi, fo):
        lim = np.sqrt(6.0 / (fi + fo))
        w = rng.uniform(-lim, lim, size=(fi, fo)).astype(np.float32)
        b = rng.uniform(-0.1, 0.1, size=(fo,)).astype(np.float32)
        return w, b
    w1, b1 = lin(cin, hidden)
    w2, b2 = lin(hidden, hidden)
    w3, b3 = lin(hidden, cout)
    return dict(w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3)


def model(seed, lm_w, lm_h, feat_w, feat_h, cs, t_count, ct, hidden,
          temporal_dtype="f32", address_mode=0, temporal_std=1.0):
    """One decodable model: BC4 planes + temporal line + MLP (all seeded)."""
    rng = _rng(seed)
    bc4 = bc4_planes(rng, feat_w, feat_h, cs)
    temporal = rng.normal(0.0, temporal_std, size=(t_count, ct)).astype(np.float32)
    if temporal_dtype == "f16":
        temporal = temporal.astype(np.float16)
    m = dict(lm_w=lm_w, lm_h=lm_h, feat_w=feat_w, feat_h=feat_h, cs=cs,
             t_count=t_count, ct=ct, hidden=hidden, bc4=bc4, temporal=temporal,
             address_mode=address_mode)
    m.update(xavier_mlp(rng, cs + ct, hidden, 3))
    return m


def random_queries(seed, n):
    """n iid (u, v, t) ~ U[0,1)^3 as float32 [n][3]."""
    rng = _rng(seed)
    return rng.random((n, 3), dtype=np.float32)


def texel_queries(lm_w, lm_h, ts):
    """Every texel centre of an lm_w x lm_h lightmap at each time in `ts`.

    The query for texel (ix, iy) is (u, v) = ((ix + 0.5)/lm_w, (iy + 0.5)/lm_h);
    output rows are ordered [t][iy][ix].
    """
    ix = (np.arange(lm_w, dtype=np.float64) + 0.5) / lm_w
    iy = (np.arange(lm_h, dtype=np.float64) + 0.5) / lm_h
    uu, vv = np.meshgrid(ix, iy)
    out = []
    for t in ts:
        q = np.empty((lm_h * lm_w, 3), dtype=np.float32)
        q[:, 0] = uu.ravel()
        q[:, 1] = vv.ravel()
        q[:, 2] = np.float32(t)
        out.append(q)
    return np.concatenate(out, axis=0)


def small_points_config(seed=1):
    """256x256 lightmap, T=8, 64x64x8 BC4 planes, temporal 8x8 FP32 N(0,1),
    MLP 16->32->32->3; every texel at 4 times t ~ U[0,1)."""
    m = model(seed, 256, 256, 64, 64, 8, 8, 8, 32, temporal_dtype="f32")
    rng = _rng(seed + 1000)
    ts = rng.random(4, dtype=np.float32)
    return m, texel_queries(256, 256, ts)


def points_model_2048(seed=2):
    """2048x2048 atlas, T=24, 1024x1024x16 BC4 planes, temporal 24x8 FP16,
    MLP 24->64->64->3."""
    return model(seed, 2048, 2048, 1024, 1024, 16, 24, 8, 64, temporal_dtype="f16")


# --------------------------------------------------------------------------
# Virtual-texture page requests
# --------------------------------------------------------------------------

PAGE_LIGHTMAP_SIZES = (512, 512, 1024, 1024, 2048, 2048, 4096, 4096)


def page_models(seed=4, sizes=PAGE_LIGHTMAP_SIZES, cs=16, t_count=24, ct=8, hidden=64,
                temporal_dtype="f16"):
    """One model per lightmap; features at half resolution, 16 BC4 planes."""
    return [model(seed * 1000 + i, s, s, s // 2, s // 2, cs, t_count, ct, hidden,
                  temporal_dtype=temporal_dtype) for i, s in enumerate(sizes)]


def zipf_page_requests(seed, lm_sizes, n_req, page=128, s=1.1, slots_x=64):
    """n_req page requests drawn Zipf(s) over all pages of all lightmaps.

    Page list: lightmap-major, then page row, then page column.  A seeded
    permutation maps Zipf rank -> page; draws use the inverse CDF of the
    bounded Zipf law P(r) ~ r^-s, r = 1..n_pages.  Each request gets its own
    t ~ U[0,1) and its own destination slot (slot i at column i % slots_x,
    row i // slots_x of the physical texture, in units of `page` texels).
    """
    rng = _rng(seed)
    pages = []
    for mi, sz in enumerate(lm_sizes):
        npg = sz // page
        for py in range(npg):
            for px in range(npg):
                pages.append((mi, px * page, py * page))
    n_pages = len(pages)
    perm = rng.permutation(n_pages)
    ranks = np.arange(1, n_pages + 1, dtype=np.float64)
    pmf = ranks ** (-s)
    cdf = np.cumsum(pmf / pmf.sum())
    draws = np.searchsorted(cdf, rng.random(n_req), side="right")
    draws = np.minimum(draws, n_pages - 1)
    ts = rng.random(n_req, dtype=np.float32)
    req = np.zeros(n_req, dtype=PAGE_REQ_DTYPE)
    for i in range(n_req):
        mi, x0, y0 = pages[perm[draws[i]]]
        req[i] = (mi, x0, y0, page, page, ts[i], (i % slots_x) * page, (i // slots_x) * page)
    return req


def ragged_page_requests(seed, lm_sizes, n_req, max_side=128, slots_x=8, slot=128):
    """Requests of uneven sizes w, h in 1..max_side at random in-bounds origins,
    each in its own destination slot; includes full-size and 1-texel pages."""
    rng = _rng(seed)
    req = np.zeros(n_req, dtype=PAGE_REQ_DTYPE)
    for i in range(n_req):
        mi = int(rng.integers(0, len(lm_sizes)))
        sz = lm_sizes[mi]
        if i == 0:
            w = h = min(max_side, sz)
        elif i == 1:
            w = h = 1
        else:
            w = int(rng.integers(1, min(max_side, sz) + 1))
            h = int(rng.integers(1, min(max_side, sz) + 1))
        x0 = int(rng.integers(0, sz - w + 1))
        y0 = int(rng.integers(0, sz - h + 1))
        t = np.float32(rng.random())
        req[i] = (mi, x0, y0, w, h, t, (i % slots_x) * slot, (i // slots_x) * slot)
    return req


# --------------------------------------------------------------------------
# Fit (training) inputs
# --------------------------------------------------------------------------

def fit_targets(seed, width, height, t_count, n_gauss=32, ambient=0.05):
    """Procedural HDR lightmap set, FP16 [T][H][W][3].

    Each texel is ambient + sum_g A_g * exp(-|x - c_g|^2 / (2 sigma_g^2)) *
    max(0, cos(2 pi t_j + phi_g)), with t_j = j / T, c_g ~ U[0,W)xU[0,H),
    sigma_g ~ U[8, 64] texels, A_g ~ 4 U[0,1]^3 (RGB) and phi_g ~ U[0, 2 pi):
    a stand-in for a day cycle of baked lighting.
    """
    rng = _rng(seed)
    cx = rng.uniform(0, width, n_gauss)
    cy = rng.uniform(0, height, n_gauss)
    sig = rng.uniform(8.0, 64.0, n_gauss)
    amp = rng.uniform(0.0, 1.0, (n_gauss, 3)) * 4.0
    phi = rng.uniform(0.0, 2 * np.pi, n_gauss)
    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    out = np.empty((t_count, height, width, 3), dtype=np.float16)
    tj = np.arange(t_count, dtype=np.float64) / t_count
    sun = np.maximum(0.0, np.cos(2 * np.pi * tj[:, None] + phi[None, :]))  # [T][G]
    acc = np.zeros((t_count, height, width, 3), dtype=np.float32)
    for g in range(n_gauss):
        gx = np.exp(-((xs - cx[g]) ** 2) / (2 * sig[g] ** 2)).astype(np.float32)
        gy = np.exp(-((ys - cy[g]) ** 2) / (2 * sig[g] ** 2)).astype(np.float32)
        spat = gy[:, None] * gx[None, :]
        for j in range(t_count):
            if sun[j, g] == 0.0:
                continue
            acc[j] += (spat[:, :, None] * (amp[g] * sun[j, g]).astype(np.float32)[None, None, :])
    out[...] = (acc + ambient).astype(np.float16)
    return out


def fit_init(seed, feat_w, feat_h, cs, t_count, ct, hidden, temporal_std=0.1):
    """Initial fit parameters: endpoints and weights ~U(0,1) per block and
    plane, temporal line ~N(0, 0.1^2), Xavier MLP.  Layouts: ea/eb
    [feat_h/4][feat_w/4][cs], w [feat_h/4][feat_w/4][cs][16], temporal [T][ct]."""
    rng = _rng(seed)
    bh, bw = feat_h // 4, feat_w // 4
    p = dict(
        ea=rng.random((bh, bw, cs), dtype=np.float32),
        eb=rng.random((bh, bw, cs), dtype=np.float32),
        w=rng.random((bh, bw, cs, 16), dtype=np.float32),
        temporal=rng.normal(0.0, temporal_std, (t_count, ct)).astype(np.float32),
    )
    p.update(xavier_mlp(rng, cs + ct, hidden, 3))
    return p


def fit_samples(seed, n, width, height, t_count, keyframe_every=4):
    """n fit samples as float32 queries [n][3] (u, v, t): random texel centres
    ((ix + 0.5) / width, (iy + 0.5) / height) at t ~ U[0,1); every
    `keyframe_every`-th sample sits exactly on a keyframe time j / t_count."""
    rng = _rng(seed)
    ix = rng.integers(0, width, n)
    iy = rng.integers(0, height, n)
    t = rng.random(n)
    if keyframe_every:
        kf = np.arange(n) % keyframe_every == 0
        t[kf] = rng.integers(0, t_count, int(kf.sum())) / t_count
    s = np.empty((n, 3), dtype=np.float32)
    s[:, 0] = (ix + 0.5) / width
    s[:, 1] = (iy + 0.5) / height
    s[:, 2] = t
    return s


# --------------------------------------------------------------------------
# Hybrid feature map models (the paper's full decoder, Sec. 3.3 and Sec. 4)
# --------------------------------------------------------------------------

# Profiles of the paper's configuration table: F3D resolution (x 12 t-slices x 4
# channels) and hidden width, for one 128 x 128 tile of a 26-lightmap set whose
# other maps have the sizes of the paper's feature-map table (F_uv 128^2 x 4,
# F_ut and F_vt 64 x 24 x 2).
HYBRID_PROFILES = {"L": (16, 16), "M": (32, 16), "H": (64, 16), "M.64": (32, 64)}
HYBRID_TILE = dict(lm=128, uv=128, vol_t=12, ut=(64, 24), vt=(64, 24), n_lightmaps=26)


def bc7_blocks(rng, w, h):
    """Random BC7 blocks [h/4][w/4][16] with every mode equally likely: uniform
    random bytes whose first byte is rewritten to a mode header (m zero bits, a
    one, then random bits)."""
    b = np.frombuffer(rng.bytes((h // 4) * (w // 4) * 16), dtype=np.uint8).reshape(h // 4, w // 4, 16).copy()
    mode = rng.integers(0, 8, (h // 4, w // 4))
    head = (b[:, :, 0].astype(np.int64) << (mode + 1)) | (1 << mode)
    b[:, :, 0] = (head & 255).astype(np.uint8)
    return b


def hybrid_model(seed, lm_w, lm_h, uv_w, uv_h, vol_w, vol_h, vol_t, ut_w, ut_t, vt_h, vt_t, hidden,
                 address_mode=0, feat_format=0):
    """One hybrid model: uniform random BC4 blocks for F_uv and every F3D t-slice
    (4 planes each; feat_format 1: random BC7 blocks, keys uv_bc7 / vol_bc7),
    uniform random bytes for the UNORM8 planes F_ut [ut_t][ut_w][2] and F_vt
    [vt_t][vt_h][2], and a Xavier MLP 16 -> hidden -> hidden -> 3."""
    rng = _rng(seed)
    if feat_format == 1:
        uv = bc7_blocks(rng, uv_w, uv_h)
        vol = np.stack([bc7_blocks(rng, vol_w, vol_h) for _ in range(vol_t)])
    else:
        uv = bc4_planes(rng, uv_w, uv_h, 4)
        vol = np.stack([bc4_planes(rng, vol_w, vol_h, 4) for _ in range(vol_t)])
    ut = np.frombuffer(rng.bytes(ut_t * ut_w * 2), dtype=np.uint8).reshape(ut_t, ut_w, 2).copy()
    vt = np.frombuffer(rng.bytes(vt_t * vt_h * 2), dtype=np.uint8).reshape(vt_t, vt_h, 2).copy()
    key = "bc7" if feat_format == 1 else "bc4"
    m = {"kind": "hybrid", "lm_w": lm_w, "lm_h": lm_h, "uv_w": uv_w, "uv_h": uv_h, f"uv_{key}": uv,
         "vol_shape": (vol_t, vol_h, vol_w), f"vol_{key}": vol, "ut": ut, "vt": vt, "hidden": hidden,
         "address_mode": address_mode, "feat_format": feat_format}
    m.update(xavier_mlp(rng, 16, hidden, 3))
    return m


def hybrid_tile_model(seed, profile="M.64", address_mode=0, feat_format=0):
    """A 128 x 128 tile model of one of the paper's profiles (L, M, H, M.64)."""
    r, hidden = HYBRID_PROFILES[profile]
    T = HYBRID_TILE
    return hybrid_model(seed, T["lm"], T["lm"], T["uv"], T["uv"], r, r, T["vol_t"], T["ut"][0], T["ut"][1],
                        T["vt"][0], T["vt"][1], hidden, address_mode, feat_format)


def hybrid_tile_requests(seed, n_tiles, n_req, slots_x=64, page=128):
    """n_req whole-tile page requests over n_tiles tile models (request i decodes
    tile model (a seeded uniform draw) at its own t ~ U[0,1) into slot i)."""
    rng = _rng(seed)
    tiles = rng.integers(0, n_tiles, n_req)
    ts = rng.random(n_req, dtype=np.float32)
    req = np.zeros(n_req, dtype=PAGE_REQ_DTYPE)
    for i in range(n_req):
        req[i] = (int(tiles[i]), 0, 0, page, page, ts[i], (i % slots_x) * page, (i // slots_x) * page)
    return req


def _hybrid_keys(feat_format):
    blk = ("uv_bc7", "vol_bc7") if feat_format == 1 else ("uv_bc4", "vol_bc4")
    return blk + ("ut", "vt", "w1", "b1", "w2", "b2", "w3", "b3")


def hybrid_tile_set(seed, n_tiles, profile="M.64", feat_format=0):
    """n_tiles tile models of one profile, stacked along a leading axis (model i
    is hybrid_tile_model(seed * 100003 + i, profile)); see hybrid_tile_of."""
    ms = [hybrid_tile_model(seed * 100003 + i, profile, feat_format=feat_format) for i in range(n_tiles)]
    out = {k: np.stack([m[k] for m in ms]) for k in _hybrid_keys(feat_format)}
    out.update({k: ms[0][k] for k in ("kind", "lm_w", "lm_h", "uv_w", "uv_h", "vol_shape", "hidden",
                                      "address_mode", "feat_format")})
    out["n_tiles"] = n_tiles
    return out


def hybrid_tile_of(s, i):
    """Model i of a hybrid_tile_set as a single-model dict."""
    fmt = s.get("feat_format", 0)
    m = {k: s[k][i] for k in _hybrid_keys(fmt)}
    m.update({k: s[k] for k in ("kind", "lm_w", "lm_h", "uv_w", "uv_h", "vol_shape", "hidden", "address_mode")})
    m["feat_format"] = fmt
    return m


# --------------------------------------------------------------------------
# Non-uniform keyframes with a light-switch event (Sec. 3.1, supplement S4.1)
# --------------------------------------------------------------------------

def switch_key_times(n_hourly=24, t_switch=0.73, gap=1.0 / 96):
    """Keyframe times of a day baked hourly (j / n_hourly) plus two extra sets
    around a light-switch event at t_switch (t_switch -+ gap): float32, sorted,
    n_hourly + 2 values in [0, 1)."""
    t = np.concatenate([np.arange(n_hourly) / n_hourly, [t_switch - gap, t_switch + gap]])
    t = np.unique(np.mod(t, 1.0).astype(np.float32))
    assert t.size == n_hourly + 2
    return t


def fit_targets_at_times(seed, width, height, times, n_gauss=32, ambient=0.05, t_on=0.73, t_off=0.9,
                         lamp_amp=6.0, lamp_sigma=24.0):
    """Procedural HDR lightmaps FP16 [T][H][W][3] at the given times: the
    Gaussian sun-lit blobs of fit_targets (with cos(2 pi t + phi) at the actual
    t) plus a local lamp, a Gaussian of amplitude lamp_amp at a seeded
    position, switched on for t_on <= t < t_off (a light-switch event)."""
    rng = _rng(seed)
    cx, cy = rng.uniform(0, width, n_gauss), rng.uniform(0, height, n_gauss)
    sig = rng.uniform(8.0, 64.0, n_gauss)
    amp = rng.uniform(0.0, 1.0, (n_gauss, 3)) * 4.0
    phi = rng.uniform(0.0, 2 * np.pi, n_gauss)
    lx, ly = rng.uniform(0.2, 0.8) * width, rng.uniform(0.2, 0.8) * height
    lamp_rgb = np.array([1.0, 0.8, 0.5]) * lamp_amp
    xs = np.arange(width, dtype=np.float64) + 0.5
    ys = np.arange(height, dtype=np.float64) + 0.5
    times = np.asarray(times, np.float64)
    out = np.empty((len(times), height, width, 3), dtype=np.float16)
    lamp = (np.exp(-((ys[:, None] - ly) ** 2 + (xs[None, :] - lx) ** 2) / (2 * lamp_sigma ** 2)))[:, :, None] * lamp_rgb
    for j, t in enumerate(times):
        acc = np.full((height, width, 3), ambient, np.float64)
        sun = np.maximum(0.0, np.cos(2 * np.pi * t + phi))
        for g in range(n_gauss):
            if sun[g] == 0.0:
                continue
            gx = np.exp(-((xs - cx[g]) ** 2) / (2 * sig[g] ** 2))
            gy = np.exp(-((ys - cy[g]) ** 2) / (2 * sig[g] ** 2))
            acc += (gy[:, None] * gx[None, :])[:, :, None] * (amp[g] * sun[g])
        if t_on <= t < t_off:
            acc += lamp
        out[j] = acc.astype(np.float16)
    return out


def lightmap_mask(seed, width, height, n_islands=12, fill=0.7):
    """Validity mask [H][W] uint8 of a UV-packed lightmap: rectangular charts
    (seeded islands) covering about `fill` of the texels, 1 = valid."""
    rng = _rng(seed)
    m = np.zeros((height, width), np.uint8)
    while m.mean() < fill:
        w = int(rng.integers(width // 16, width // 3))
        h = int(rng.integers(height // 16, height // 3))
        x, y = int(rng.integers(0, width - w)), int(rng.integers(0, height - h))
        m[y:y + h, x:x + w] = 1
    return m



def hybrid_fit_init(seed, lm_w, lm_h, uv_w, uv_h, vol_w, vol_h, vol_t, ut_w, ut_t, vt_h, vt_t, hidden,
                    address_mode=0, shared_w=False):
    """Initial parameters of a hybrid-decoder fit: endpoints and weights U(0,1) per block and channel of F_uv
    and of every F3D slice (shared_w: one weight per texel for all four channels, Eq. 7), F_ut / F_vt values
    U(0,1), Xavier MLP 16 -> hidden -> hidden -> 3."""
    rng = _rng(seed)
    ubh, ubw, vbh, vbw = uv_h // 4, uv_w // 4, vol_h // 4, vol_w // 4
    wc = () if shared_w else (4,)
    p = dict(lm_w=lm_w, lm_h=lm_h, uv_w=uv_w, uv_h=uv_h, vol_shape=(vol_t, vol_h, vol_w), hidden=hidden,
             address_mode=address_mode,
             uv_ea=rng.random((ubh, ubw, 4), dtype=np.float32), uv_eb=rng.random((ubh, ubw, 4), dtype=np.float32),
             uv_wt=rng.random((ubh, ubw) + wc + (16,), dtype=np.float32),
             vol_ea=rng.random((vol_t, vbh, vbw, 4), dtype=np.float32),
             vol_eb=rng.random((vol_t, vbh, vbw, 4), dtype=np.float32),
             vol_wt=rng.random((vol_t, vbh, vbw) + wc + (16,), dtype=np.float32),
             ut=rng.random((ut_t, ut_w, 2), dtype=np.float32), vt=rng.random((vt_t, vt_h, 2), dtype=np.float32))
    p.update(xavier_mlp(rng, 16, hidden, 3))
    return p
