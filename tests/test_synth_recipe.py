"""The seeded inputs follow the recipe the design states for each workload
(uniform BC4 and BC7 blocks, Xavier-uniform MLPs with U(-0.1, 0.1) biases,
U[0,1)^3 queries, bounded Zipf(1.1) page requests over the 2720 pages of the
eight page-decode lightmaps, procedural targets above their 0.05 ambient floor,
hourly keyframes plus two around the light switch).  Checked by counting and
by the laws' own moments, not by re-running the generators' steps."""
import numpy as np

import synth

PAGE_SIZES = (512, 512, 1024, 1024, 2048, 2048, 4096, 4096)


def test_bc4_blocks_are_uniform():
    b = synth.bc4_planes(synth._rng(7), 256, 256, 16).reshape(-1, 8)   # 65,536 blocks
    n = len(b)
    # six-value mode (r0 <= r1) has probability (1 + 1/256) / 2 for uniform endpoint bytes
    six = np.mean(b[:, 0] <= b[:, 1])
    p = 0.5 + 1.0 / 512
    assert abs(six - p) < 4 * np.sqrt(p * (1 - p) / n)
    # the 3-bit indices of all 16 texels are uniform over 0..7
    bits = np.unpackbits(b[:, 2:].copy(), axis=1, bitorder="little").reshape(n, 48)
    idx = (bits.reshape(n, 16, 3) * np.array([1, 2, 4])).sum(-1).ravel()
    counts = np.bincount(idx, minlength=8)
    e = idx.size / 8
    assert np.all(np.abs(counts - e) < 5 * np.sqrt(e))


def test_bc7_blocks_mix_every_mode():
    b = synth.bc7_blocks(synth._rng(8), 512, 512)   # 16,384 blocks
    first = b.reshape(-1, 16)[:, 0]
    mode = np.array([(v & -v).bit_length() - 1 if v else 8 for v in first.tolist()])
    counts = np.bincount(mode, minlength=9)
    e = len(mode) / 8
    assert counts[8] == 0                       # no reserved-mode block
    assert np.all(np.abs(counts[:8] - e) < 5 * np.sqrt(e))


def test_xavier_mlp_bounds_and_moments():
    m = synth.xavier_mlp(synth._rng(9), 24, 64, 3)
    for wk, bk, (fi, fo) in (("w1", "b1", (24, 64)), ("w2", "b2", (64, 64)), ("w3", "b3", (64, 3))):
        w, b = m[wk].astype(np.float64), m[bk].astype(np.float64)
        lim = np.sqrt(6.0 / (fi + fo))
        assert w.shape == (fi, fo) and b.shape == (fo,)
        assert np.all(np.abs(w) <= lim) and np.all(np.abs(b) < 0.1)
        assert np.abs(w).max() > 0.8 * lim       # spans its range
        # U(-L, L) has mean 0 and variance L^2 / 3
        assert abs(w.mean()) < 4 * lim / np.sqrt(3 * w.size)
        assert abs(w.var() / (lim * lim / 3) - 1) < 6 / np.sqrt(w.size)


def test_queries_are_uniform_in_the_unit_cube():
    q = synth.random_queries(10, 1 << 16)
    assert q.dtype == np.float32 and q.shape == (1 << 16, 3)
    assert np.all((q >= 0) & (q < 1))
    assert np.all(np.abs(q.mean(0) - 0.5) < 4 * np.sqrt(1 / 12 / len(q)))


def test_zipf_requests_follow_the_bounded_law():
    n_req = 4096
    req = synth.zipf_page_requests(4, PAGE_SIZES, n_req)
    n_pages = sum((s // 128) ** 2 for s in PAGE_SIZES)
    assert n_pages == 2720
    assert np.all(req["w"] == 128) and np.all(req["h"] == 128)
    sizes = np.array(PAGE_SIZES)[req["model"]]
    assert np.all((req["x0"] % 128 == 0) & (req["y0"] % 128 == 0))
    assert np.all((req["x0"] + 128 <= sizes) & (req["y0"] + 128 <= sizes))
    assert np.all((req["t"] >= 0) & (req["t"] < 1))
    slots = set(zip(req["dst_x"].tolist(), req["dst_y"].tolist()))
    assert len(slots) == n_req                   # every request has its own slot
    # rank-frequency: the law P(r) = r^-1.1 / H over r = 1..2720
    pmf = np.arange(1, n_pages + 1, dtype=np.float64) ** -1.1
    pmf /= pmf.sum()
    key = req["model"].astype(np.int64) * (1 << 40) + req["y0"].astype(np.int64) * (1 << 20) + req["x0"]
    counts = np.sort(np.unique(key, return_counts=True)[1])[::-1]
    top = n_req * pmf[0]
    assert abs(counts[0] - top) < 4 * np.sqrt(top)
    unique_expected = np.sum(1 - (1 - pmf) ** n_req)
    assert abs(len(counts) - unique_expected) < 0.05 * unique_expected


def test_fit_targets_floor_and_day_cycle():
    t = synth.fit_targets(3, 64, 64, 24).astype(np.float64)
    assert t.shape == (24, 64, 64, 3) and np.all(np.isfinite(t))
    assert t.min() >= 0.05 * (1 - 2.0 ** -10)    # ambient floor (FP16-rounded)
    assert t.max() <= 0.05 + 4 * 32 + 1e-3       # at most every Gaussian at full amplitude
    per_t = t.mean(axis=(1, 2, 3))
    assert per_t.max() > 1.5 * per_t.min()       # the light changes over the day


def test_switch_keyframes():
    k = synth.switch_key_times()
    assert k.dtype == np.float32 and k.size == 26
    assert np.all(np.diff(k) > 0) and k[0] == 0 and k[-1] < 1
    hourly = np.arange(24) / 24
    extra = np.setdiff1d(np.round(k.astype(np.float64), 6), np.round(hourly, 6))
    assert extra.size == 2 and np.all(np.abs(extra - 0.73) < 0.011)


def test_lightmap_mask_fill():
    m = synth.lightmap_mask(11, 256, 256)
    assert m.dtype == np.uint8 and set(np.unique(m).tolist()) <= {0, 1}
    assert 0.7 <= m.mean() < 0.9
