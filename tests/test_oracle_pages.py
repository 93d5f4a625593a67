"""Pin of the oracle's page decode (Sec. 3.5: a page request is a rectangle of
lightmap texels decoded at the request's own t into a physical texture).

The page decode must equal the oracle's point decode (pinned on its own by
the BC4, sampling and MLP tests) at each texel centre
((x0 + i + 0.5) / lm_w, (y0 + j + 0.5) / lm_h, t) of the request's model,
element for element at physical texel (dst_x + i, dst_y + j), with A = 1,
and must leave every texel outside the requests untouched.  The maps are
not square and the requests not square either, so an x/y swap, a half-texel
shift, a wrong pitch or the wrong model or t per request fails here.
"""
import numpy as np

import oracle
import synth


def _models():
    return [
        synth.model(201, 64, 32, 32, 16, 8, 8, 8, 32, temporal_dtype="f32"),
        synth.model(202, 128, 256, 64, 128, 16, 24, 8, 64, temporal_dtype="f16", address_mode=1),
        synth.model(203, 32, 32, 32, 32, 8, 5, 8, 16, temporal_dtype="f32"),
    ]


def _requests(models):
    # (model, x0, y0, w, h, t): corners of each map, ragged sizes, w != h
    spec = [
        (0, 0, 0, 7, 3, 0.0),
        (0, 64 - 5, 32 - 9, 5, 9, 0.999),
        (1, 0, 256 - 16, 16, 16, 0.5),
        (1, 128 - 33, 0, 33, 2, 0.123),
        (1, 40, 100, 1, 1, 0.75),
        (2, 0, 0, 32, 32, 0.6),
        (2, 31, 17, 1, 15, 0.2),
        (0, 10, 4, 20, 11, 0.25),
    ]
    reqs = np.zeros(len(spec), dtype=synth.PAGE_REQ_DTYPE)
    dx = 0
    for i, (mi, x0, y0, w, h, t) in enumerate(spec):
        assert x0 + w <= models[mi]["lm_w"] and y0 + h <= models[mi]["lm_h"]
        reqs[i] = (mi, x0, y0, w, h, np.float32(t), dx + 1, 3 + (i % 3))
        dx += w + 2
    return reqs, dx + 2, 3 + 2 + 40


def test_pages_equal_points_at_texel_centres():
    models = _models()
    reqs, phys_w, phys_h = _requests(models)
    got = oracle.decode_pages(models, reqs, phys_w, phys_h)
    covered = np.zeros((phys_h, phys_w), bool)
    for r in reqs:
        m = models[r["model"]]
        jj, ii = np.meshgrid(np.arange(r["h"]), np.arange(r["w"]), indexing="ij")
        u = ((r["x0"] + ii + 0.5) / m["lm_w"]).astype(np.float32)
        v = ((r["y0"] + jj + 0.5) / m["lm_h"]).astype(np.float32)
        q = np.stack([u.ravel(), v.ravel(), np.full(u.size, r["t"], np.float32)], 1)
        want = oracle.decode_points(m, q).reshape(r["h"], r["w"], 3)
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        assert np.array_equal(got[sl][..., :3], want)
        assert np.all(got[sl][..., 3] == 1.0)
        covered[sl] = True
    assert np.all(np.isnan(got[~covered]))


def test_pages_model_and_time_are_per_request():
    models = _models()
    reqs, phys_w, phys_h = _requests(models)
    base = oracle.decode_pages(models, reqs, phys_w, phys_h, fill=0.0)
    for k in range(len(reqs)):
        r2 = reqs.copy()
        r2["t"][k] = np.float32((float(r2["t"][k]) + 0.37) % 1.0)
        got = oracle.decode_pages(models, r2, phys_w, phys_h, fill=0.0)
        r = reqs[k]
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        changed = np.any(got != base, axis=-1)
        assert changed[sl].any()                      # the request's own t is used ...
        changed[sl] = False
        assert not changed.any()                      # ... and nobody else's
