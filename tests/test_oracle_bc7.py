"""Pins of the oracle's BC7 block format and encoder (the paper's storage for
F_uv and the F3D slices, Sec. 3.4 and supplement S2).

What the format fixes and these tests check without the oracle's own code:
- field widths: every mode's fields fill exactly 128 bits (every encoder
  candidate of every mode and partition writes a complete block);
- partition tables: texel 0 is in subset 0, every subset is non-empty and
  contains its anchor texel, the 64 shapes of each table are distinct; a few
  shapes that the format's figures show (halves, quarters, stripes);
- endpoint layout: blocks written here field by field (mode, partition,
  rotation, selector, endpoints channel-major, p-bits, indices with short
  anchors) decode to endpoint 0 of each texel's subset when every index is 0
  and to endpoint 1 when every non-anchor index is maximal, with bit
  replication of the endpoint codes;
- rotation and the index selector of modes 4 and 5;
- the reserved mode decodes to zero;
- encoder: the returned error is the error of the block's decode; it is the
  minimum over every candidate; blocks of exactly representable texels
  encode with error 0; constant blocks are within one level per channel.
The partition and anchor tables are further checked against the GPU's own
fixed-function BC7 decoder (tests/test_gpu_bc7.py).
"""
import numpy as np
import pytest

import oracle

# the published mode table: subsets, partition bits, rotation bits, selector bits, colour bits, alpha bits,
# p-bit per endpoint, p-bit per subset, index bits, secondary index bits
MODES = {0: (3, 4, 0, 0, 4, 0, 1, 0, 3, 0), 1: (2, 6, 0, 0, 6, 0, 0, 1, 3, 0), 2: (3, 6, 0, 0, 5, 0, 0, 0, 2, 0),
         3: (2, 6, 0, 0, 7, 0, 1, 0, 2, 0), 4: (1, 0, 2, 1, 5, 6, 0, 0, 2, 3), 5: (1, 0, 2, 0, 7, 8, 0, 0, 2, 2),
         6: (1, 0, 0, 0, 7, 7, 1, 0, 4, 0), 7: (2, 6, 0, 0, 5, 5, 1, 0, 2, 0)}


class Writer:
    def __init__(self):
        self.v, self.n = 0, 0

    def put(self, bits, value):
        assert 0 <= value < (1 << bits) or bits == 0
        self.v |= value << self.n
        self.n += bits

    def block(self):
        assert self.n == 128, self.n
        return np.frombuffer(self.v.to_bytes(16, "little"), np.uint8).copy()


def replicate(code, n):
    return code if n >= 8 else (code << (8 - n)) | (code >> (2 * n - 8))


def write_block(mode, part, rot, isb, codes, pbits, idx1, idx2):
    """codes[s][e][c] (c over the mode's channels), pbits per endpoint [s][e] or per subset [s]."""
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    w = Writer()
    w.put(mode + 1, 1 << mode)
    w.put(pb, part)
    w.put(rb, rot)
    w.put(ib_, isb)
    nch = 4 if ab else 3
    for c in range(nch):
        for s in range(ns):
            for e in range(2):
                w.put(cb if c < 3 else ab, codes[s][e][c])
    if epb:
        for s in range(ns):
            for e in range(2):
                w.put(1, pbits[s][e])
    if spb:
        for s in range(ns):
            w.put(1, pbits[s])
    anchors = {oracle.bc7_anchor(ns, part, s) for s in range(ns)}
    for p in range(16):
        w.put(ib - (p in anchors), idx1[p])
    if ib2:
        for p in range(16):
            w.put(ib2 - (p == 0), idx2[p])
    return w.block()


def expected_endpoint(mode, codes, pbits, s, e):
    """8-bit RGBA of endpoint e of subset s after p-bit append and bit replication."""
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    out = []
    for c in range(4):
        if c == 3 and not ab:
            out.append(255)
            continue
        n = cb if c < 3 else ab
        v = codes[s][e][c]
        if epb:
            v, n = (v << 1) | pbits[s][e], n + 1
        elif spb:
            v, n = (v << 1) | pbits[s], n + 1
        out.append(replicate(v, n))
    return out


def random_fields(rng, mode, part):
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    codes = [[[int(rng.integers(0, 1 << (cb if c < 3 else ab))) for c in range(4 if ab else 3)] for _ in range(2)]
             for _ in range(ns)]
    pbits = ([[int(rng.integers(0, 2)) for _ in range(2)] for _ in range(ns)] if epb else
             [int(rng.integers(0, 2)) for _ in range(ns)])
    return codes, pbits


def test_partition_tables_are_valid():
    for ns in (2, 3):
        shapes = set()
        for part in range(64):
            sub = [oracle.bc7_subset(ns, part, p) for p in range(16)]
            assert sub[0] == 0
            assert set(sub) == set(range(ns)), (ns, part)
            for s in range(ns):
                assert sub[oracle.bc7_anchor(ns, part, s)] == s, (ns, part, s)
            shapes.add(tuple(sub))
        assert len(shapes) == 64
    assert oracle.bc7_anchor(2, 5, 0) == 0


def test_partition_shapes_from_the_format_figures():
    def shape(ns, part):
        return "".join(str(oracle.bc7_subset(ns, part, p)) for p in range(16))
    assert shape(2, 0) == "0011" * 4              # left half | right half
    assert shape(2, 13) == "0000" * 2 + "1111" * 2  # top half / bottom half
    assert shape(2, 15) == "0000" * 3 + "1111"    # bottom row
    assert shape(2, 32) == "0101" * 4             # column stripes
    assert shape(2, 33) == "0000111100001111"     # row stripes
    assert shape(3, 8) == "0000" * 2 + "1111" + "2222"
    assert shape(3, 11) == "0012" * 4


@pytest.mark.parametrize("mode", range(8))
def test_every_candidate_fills_128_bits(mode):
    rng = np.random.default_rng(mode)
    x = rng.integers(0, 256, (16, 4), dtype=np.uint8)
    x[:, 3] = 255
    nparts = {0: 16, 1: 64, 2: 64, 3: 64, 7: 64}.get(mode, 1)
    rots = 4 if mode in (4, 5) else 1
    isbs = 2 if mode == 4 else 1
    for part in range(nparts):
        for rot in range(rots):
            for isb in range(isbs):
                blk, err = oracle.bc7_candidate(x, mode, part, rot, isb)
                assert err >= 0, (mode, part, rot, isb)
                assert (blk[0] & ((1 << (mode + 1)) - 1)) == (1 << mode)
                dec = oracle.bc7_decode_block(blk).astype(np.int64)
                assert err == int(((dec - x) ** 2).sum())


@pytest.mark.parametrize("mode", range(8))
def test_endpoint_layout_by_extreme_indices(mode):
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    rng = np.random.default_rng(10 + mode)
    for part in ([0, 1, 13, 37, 63][: (1 if ns == 1 else 5)] if mode else [0, 3, 9, 15]):
        codes, pbits = random_fields(rng, mode, part)
        zeros = [0] * 16
        blk = write_block(mode, part, 0, 0, codes, pbits, zeros, zeros)
        dec = oracle.bc7_decode_block(blk)
        for p in range(16):
            s = oracle.bc7_subset(ns, part, p)
            assert list(dec[p]) == expected_endpoint(mode, codes, pbits, s, 0), (mode, part, p)
        anchors = {oracle.bc7_anchor(ns, part, s) for s in range(ns)}
        top = [(1 << ib) - 1 if p not in anchors else 0 for p in range(16)]
        top2 = [(1 << ib2) - 1 if p != 0 else 0 for p in range(16)] if ib2 else zeros
        blk = write_block(mode, part, 0, 0, codes, pbits, top, top2)
        dec = oracle.bc7_decode_block(blk)
        for p in range(16):
            s = oracle.bc7_subset(ns, part, p)
            want = expected_endpoint(mode, codes, pbits, s, 0 if p in anchors else 1)
            if ib2 and p != 0:
                want[3] = expected_endpoint(mode, codes, pbits, s, 1)[3]
            if ib2 and p == 0:
                want[3] = expected_endpoint(mode, codes, pbits, s, 0)[3]
            assert list(dec[p]) == want, (mode, part, p)


@pytest.mark.parametrize("mode", [4, 5])
def test_rotation_and_index_selector(mode):
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    rng = np.random.default_rng(30 + mode)
    codes, pbits = random_fields(rng, mode, 0)
    # colour on index 0 (endpoint 0), alpha on its maximal index (endpoint 1) for texels 1..15
    idx1 = [0] * 16
    idx2 = [0] + [(1 << ib2) - 1] * 15
    e0 = expected_endpoint(mode, codes, pbits, 0, 0)
    e1 = expected_endpoint(mode, codes, pbits, 0, 1)
    for rot in range(4):
        for isb in range(2 if mode == 4 else 1):
            dec = oracle.bc7_decode_block(write_block(mode, 0, rot, isb, codes, pbits, idx1, idx2))
            v = list(dec[5])
            # isb = 0: colour from the primary (0 -> e0), alpha from the secondary (max -> e1); isb = 1 swaps them
            want = [e1[0], e1[1], e1[2], e0[3]] if isb else [e0[0], e0[1], e0[2], e1[3]]
            if rot:
                want[rot - 1], want[3] = want[3], want[rot - 1]
            assert v == want, (mode, rot, isb)


def test_reserved_mode_decodes_to_zero():
    blk = np.zeros(16, np.uint8)
    blk[1:] = 0xA5
    assert not oracle.bc7_decode_block(blk).any()


def test_encoder_is_the_minimum_over_candidates():
    rng = np.random.default_rng(40)
    for trial in range(6):
        x = rng.integers(0, 256, (16, 4), dtype=np.uint8)
        if trial % 2:
            x[:, 3] = 255
            x[:, :3] = np.clip(x[:1, :3].astype(int) + rng.integers(-20, 21, (16, 3)), 0, 255)
        blk, err = oracle.bc7_encode_block(x)
        dec = oracle.bc7_decode_block(blk).astype(np.int64)
        assert err == int(((dec - x) ** 2).sum())
        best = []
        best.append(oracle.bc7_candidate(x, 6)[1])
        best += [oracle.bc7_candidate(x, 5, 0, r)[1] for r in range(4)]
        best += [oracle.bc7_candidate(x, 4, 0, r, i)[1] for r in range(4) for i in range(2)]
        best += [oracle.bc7_candidate(x, 7, q)[1] for q in range(64)]
        if (x[:, 3] == 255).all():
            best += [oracle.bc7_candidate(x, m, q)[1] for m in (3, 1, 2) for q in range(64)]
            best += [oracle.bc7_candidate(x, 0, q)[1] for q in range(16)]
        assert err == min(best)


@pytest.mark.parametrize("mode", [6, 5, 7, 3, 1])
def test_representable_blocks_encode_exactly(mode):
    """Texels decoded from a block whose endpoints are the per-channel minimum and maximum of its subset's
    texels (so that the encoder's endpoint choice recovers them) re-encode with error 0."""
    ns, pb, rb, ib_, cb, ab, epb, spb, ib, ib2 = MODES[mode]
    rng = np.random.default_rng(50 + mode)
    done = 0
    for _ in range(200):
        part = int(rng.integers(0, 64)) if ns > 1 else 0
        codes, pbits = random_fields(rng, mode, part)
        for s in range(ns):
            for c in range(len(codes[s][0])):
                lo, hi = sorted((codes[s][0][c], codes[s][1][c]))
                codes[s][0][c], codes[s][1][c] = lo, hi
            if epb:
                pbits[s] = [0, 1] if pbits[s][0] > pbits[s][1] else pbits[s]
        anchors = {oracle.bc7_anchor(ns, part, s) for s in range(ns)}
        idx1 = [int(rng.integers(0, 1 << (ib - (p in anchors)))) for p in range(16)]
        idx2 = [int(rng.integers(0, 1 << (ib2 - (p == 0)))) for p in range(16)] if ib2 else [0] * 16
        # make every subset use both extreme indices so its bounding box is its endpoints
        for s in range(ns):
            mem = [p for p in range(16) if oracle.bc7_subset(ns, part, p) == s and p not in anchors]
            if len(mem) < 1:
                break
            a = oracle.bc7_anchor(ns, part, s)
            idx1[a] = 0
            idx1[mem[0]] = (1 << ib) - 1
            if ib2:
                idx2[0] = 0
                idx2[mem[0]] = (1 << ib2) - 1
        x = oracle.bc7_decode_block(write_block(mode, part, 0, 0, codes, pbits, idx1, idx2))
        lo_ok = True
        for s in range(ns):
            sel = [p for p in range(16) if oracle.bc7_subset(ns, part, p) == s]
            e0 = expected_endpoint(mode, codes, pbits, s, 0)
            e1 = expected_endpoint(mode, codes, pbits, s, 1)
            lo_ok &= list(x[sel].min(0)) == [min(a, b) for a, b in zip(e0, e1)]
            lo_ok &= list(x[sel].max(0)) == [max(a, b) for a, b in zip(e0, e1)]
        if not lo_ok:
            continue
        _, err = oracle.bc7_candidate(x, mode, part)
        assert err == 0, (mode, part)
        assert oracle.bc7_encode_block(x)[1] == 0
        done += 1
    assert done >= 20


def test_constant_blocks_within_one_level():
    rng = np.random.default_rng(60)
    for _ in range(50):
        x = np.repeat(rng.integers(0, 256, (1, 4), dtype=np.uint8), 16, 0)
        blk, err = oracle.bc7_encode_block(x)
        dec = oracle.bc7_decode_block(blk).astype(int)
        assert np.abs(dec - x).max() <= 1


def test_image_encode_decode_layout():
    rng = np.random.default_rng(70)
    img = rng.integers(0, 256, (8, 12, 4), dtype=np.uint8)
    blocks, err = oracle.bc7_encode(img)
    assert blocks.shape == (2, 3, 16)
    dec = oracle.bc7_decode(blocks, 12, 8)
    assert err == int(((dec.astype(np.int64) - img) ** 2).sum())
    for by in range(2):
        for bx in range(3):
            want = oracle.bc7_decode_block(blocks[by, bx]).reshape(4, 4, 4)
            assert np.array_equal(dec[4 * by:4 * by + 4, 4 * bx:4 * bx + 4], want)


# --------------------------------------------------------------------------
# The hybrid decoder over BC7 maps
# --------------------------------------------------------------------------

def bc7_model(seed=81, mode=0):
    import synth
    return synth.hybrid_model(seed, 64, 32, 32, 16, 16, 8, 8, 20, 9, 28, 7, 16, address_mode=mode, feat_format=1)


def test_random_blocks_cover_every_mode():
    import synth
    b = synth.bc7_blocks(np.random.default_rng(1), 64, 64)
    modes = [int(np.flatnonzero([(v >> k) & 1 for k in range(8)])[0]) for v in b[:, :, 0].ravel()]
    assert set(modes) == set(range(8))


@pytest.mark.parametrize("mode", [0, 1])
def test_hybrid_bc7_uv_at_texel_centres_and_midpoints(mode):
    """At F_uv texel centres V_uv is the decoded byte / 255; halfway between two centres (exact coordinates for
    power-of-two sizes) it is their average."""
    m = bc7_model(82, mode)
    img = oracle.bc7_decode(m["uv_bc7"], m["uv_w"], m["uv_h"]).astype(np.float64) / 255.0
    iy, ix = np.meshgrid(np.arange(m["uv_h"]), np.arange(m["uv_w"]), indexing="ij")
    q = np.zeros((ix.size, 3), np.float32)
    q[:, 0] = (ix.ravel() + 0.5) / m["uv_w"]
    q[:, 1] = (iy.ravel() + 0.5) / m["uv_h"]
    q[:, 2] = 0.3
    _, x = oracle.hybrid_decode_points(m, q, features=True)
    assert np.array_equal(x[:, 4:8], img[iy.ravel(), ix.ravel()])
    qm = q.copy()
    qm[:, 0] = (ix.ravel() + 1.0) / m["uv_w"]          # halfway to the right neighbour
    sel = ix.ravel() < m["uv_w"] - 1
    _, xm = oracle.hybrid_decode_points(m, qm[sel], features=True)
    want = 0.5 * (img[iy.ravel(), ix.ravel()] + img[iy.ravel(), np.minimum(ix.ravel() + 1, m["uv_w"] - 1)])[sel]
    assert np.allclose(xm[:, 4:8], want, rtol=0, atol=1e-15)


def test_hybrid_bc7_volume_at_slice_and_texel_centres():
    m = bc7_model(83)
    vol_t, vol_h, vol_w = m["vol_shape"]
    iy, ix = np.meshgrid(np.arange(vol_h), np.arange(vol_w), indexing="ij")
    for k in range(vol_t):
        img = oracle.bc7_decode(m["vol_bc7"][k], vol_w, vol_h).astype(np.float64) / 255.0
        q = np.zeros((ix.size, 3), np.float32)
        q[:, 0] = (ix.ravel() + 0.5) / vol_w
        q[:, 1] = (iy.ravel() + 0.5) / vol_h
        q[:, 2] = (k + 0.5) / vol_t
        _, x = oracle.hybrid_decode_points(m, q, features=True)
        assert np.array_equal(x[:, 0:4], img[iy.ravel(), ix.ravel()]), k


def test_lines_with_mixed_channel_directions():
    """Texels on a line from A to B whose channels run in different directions (some rise, some fall): the
    box diagonal follows the data (covariance signs), so mode 6 stays within a few levels."""
    rng = np.random.default_rng(90)
    for _ in range(30):
        A = rng.integers(0, 256, 4)
        B = rng.integers(0, 256, 4)
        k = rng.integers(0, 16, 16)
        k[:2] = (0, 15)
        x = np.rint(A[None] * (1 - k[:, None] / 15) + B[None] * (k[:, None] / 15)).astype(np.uint8)
        blk, err = oracle.bc7_candidate(x, 6)
        assert np.abs(oracle.bc7_decode_block(blk).astype(int) - x).max() <= 3
