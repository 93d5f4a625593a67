"""GPU parity of BC7 (the paper's block format for F_uv and the F3D slices,
Sec. 3.4) against the oracle, and of the oracle against the GPU's own
fixed-function BC7 decoder (the texture unit), an implementation of the
format independent of both:

- decode: random blocks of every mode, bit-exact: CUDA = oracle = texture unit;
- encode: bit-exact blocks and total squared error against the oracle's
  encoder on noise, smooth, opaque and constant images; its blocks decode on
  the texture unit to the oracle's decode;
- the 8-bit export of four BC4 planes against round(P35 / 35) of the oracle's
  palette integers;
- the hybrid decoder over BC7 maps (points FP32 / FP16, pages FP32 / FP16
  with a border) against the oracle, at the BC4 hybrid tests' gates.
"""
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


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def images(seed):
    """RGBA8 test images 64 x 64: noise, smooth ramps with noise, opaque smooth, constant blocks."""
    rng = np.random.default_rng(seed)
    yy, xx = np.meshgrid(np.arange(64), np.arange(64), indexing="ij")
    noise = rng.integers(0, 256, (64, 64, 4), dtype=np.uint8)
    smooth = np.stack([(xx * 3 + yy) % 256, (yy * 2 + 40) % 256, (xx + yy * 3) % 256, 255 - xx * 2], -1)
    smooth = np.clip(smooth + rng.integers(-6, 7, smooth.shape), 0, 255).astype(np.uint8)
    opaque = smooth.copy()
    opaque[..., 3] = 255
    const = np.repeat(np.repeat(rng.integers(0, 256, (16, 16, 4), dtype=np.uint8), 4, 0), 4, 1)
    return {"noise": noise, "smooth": smooth, "opaque": opaque, "const": const}


def test_decode_matches_oracle_and_texture_unit(ndgi):
    blocks = synth.bc7_blocks(np.random.default_rng(1), 64, 128)
    blocks[0, 0, :] = 0                                   # a reserved-mode block
    ref = oracle.bc7_decode(blocks, 64, 128)
    got = ndgi.ndgi_bc7_decode(cu(blocks)).cpu().numpy()
    hw = ndgi.ndgi_debug_bc7_hw_decode(cu(blocks)).cpu().numpy()
    assert np.array_equal(got, ref)
    assert np.array_equal(hw[4:], ref[4:])                # the texture unit, away from the reserved block
    mism = np.argwhere(hw != ref)
    assert mism.size == 0 or (mism[:, 0] < 4).all()


@pytest.mark.parametrize("mode", range(8))
def test_every_partition_on_the_texture_unit(ndgi, mode):
    """For each mode, a block per partition (random fields): the oracle's partition and anchor tables equal the
    texture unit's."""
    rng = np.random.default_rng(10 + mode)
    n_parts = {0: 16, 1: 64, 2: 64, 3: 64, 7: 64}.get(mode, 4)
    b = np.frombuffer(rng.bytes(n_parts * 16 * 4), np.uint8).reshape(n_parts, 4, 16).copy()
    pb = {0: 4, 1: 6, 2: 6, 3: 6, 7: 6}.get(mode, 0)
    for q in range(n_parts):
        for k in range(4):
            v = int.from_bytes(b[q, k].tobytes(), "little")
            head = (1 << mode) | ((q if pb else k) << (mode + 1))      # mode, then partition (or rotation bits)
            v = (v & ~((1 << (mode + 1 + max(pb, 2))) - 1)) | head
            b[q, k] = np.frombuffer(v.to_bytes(16, "little"), np.uint8)
    ref = oracle.bc7_decode(b, 16, 4 * n_parts)
    hw = ndgi.ndgi_debug_bc7_hw_decode(cu(b)).cpu().numpy()
    got = ndgi.ndgi_bc7_decode(cu(b)).cpu().numpy()
    assert np.array_equal(hw, ref), np.argwhere(hw != ref)[:5]
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("kind", ["noise", "smooth", "opaque", "const"])
def test_encode_matches_oracle(ndgi, kind):
    img = images(20)[kind]
    ref_blocks, ref_err = oracle.bc7_encode(img)
    err = torch.zeros(1, dtype=torch.int64, device="cuda")
    got = ndgi.ndgi_bc7_encode(cu(img), sq_err=err).cpu().numpy()
    assert int(err.item()) == ref_err
    assert np.array_equal(got, ref_blocks)
    hw = ndgi.ndgi_debug_bc7_hw_decode(cu(got)).cpu().numpy()
    assert np.array_equal(hw, oracle.bc7_decode(ref_blocks, 64, 64))
    if kind == "const":
        assert np.abs(hw.astype(int) - img).max() <= 1
    modes = {int(np.flatnonzero([(v >> k) & 1 for k in range(8)])[0]) for v in got[:, :, 0].ravel()}
    print(f"bc7 encode {kind}: rms {np.sqrt(ref_err / img.size):.2f}, modes {sorted(modes)}")


def test_encode_stacked_slices_and_bad_arguments(ndgi):
    from paper_2604_12625_gb300 import _abi as A
    import ctypes as C
    img = images(21)["smooth"][:, :32]                    # 64 x 32: two 32 x 32 slices stacked along h
    got = ndgi.ndgi_bc7_encode(cu(img)).cpu().numpy()
    for k in range(2):
        ref, _ = oracle.bc7_encode(np.ascontiguousarray(img[32 * k:32 * (k + 1)]))
        assert np.array_equal(got[8 * k:8 * (k + 1)], ref)
    L = A.lib()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    assert L.ndgi_bc7_encode(buf.data_ptr(), 6, 8, buf.data_ptr(), None, s) == A.NDGI_ERR_INVALID_ARG
    assert L.ndgi_bc7_decode(None, 8, 8, buf.data_ptr(), s) == A.NDGI_ERR_INVALID_ARG
    assert L.ndgi_bc7_decode(buf.data_ptr() + 4, 8, 8, buf.data_ptr(), s) == A.NDGI_ERR_INVALID_ARG


def test_bc4x4_export_to_rgba8(ndgi):
    rng = np.random.default_rng(30)
    bc4 = synth.bc4_planes(rng, 32, 16, 4)                # [4][8][4][8]
    got = ndgi.ndgi_bc4x4_to_rgba8(cu(bc4)).cpu().numpy()
    want = np.zeros((16, 32, 4), np.uint8)
    for by in range(4):
        for bx in range(8):
            for c in range(4):
                for p in range(16):
                    p35 = oracle.lib().om_bc4_p35(oracle._ptr(np.ascontiguousarray(bc4[by, bx, c])), p)
                    want[4 * by + p // 4, 4 * bx + p % 4, c] = int(np.floor(p35 / 35 + 0.5))
    assert np.array_equal(got, want)


# --------------------------------------------------------------------------
# The hybrid decoder over BC7 maps
# --------------------------------------------------------------------------

def bc7_hybrid(seed, uv=128, vol=32, hidden=64, mode=0):
    return synth.hybrid_model(seed, 128, 128, uv, uv, vol, vol, 12, 64, 24, 64, 24, hidden, address_mode=mode,
                              feat_format=1)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("mode", [0, 1])
def test_hybrid_bc7_points(ndgi, prec, mode):
    from test_gpu_hybrid import GATE
    m = bc7_hybrid(40 + mode, mode=mode)
    hm = ndgi.HybridModel.from_arrays(m)
    assert hm.feat_format == 1
    q = edge_queries(20_000, 41)
    if mode == 1:
        q[:2000, :2] = np.random.default_rng(42).uniform(-1.5, 2.5, (2000, 2)).astype(np.float32)
    got = ndgi.ndgi_hybrid_decode_points(hm, cu(q), prec).cpu().numpy()
    ref = oracle.hybrid_decode_points(m, q, precision=prec)
    err = rel_err(got, ref)
    print(f"hybrid BC7 points {prec} mode {mode}: max|err|/range = {err:.3e}")
    assert err <= GATE[prec]


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("layout", ["staged", "unstaged"])
def test_hybrid_bc7_pages_with_border(ndgi, prec, layout):
    """staged: F_uv at the lightmap's size (one tap per texel) and a 32^2 F3D (its footprint staged);
    unstaged: F_uv at half size (bilinear taps) and a 256^2 F3D (per-texel trilinear gather)."""
    from test_gpu_hybrid import GATE, page_err, ragged_requests
    uv, vol = (128, 32) if layout == "staged" else (64, 256)
    maps = [bc7_hybrid(140 + i, uv, vol, mode=i % 2) for i in range(3)]
    models = [ndgi.HybridModel.from_arrays(m) for m in maps]
    table = ndgi.HybridTable(models, prec)
    table.set_border(4)
    reqs = ragged_requests(141, 3, 6, 3)
    reqs["w"] = np.maximum(reqs["w"], 4)
    reqs["h"] = np.maximum(reqs["h"], 4)
    reqs["x0"] = np.minimum(reqs["x0"], 128 - reqs["w"])
    reqs["y0"] = np.minimum(reqs["y0"], 128 - reqs["h"])
    reqs["dst_x"] = (np.arange(6) % 3) * 144 + 4
    reqs["dst_y"] = (np.arange(6) // 3) * 144 + 4
    phys = torch.zeros((2 * 144, 3 * 144, 4), dtype=torch.float32, device="cuda")
    r, _ = ndgi.page_requests_to_device(reqs)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    ref = oracle.hybrid_decode_pages(maps, reqs, 3 * 144, 2 * 144, precision=prec, fill=0.0, border=4)
    padded = reqs.copy()
    padded["dst_x"] -= 4
    padded["dst_y"] -= 4
    padded["w"] += 8
    padded["h"] += 8
    err = page_err(phys.cpu().numpy(), ref, padded)
    print(f"hybrid BC7 pages {layout} {prec}: max|err|/page range = {err:.3e}")
    assert err <= GATE[prec]
    table.close()


def test_hybrid_bc7_bpp(ndgi):
    hm4 = ndgi.HybridModel.from_arrays(synth.hybrid_tile_model(150, "M.64"))
    hm7 = ndgi.HybridModel.from_arrays(bc7_hybrid(151))
    from paper_2604_12625_gb300 import _abi as A
    import ctypes as C
    L = A.lib()
    assert L.ndgi_model_bpp(C.byref(hm7.desc), 26, 0, 16) == L.ndgi_model_bpp(C.byref(hm7.desc), 26, 8, 16)
    assert L.ndgi_model_bpp(C.byref(hm4.desc), 26, 0, 16) == L.ndgi_model_bpp(C.byref(hm4.desc), 26, 16, 16)


def test_hybrid_bc7_pages_timeout_path(ndgi):
    """The BC7 instantiation of the tensor-core page kernel takes the same bounded timeout path (injected before
    any MMA), latches it in the table's word only, and the next frame decodes correctly."""
    from paper_2604_12625_gb300 import _abi as A
    from test_gpu_hybrid import GATE, page_err, ragged_requests
    s = synth.hybrid_tile_set(160, 2, "M.64", feat_format=1)
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, "fp16")
    table = ndgi.HybridTable(models, "fp16")
    reqs = ragged_requests(161, 2, 4, 2)
    r, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.zeros((2 * 128, 2 * 128, 4), dtype=torch.float32, device="cuda")
    ndgi.ndgi_hybrid_debug_inject(None, "fp16", table=table, flags=1)
    table.decode(r, len(reqs), phys)
    st, word = table.check()
    assert st == A.NDGI_ERR_TIMEOUT and word & 16
    ndgi.ndgi_hybrid_debug_inject(None, "fp16", table=table, flags=0)
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    maps = [synth.hybrid_tile_of(s, i) for i in range(2)]
    ref = oracle.hybrid_decode_pages(maps, reqs, 2 * 128, 2 * 128, precision="fp16", fill=0.0)
    assert page_err(phys.cpu().numpy(), ref, reqs) <= GATE["fp16"]
    table.close()


def test_hybrid_bc7_full_frame_sampled(ndgi):
    """The benchmark's BC7 frame (4096 M.64 tile models, whole-tile requests, RGBA16F) on sampled requests."""
    from test_gpu_hybrid import GATE
    s = synth.hybrid_tile_set(94, 4096, "M.64", feat_format=1)
    models = ndgi.HybridModel.from_set(s)
    ndgi.hybrid_prepare_set(models, "fp16")
    table = ndgi.HybridTable(models, "fp16")
    reqs = synth.hybrid_tile_requests(91, 4096, 4096, slots_x=64)
    r, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.zeros((8192, 8192, 4), dtype=torch.float16, device="cuda")
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    pick = np.random.default_rng(162).choice(len(reqs), 6, replace=False)
    used = sorted(set(int(reqs[i]["model"]) for i in pick))
    remap = {mi: k for k, mi in enumerate(used)}
    sub = reqs[pick].copy()
    sub["model"] = [remap[int(mi)] for mi in sub["model"]]
    ref = oracle.hybrid_decode_pages([synth.hybrid_tile_of(s, mi) for mi in used], sub, 8192, 8192,
                                     precision="fp16", fill=0.0)
    got = phys.float().cpu().numpy()
    for q in sub:
        sl = (slice(q["dst_y"], q["dst_y"] + 128), slice(q["dst_x"], q["dst_x"] + 128))
        a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        err = float(np.abs(a - b).max() / (b.max() - b.min()))
        # FP16 path gate plus the RGBA16F storage rounding of each value
        assert np.all(np.abs(a - b) <= GATE["fp16"] * (b.max() - b.min()) + np.abs(b) * 2.0 ** -11), err
    table.close()
    del phys
    torch.cuda.empty_cache()


@pytest.mark.parametrize("fmt_bc7", [False, True])
def test_hybrid_pages_rgba8_output(ndgi, fmt_bc7):
    """RGBA8 UNORM output (the paper's 8-bit, 4-channel physical texture): each byte is the FP16 decode's value
    clamped to [0, 1] and rounded to 8 bits, so it lies within the FP16 gate plus half a level of the oracle's
    value; A = 255; texels outside the requests stay untouched."""
    from test_gpu_hybrid import GATE, ragged_requests
    maps = [synth.hybrid_model(170 + i, 128, 128, 128, 128, 32, 32, 12, 64, 24, 64, 24, 64,
                               feat_format=1 if fmt_bc7 else 0) for i in range(2)]
    for m in maps:   # outputs mostly inside [0, 1]: scale the last layer down and centre it
        m["w3"] = (m["w3"] * 0.1).astype(np.float32)
        m["b3"] = np.full(3, 0.5, np.float32)
    models = [ndgi.HybridModel.from_arrays(m) for m in maps]
    table = ndgi.HybridTable(models, "fp16")
    reqs = ragged_requests(171, 2, 6, 3)
    r, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.full((2 * 128, 3 * 128, 4), 7, dtype=torch.uint8, device="cuda")
    table.decode(r, len(reqs), phys)
    assert table.check() == (0, 0)
    got = phys.cpu().numpy()
    ref = oracle.hybrid_decode_pages(maps, reqs, 3 * 128, 2 * 128, precision="fp16", fill=np.nan)
    inside = ~np.isnan(ref[..., 0])
    assert np.all(got[~inside] == 7)
    assert np.all(got[inside][:, 3] == 255)
    for q in reqs:
        sl = (slice(q["dst_y"], q["dst_y"] + q["h"]), slice(q["dst_x"], q["dst_x"] + q["w"]))
        b = ref[sl][..., :3]
        rng = max(float(b.max() - b.min()), 1e-3)
        a = got[sl][..., :3].astype(np.float64) / 255.0
        assert np.all(np.abs(a - np.clip(b, 0, 1)) <= GATE["fp16"] * rng + 0.5 / 255 + 1e-6)
    inside_vals = ref[inside][:, :3]
    assert 0.2 < np.mean((inside_vals > 0) & (inside_vals < 1))   # the test exercises the unclamped range
    table.close()
