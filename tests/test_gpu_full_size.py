"""GPU parity of the FP16 tensor-core page decode at the full sizes of the
two page workloads, against the FP64 oracle on the stored FP16 parameters.

- The batched frame: all 8 lightmaps (2 each of 512^2, 1024^2, 2048^2 and
  4096^2, BC4 features at half resolution x 16 planes, temporal 24 x 8 FP16,
  MLP 24-64-64-3), the 4096 Zipf(1.1) requests of the benchmark frame plus
  the corner pages of both 4096^2 maps, decoded in one launch.
- The scale shape: a 16384^2 lightmap with 8192^2 x 16 BC4 planes (512 MiB),
  temporal 48 x 16 FP16, MLP 32-64-64-3, decoded over a 4096^2 region at one
  t plus the map's four corner pages at their own t.

The oracle takes sampled pages one by one (every corner page included); the
gate is the FP16 path's 2e-3 of each page's range, on an RGBA32F texture so
no storage rounding enters.  Both tensor-core page kernels (4 x 1 and the
warp-specialised 8 x 1) run and must agree bit for bit.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GATE = 2e-3


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def page_err(phys, ref, reqs):
    worst = 0.0
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = phys[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        worst = max(worst, float(np.abs(a - b).max() / max(b.max() - b.min(), 1e-6)))
    return worst


def corner_pages(mi, size, t0, first_slot, slots_x, page=128):
    out = np.zeros(4, dtype=synth.PAGE_REQ_DTYPE)
    for i, (cx, cy) in enumerate(((0, 0), (1, 0), (0, 1), (1, 1))):
        s = first_slot + i
        out[i] = (mi, cx * (size - page), cy * (size - page), page, page, np.float32((t0 + 0.21 * i) % 1.0),
                  (s % slots_x) * page, (s // slots_x) * page)
    return out


def decode_both_shapes(ndgi, plan, phys, reqs):
    r, n = ndgi.page_requests_to_device(reqs)
    out = []
    for shape in ((1, 4, 1), (1, 8, 1)):
        plan.set_shape(*shape)
        phys.zero_()
        plan.decode(r, n)
        assert plan.check() == (0, 0)
        ndgi.ndgi_check()
        out.append(phys.cpu().numpy())
    assert np.array_equal(out[0], out[1])
    return out[1]


def test_full_batched_frame_fp16(ndgi):
    maps = synth.page_models(4)
    models = [ndgi.Model.from_arrays(m) for m in maps]
    slots_x = 64
    zipf = synth.zipf_page_requests(4, synth.PAGE_LIGHTMAP_SIZES, 4096, page=128, slots_x=slots_x)
    corners = np.concatenate([corner_pages(mi, 4096, 0.1 * mi, 4096 + 4 * k, slots_x)
                              for k, mi in enumerate((6, 7))])
    reqs = np.concatenate([zipf, corners])
    phys_h = ((len(reqs) + slots_x - 1) // slots_x) * 128
    phys = torch.zeros((phys_h, slots_x * 128, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp16", len(reqs), phys)
    got = decode_both_shapes(ndgi, plan, phys, reqs)
    plan.close()
    on_big = np.flatnonzero(zipf["model"] >= 6)
    pick = np.random.default_rng(8).choice(len(zipf), 40, replace=False)
    sub = np.concatenate([zipf[pick], zipf[on_big[:8]], corners])
    ref = oracle.decode_pages(maps, sub, slots_x * 128, phys_h, precision="fp16", fill=0.0)
    err = page_err(got, ref, sub)
    print(f"C4 frame, {len(sub)} sampled pages: max |err| / page range = {err:.3e}")
    assert err <= GATE
    assert np.all(got[..., 3][: (len(reqs) // slots_x) * 128] == 1.0)


def test_scale_shape_region_fp16(ndgi):
    m = synth.model(5, 16384, 16384, 8192, 8192, 16, 48, 16, 64, temporal_dtype="f16")
    model = ndgi.Model.from_arrays(m)
    side, slots_x = 32, 33                       # a 4096^2 region as 32 x 32 pages, then the corners
    reqs = np.zeros(side * side, dtype=synth.PAGE_REQ_DTYPE)
    ox, oy = 6144, 2048
    for i in range(side * side):
        px, py = i % side, i // side
        reqs[i] = (0, ox + px * 128, oy + py * 128, 128, 128, np.float32(0.37), px * 128, py * 128)
    corners = corner_pages(0, 16384, 0.55, 0, slots_x)
    corners["dst_x"] = side * 128
    corners["dst_y"] = np.arange(4) * 128
    reqs = np.concatenate([reqs, corners])
    phys = torch.zeros((side * 128, slots_x * 128, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan([model], "fp16", len(reqs), phys)
    got = decode_both_shapes(ndgi, plan, phys, reqs)
    plan.close()
    pick = np.random.default_rng(9).choice(side * side, 16, replace=False)
    sub = np.concatenate([reqs[pick], corners])
    ref = oracle.decode_pages([m], sub, slots_x * 128, side * 128, precision="fp16", fill=0.0)
    err = page_err(got, ref, sub)
    print(f"scale shape, {len(sub)} sampled pages: max |err| / page range = {err:.3e}")
    assert err <= GATE
    assert np.all(got[:, : side * 128, 3] == 1.0) and np.all(got[:512, side * 128:, 3] == 1.0)
