"""GPU parity of the batched page decode (Sec. 3.5 / supplement S3) against the
FP64 oracle: ragged request sizes 1..128, duplicate pages, a zero-request
frame, graph replay with a changed request list, and requests rejected by the
device-side checks.  Error per page is measured against that page's range
(the per-tile dynamic range of supplement S4.2)."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


SIZES = (256, 256, 512, 1024)


@pytest.fixture(scope="module")
def maps():
    return synth.page_models(41, sizes=SIZES, temporal_dtype="f16")


def per_page_err(phys, ref, reqs):
    worst = 0.0
    for r in reqs:
        sl = (slice(r["dst_y"], r["dst_y"] + r["h"]), slice(r["dst_x"], r["dst_x"] + r["w"]))
        a, b = phys[sl][..., :3].astype(np.float64), ref[sl][..., :3]
        rng = max(b.max() - b.min(), 1e-6)
        worst = max(worst, float(np.abs(a - b).max() / rng))
        assert np.all(phys[sl][..., 3] == 1.0)
    return worst


def run_plan(ndgi, maps, reqs, precision, dtype, phys_side=1024):
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.full((phys_side, phys_side, 4), float("nan"), dtype=dtype, device="cuda")
    plan = ndgi.PagesPlan(models, precision, 4096, phys)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.decode(r, n)
    st, err = plan.check()
    assert st == 0 and err == 0
    return plan, phys, models


def test_pages_fp32_ragged(ndgi, maps):
    reqs = synth.ragged_page_requests(5, SIZES, 40, slots_x=8, slot=128)
    plan, phys, _ = run_plan(ndgi, maps, reqs, "fp32", torch.float32)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024)
    assert per_page_err(phys.cpu().numpy(), ref, reqs) <= 1e-5
    untouched = np.isnan(ref[..., 0])
    assert np.all(np.isnan(phys.cpu().numpy()[..., 0][untouched]))
    plan.close()


def test_pages_duplicates_and_replay(ndgi, maps):
    reqs = synth.zipf_page_requests(6, SIZES, 48, page=128, slots_x=8)
    assert len({(r["model"], r["x0"], r["y0"]) for r in reqs}) < len(reqs)   # duplicates present
    plan, phys, _ = run_plan(ndgi, maps, reqs, "fp32", torch.float32)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024)
    assert per_page_err(phys.cpu().numpy(), ref, reqs) <= 1e-5
    # replay the same graph with a different request list written into the same buffers
    r, n = ndgi.page_requests_to_device(reqs)
    reqs2 = synth.ragged_page_requests(7, SIZES, 30, slots_x=8, slot=128)
    r2 = torch.from_numpy(np.ascontiguousarray(reqs2).view(np.int32).reshape(-1, 8).copy()).cuda()
    r[: len(reqs2)].copy_(r2)
    n.fill_(len(reqs2))
    phys.fill_(float("nan"))
    plan.decode(r, n)
    ref2 = oracle.decode_pages(maps, reqs2, 1024, 1024)
    assert per_page_err(phys.cpu().numpy(), ref2, reqs2) <= 1e-5
    # zero-request frame leaves the texture untouched
    phys.fill_(-7.0)
    n.fill_(0)
    plan.decode(r, n)
    torch.cuda.synchronize()
    assert torch.all(phys == -7.0)
    plan.close()


def test_pages_rgba16f(ndgi, maps):
    reqs = synth.ragged_page_requests(8, SIZES, 20, slots_x=8, slot=128)
    plan, phys, _ = run_plan(ndgi, maps, reqs, "fp32", torch.float16)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024)
    got = phys.float().cpu().numpy()
    # FP16 storage rounds each value once: |err| <= 2^-11 |value|
    for rq in reqs:
        sl = (slice(rq["dst_y"], rq["dst_y"] + rq["h"]), slice(rq["dst_x"], rq["dst_x"] + rq["w"]))
        a, b = got[sl][..., :3], ref[sl][..., :3]
        assert np.all(np.abs(a - b) <= 2.0 ** -11 * np.abs(b) + 1e-6)
    plan.close()


def test_pages_device_checks(ndgi, maps):
    good = synth.ragged_page_requests(9, SIZES, 4, slots_x=8, slot=128)
    bad = good.copy()
    bad[1]["model"] = 99                 # no such model
    bad[2]["x0"] = SIZES[bad[2]["model"]]  # source outside the lightmap
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.zeros((1024, 1024, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp32", 16, phys)
    r, n = ndgi.page_requests_to_device(bad)
    plan.decode(r, n)
    st, err = plan.check()
    assert st == 6 and err != 0
    # the valid requests were still decoded
    ref = oracle.decode_pages(maps, bad[[0, 3]], 1024, 1024)
    assert per_page_err(phys.cpu().numpy(), ref, bad[[0, 3]]) <= 1e-5
    # request count above the plan's capacity is latched too
    n.fill_(17)
    plan.decode(r, n)
    st, err = plan.check()
    assert st == 6
    st, err = plan.check()
    assert st == 0 and err == 0
    plan.close()


def test_pages_autotune_keeps_results(ndgi, maps):
    reqs = synth.zipf_page_requests(10, SIZES, 64, page=128, slots_x=8)
    models = [ndgi.Model.from_arrays(m) for m in maps]
    phys = torch.zeros((1024, 1024, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp32", 64, phys)
    r, n = ndgi.page_requests_to_device(reqs)
    plan.autotune(r, n, len(reqs))
    phys.zero_()
    plan.decode(r, n)
    ref = oracle.decode_pages(maps, reqs, 1024, 1024)
    assert per_page_err(phys.cpu().numpy(), ref, reqs) <= 1e-5
    plan.close()
