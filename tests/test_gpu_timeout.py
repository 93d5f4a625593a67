"""The tensor-core kernels' timeout path, on the GPU, without a real stall.

A test hook makes a decode's lanes wait, with a short limit, for a barrier
phase that nothing completes, before any MMA is issued; the kernel then
unwinds along its real timeout path (the lanes stop at their next barrier,
tensor memory is freed) and latches the timeout in the caller's error word:
the prepared workspace's for point decodes, the plan's for page decodes.
Each check must report NDGI_ERR_TIMEOUT for that call only, leave other
workspaces' words clear, and the next normal call must decode correctly.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NDGI_OK, NDGI_ERR_TIMEOUT = 0, 5


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


def test_point_decode_timeout_is_per_workspace(ndgi):
    ma = ndgi.Model.from_arrays(synth.points_model_2048(2))
    mb = ndgi.Model.from_arrays(synth.model(3, 512, 512, 256, 256, 16, 24, 8, 64, temporal_dtype="f16"))
    q = torch.from_numpy(synth.random_queries(4, 100_000)).cuda()
    ref_a = ndgi.ndgi_decode_points(ma, q, "fp16")
    ref_b = ndgi.ndgi_decode_points(mb, q, "fp16")
    assert ndgi.ndgi_workspace_check(ma, "fp16") == (NDGI_OK, 0)
    ndgi.ndgi_debug_workspace_inject(ma, "fp16", 1)
    ndgi.ndgi_decode_points(ma, q, "fp16")            # takes the timeout path
    got_b = ndgi.ndgi_decode_points(mb, q, "fp16")    # another workspace: unaffected
    ndgi.ndgi_check()                                 # no CUDA error: the context is intact
    st, word = ndgi.ndgi_workspace_check(ma, "fp16")
    assert st == NDGI_ERR_TIMEOUT and word & 16
    assert ndgi.ndgi_workspace_check(ma, "fp16") == (NDGI_OK, 0)   # read clears it
    assert ndgi.ndgi_workspace_check(mb, "fp16") == (NDGI_OK, 0)
    assert torch.equal(got_b, ref_b)
    ndgi.ndgi_debug_workspace_inject(ma, "fp16", 0)
    again = ndgi.ndgi_decode_points(ma, q, "fp16")
    assert ndgi.ndgi_workspace_check(ma, "fp16") == (NDGI_OK, 0)
    assert torch.equal(again, ref_a)


@pytest.mark.parametrize("shape", [(1, 4, 1), (1, 8, 1), (1, 2, 2)])
def test_page_decode_timeout_is_per_plan(ndgi, shape):
    sizes = (256, 512)
    maps = synth.page_models(44, sizes=sizes, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    reqs = synth.ragged_page_requests(45, sizes, 12, slots_x=4, slot=128)
    r, n = ndgi.page_requests_to_device(reqs)
    phys = torch.zeros((512, 512, 4), dtype=torch.float32, device="cuda")
    other = torch.zeros_like(phys)
    plan = ndgi.PagesPlan(models, "fp16", 64, phys)
    plan2 = ndgi.PagesPlan(models, "fp16", 64, other)
    plan.set_shape(*shape)
    plan2.set_shape(*shape)
    plan.decode(r, n)
    assert plan.check() == (NDGI_OK, 0)
    ref = phys.clone()
    plan.set_debug(1)
    phys.zero_()
    plan.decode(r, n)                                 # takes the timeout path
    plan2.decode(r, n)                                # another plan: unaffected
    ndgi.ndgi_check()
    st, word = plan.check()
    assert st == NDGI_ERR_TIMEOUT and word == 16
    assert plan2.check() == (NDGI_OK, 0) and torch.equal(other, ref)
    plan.set_debug(0)
    phys.zero_()
    plan.decode(r, n)
    assert plan.check() == (NDGI_OK, 0)
    assert torch.equal(phys, ref)
    plan.close()
    plan2.close()
