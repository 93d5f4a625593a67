"""The allocation-free page decode (ndgi_decode_pages_static).

It exists for callers that cannot call cudaMalloc (fixed arenas, real-time
frame loops): its state lives in a static device array of the library.  The
test calls it through the C ABI twice in a row, with different request
lists, and checks each result against the plan-based page decode (the
existing entry point) within the FP32 tolerance of the other page tests.
This file is named to be collected last; it passes alone or after the rest.
"""
import ctypes as C

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SIZES = (256, 512)


def test_static_scratch_page_decode_matches_plan():
    import paper_2604_12625_gb300 as ndgi
    from paper_2604_12625_gb300 import _abi as A
    assert torch.cuda.is_available()
    maps = synth.page_models(77, sizes=SIZES, cs=16, t_count=24, ct=8, hidden=64, temporal_dtype="f16")
    models = [ndgi.Model.from_arrays(m) for m in maps]
    descs = (A.ModelDesc * len(models))(*[m.desc for m in models])
    err = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    plan_phys = torch.zeros((512, 512, 4), dtype=torch.float32, device="cuda")
    plan = ndgi.PagesPlan(models, "fp32", 64, plan_phys)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((3, 4)):          # two calls in a row, different requests
        reqs = synth.ragged_page_requests(seed, SIZES, 12, slots_x=4, slot=128)
        r, n = ndgi.page_requests_to_device(reqs)
        phys = torch.zeros((512, 512, 4), dtype=torch.float32, device="cuda")
        st = A.lib().ndgi_decode_pages_static(descs, len(models), C.c_void_p(r.data_ptr()),
                                              C.c_void_p(n.data_ptr()), 64, A.NDGI_RGBA32F,
                                              C.c_void_p(phys.data_ptr()), 512, 512, C.c_void_p(err.data_ptr()),
                                              stream)
        assert st == A.NDGI_OK, A.last_error()
        plan_phys.zero_()
        plan.decode(r, n)
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        got, ref = phys.cpu().numpy(), plan_phys.cpu().numpy()
        rng = float(ref[..., :3].max() - ref[..., :3].min())
        assert np.max(np.abs(got - ref)) <= 1e-5 * rng, call
        assert np.count_nonzero(got[..., 3]) == int(sum(q["w"] * q["h"] for q in reqs))
    # the call allocates nothing: device free memory is unchanged around a call
    # (the first calls above have already loaded the kernels' code)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = A.lib().ndgi_decode_pages_static(descs, len(models), C.c_void_p(r.data_ptr()), C.c_void_p(n.data_ptr()),
                                          64, A.NDGI_RGBA32F, C.c_void_p(phys.data_ptr()), 512, 512,
                                          C.c_void_p(err.data_ptr()), stream)
    assert st == A.NDGI_OK, A.last_error()
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    # a request naming a model the call was not given is skipped and latched
    # (bit 1 of the error word); the next call starts from a cleared word
    bad = reqs.copy()
    bad["model"][0] = len(models)
    rb, nb = ndgi.page_requests_to_device(bad)
    for rq, nq, want in ((rb, nb, 2), (r, n, 0)):
        st = A.lib().ndgi_decode_pages_static(descs, len(models), C.c_void_p(rq.data_ptr()),
                                              C.c_void_p(nq.data_ptr()), 64, A.NDGI_RGBA32F,
                                              C.c_void_p(phys.data_ptr()), 512, 512, C.c_void_p(err.data_ptr()),
                                              stream)
        assert st == A.NDGI_OK, A.last_error()
        torch.cuda.synchronize()
        assert int(err.item()) == want
    # RGBA16F output with no error word requested: the FP32 result rounded to FP16
    phys16 = torch.zeros((512, 512, 4), dtype=torch.float16, device="cuda")
    st = A.lib().ndgi_decode_pages_static(descs, len(models), C.c_void_p(r.data_ptr()), C.c_void_p(n.data_ptr()),
                                          64, A.NDGI_RGBA16F, C.c_void_p(phys16.data_ptr()), 512, 512, None, stream)
    assert st == A.NDGI_OK, A.last_error()
    torch.cuda.synchronize()
    assert torch.equal(phys16, phys.to(torch.float16))
    plan.close()
    # more models than the static maximum is rejected with a clear error
    many = (A.ModelDesc * 65)(*([models[0].desc] * 65))
    st = A.lib().ndgi_decode_pages_static(many, 65, C.c_void_p(r.data_ptr()), C.c_void_p(n.data_ptr()), 64,
                                          A.NDGI_RGBA32F, C.c_void_p(phys.data_ptr()), 512, 512, None, stream)
    assert st == A.NDGI_ERR_INVALID_ARG and "static maximum" in A.last_error()[1]
