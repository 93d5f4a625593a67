"""GPU checks of the host-buffer point decode (ndgi_decode_points_host).

The pipe only moves data: each chunk is decoded by ndgi_decode_points on the
device, so its results must equal a device decode of the same queries bit
for bit, whatever the chunking (ragged last chunk, chunks that cycle the
three staging buffers, one call after another on the same pipe, pinned or
pageable host memory).  A sample is also checked against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth
from _gpu import rel_err

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ndgi():
    import paper_2604_12625_gb300 as m
    assert torch.cuda.is_available()
    return m


@pytest.fixture(scope="module")
def model_and_queries(ndgi):
    m = synth.model(91, 512, 512, 256, 256, 16, 24, 8, 64, temporal_dtype="f16")
    return m, ndgi.Model.from_arrays(m)


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
def test_host_pipe_matches_device_decode(ndgi, model_and_queries, prec):
    m, model = model_and_queries
    pipe = ndgi.HostPipe(chunk=4096)
    for seed, n, pinned in ((1, 1, True), (2, 1000, True), (3, 4096 * 7 + 17, True), (4, 4096 * 3, False),
                            (5, 50_000, True)):
        q = synth.random_queries(seed, n)
        q_host = torch.from_numpy(q)
        if pinned:
            q_host = q_host.pin_memory()
        got = pipe.decode_points(model, q_host, prec)
        torch.cuda.synchronize()
        ndgi.ndgi_check()
        ref = ndgi.ndgi_decode_points(model, torch.from_numpy(q).cuda(), prec).cpu()
        assert torch.equal(got, ref), (seed, n)
    pipe.close()


def test_host_pipe_back_to_back_calls_and_oracle(ndgi, model_and_queries):
    m, model = model_and_queries
    pipe = ndgi.HostPipe(chunk=1000)
    qa = torch.from_numpy(synth.random_queries(11, 9_999)).pin_memory()
    qb = torch.from_numpy(synth.random_queries(12, 5_001)).pin_memory()
    a = pipe.decode_points(model, qa, "fp16")   # no synchronisation between the two calls
    b = pipe.decode_points(model, qb, "fp16")
    torch.cuda.synchronize()
    ndgi.ndgi_check()
    assert torch.equal(a, ndgi.ndgi_decode_points(model, qa.cuda(), "fp16").cpu())
    assert torch.equal(b, ndgi.ndgi_decode_points(model, qb.cuda(), "fp16").cpu())
    idx = np.arange(0, 5_001, 7)
    ref = oracle.decode_points(m, qb.numpy()[idx], precision="fp16")
    assert rel_err(b.numpy()[idx], ref) <= 2e-3
    empty = pipe.decode_points(model, torch.empty((0, 3), dtype=torch.float32), "fp16")
    assert empty.shape == (0, 3)
    pipe.close()


def test_host_pipe_argument_errors(ndgi, model_and_queries):
    from paper_2604_12625_gb300 import _abi
    m, model = model_and_queries
    pipe = ndgi.HostPipe(chunk=64)
    q = torch.from_numpy(synth.random_queries(13, 10))
    L = _abi.lib()
    assert L.ndgi_decode_points_host(pipe.handle, None, 0, None, q.data_ptr(), 10, None, None) != _abi.NDGI_OK
    out = torch.empty((10, 3), dtype=torch.float32)
    assert L.ndgi_decode_points_host(pipe.handle, None, 0, None, q.data_ptr(), 10, out.data_ptr(),
                                     None) == _abi.NDGI_ERR_INVALID_ARG   # NULL model
    with pytest.raises(ValueError):
        pipe.decode_points(model, q.cuda(), "fp32")   # device tensor where a host one is needed
    pipe.close()
