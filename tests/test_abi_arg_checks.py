"""Host-side argument checks of the C ABI that guard device accesses needing
natural alignment: the 64-bit atomic total of ndgi_bc7_encode, the FP64 loss
logs and FP16 targets of the fits, the FP32 inputs and FP64 outputs of
ndgi_tile_metrics.  Each call here must be rejected with
NDGI_ERR_INVALID_ARG before any CUDA call, so the pointers are plain numbers
that are never dereferenced; the module skips itself wherever a GPU is
visible, so that such a number can never reach a kernel."""
import ctypes as C

import pytest

torch = pytest.importorskip("torch")
if torch.cuda.is_available():
    pytest.skip("host-only argument checks with fake device pointers", allow_module_level=True)

from paper_2604_12625_gb300 import _abi  # noqa: E402

P = 1 << 20   # a fake, 256-byte aligned device address (never dereferenced)
FIT_MSG = "targets must be 2-byte and loss_log 8-byte aligned"


def rejected(status, needle):
    assert status == _abi.NDGI_ERR_INVALID_ARG
    _, msg = _abi.last_error()
    assert needle in msg, msg


def cfg():
    return _abi.FitConfig(steps=1, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, freeze_steps=0,
                          loss_every=1, seed=1, relaxed=0, noise_alpha=0.0)


def test_bc7_encode_total_must_be_8_byte_aligned():
    L = _abi.lib()
    rejected(L.ndgi_bc7_encode(P, 4, 4, 2 * P, P + 4, None), "sq_err must be 8-byte aligned")


def test_tile_metrics_alignment():
    L = _abi.lib()
    rejected(L.ndgi_tile_metrics(P + 2, P, None, 1, 8, 8, 3, 8, P, P, None), "pred/ref must be 4-byte")
    rejected(L.ndgi_tile_metrics(P, P, None, 1, 8, 8, 3, 8, P + 4, P, None), "psnr/ssim 8-byte")
    rejected(L.ndgi_tile_metrics(P, P, None, 1, 8, 8, 3, 8, P, P + 4, None), "psnr/ssim 8-byte")


def test_encode_fit_targets_and_loss_log_alignment():
    L = _abi.lib()
    p = _abi.FitParams(lm_w=64, lm_h=64, feat_w=32, feat_h=32, cs=16, t_count=24, ct=8, hidden=64,
                       **{k: P for k in _abi.FIT_TENSORS}, address_mode=0, key_t=None)
    c = cfg()
    rejected(L.ndgi_encode_fit(C.byref(p), P + 1, C.byref(c), 0, P, 1 << 30, P, None), FIT_MSG)
    rejected(L.ndgi_encode_fit(C.byref(p), P, C.byref(c), 0, P, 1 << 30, P + 4, None), FIT_MSG)
    rejected(L.ndgi_encode_fit_batch(C.byref(p), 2, P, C.byref(c), 0, P, 1 << 30, P + 4, None), FIT_MSG)


def test_hybrid_encode_fit_targets_and_loss_log_alignment():
    L = _abi.lib()
    p = _abi.HybridFitParams(lm_w=128, lm_h=128, uv_w=128, uv_h=128, vol_w=32, vol_h=32, vol_t=12, ut_w=64,
                             ut_t=24, vt_h=64, vt_t=24, hidden=64, address_mode=0,
                             **{k: P for k in _abi.HFIT_TENSORS}, shared_w=0)
    c = cfg()
    rejected(L.ndgi_hybrid_encode_fit(C.byref(p), P + 1, 24, None, C.byref(c), 0, P, 1 << 30, P, None), FIT_MSG)
    rejected(L.ndgi_hybrid_encode_fit(C.byref(p), P, 24, None, C.byref(c), 0, P, 1 << 30, P + 4, None), FIT_MSG)
    rejected(L.ndgi_hybrid_encode_fit_batch(C.byref(p), 2, P, 24, None, C.byref(c), 0, P, 1 << 30, P + 4, None),
             FIT_MSG)


def test_batched_fits_reject_more_models_than_grid_rows():
    L = _abi.lib()
    p = _abi.FitParams(lm_w=64, lm_h=64, feat_w=32, feat_h=32, cs=16, t_count=24, ct=8, hidden=64,
                       **{k: P for k in _abi.FIT_TENSORS}, address_mode=0, key_t=None)
    c = cfg()
    for n in (0, 65536):
        rejected(L.ndgi_encode_fit_batch(C.byref(p), n, P, C.byref(c), 0, P, 1 << 30, P, None), "1..65535")
    h = _abi.HybridFitParams(lm_w=128, lm_h=128, uv_w=128, uv_h=128, vol_w=32, vol_h=32, vol_t=12, ut_w=64,
                             ut_t=24, vt_h=64, vt_t=24, hidden=64, address_mode=0,
                             **{k: P for k in _abi.HFIT_TENSORS}, shared_w=0)
    for n in (0, 65536):
        rejected(L.ndgi_hybrid_encode_fit_batch(C.byref(h), n, P, 24, None, C.byref(c), 0, P, 1 << 30, P, None),
                 "1..65535")
