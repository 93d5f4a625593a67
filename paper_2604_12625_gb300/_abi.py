"""ctypes view of include/ndgi.h (argument marshalling only).

The library is the in-tree libndgi.so built by ``build.py``.  Importing this
module fails loudly if it is missing: there is no CPU or eager fallback.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libndgi.so")

NDGI_OK, NDGI_ERR_INVALID_ARG, NDGI_ERR_UNSUPPORTED, NDGI_ERR_CUDA, NDGI_ERR_OOM, NDGI_ERR_TIMEOUT, \
    NDGI_ERR_DEVICE_CHECK = range(7)
NDGI_FP32, NDGI_FP16, NDGI_BF16, NDGI_FP8_E4M3 = range(4)
NDGI_RGBA32F, NDGI_RGBA16F, NDGI_RGBA8 = 0, 1, 2
PRECISIONS = {"fp32": NDGI_FP32, "fp16": NDGI_FP16, "bf16": NDGI_BF16, "fp8": NDGI_FP8_E4M3}
STATUS_NAMES = {0: "NDGI_OK", 1: "NDGI_ERR_INVALID_ARG", 2: "NDGI_ERR_UNSUPPORTED", 3: "NDGI_ERR_CUDA",
                4: "NDGI_ERR_OOM", 5: "NDGI_ERR_TIMEOUT", 6: "NDGI_ERR_DEVICE_CHECK"}


class ModelDesc(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("feat_w", C.c_int32), ("feat_h", C.c_int32),
                ("cs", C.c_int32), ("bc4", C.c_void_p), ("t_count", C.c_int32), ("ct", C.c_int32),
                ("temporal", C.c_void_p), ("temporal_dtype", C.c_int32), ("hidden", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("address_mode", C.c_int32), ("key_t", C.c_void_p)]


class PageReq(C.Structure):
    _fields_ = [("model", C.c_int32), ("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32),
                ("h", C.c_int32), ("t", C.c_float), ("dst_x", C.c_int32), ("dst_y", C.c_int32)]


NDGI_FEAT_BC4X4, NDGI_FEAT_BC7 = 0, 1


class HybridDesc(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("uv_w", C.c_int32), ("uv_h", C.c_int32),
                ("uv_bc4", C.c_void_p), ("vol_w", C.c_int32), ("vol_h", C.c_int32), ("vol_t", C.c_int32),
                ("vol_bc4", C.c_void_p), ("ut_w", C.c_int32), ("ut_t", C.c_int32), ("ut", C.c_void_p),
                ("vt_h", C.c_int32), ("vt_t", C.c_int32), ("vt", C.c_void_p), ("hidden", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("address_mode", C.c_int32), ("feat_format", C.c_int32)]


HFIT_TENSORS = ("uv_ea", "uv_eb", "uv_wt", "vol_ea", "vol_eb", "vol_wt", "ut", "vt", "w1", "b1", "w2", "b2", "w3",
                "b3")


class HybridFitParams(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("lm_w", "lm_h", "uv_w", "uv_h", "vol_w", "vol_h", "vol_t", "ut_w", "ut_t",
                                         "vt_h", "vt_t", "hidden", "address_mode")] + \
               [(k, C.c_void_p) for k in HFIT_TENSORS] + [("shared_w", C.c_int32)]


class HybridFitGrads(C.Structure):
    _fields_ = [("g", C.c_void_p * 14)]


FIT_TENSORS = ("ea", "eb", "w", "temporal", "w1", "b1", "w2", "b2", "w3", "b3")


class FitParams(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("feat_w", C.c_int32), ("feat_h", C.c_int32),
                ("cs", C.c_int32), ("t_count", C.c_int32), ("ct", C.c_int32), ("hidden", C.c_int32)] + \
               [(k, C.c_void_p) for k in FIT_TENSORS] + [("address_mode", C.c_int32), ("key_t", C.c_void_p)]


class FitGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in FIT_TENSORS]


class FitConfig(C.Structure):
    _fields_ = [("steps", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("freeze_steps", C.c_int32), ("loss_every", C.c_int32),
                ("seed", C.c_uint64), ("relaxed", C.c_int32), ("noise_alpha", C.c_float)]


# (name, restype, argtypes) of every exported entry point in include/ndgi.h
_vp, _i32, _i64, _sz = C.c_void_p, C.c_int32, C.c_int64, C.c_size_t
SIGNATURES = [
    ("ndgi_version", C.c_char_p, []),
    ("ndgi_last_error", C.c_int, [C.c_char_p, _sz]),
    ("ndgi_check", C.c_int, [_vp]),
    ("ndgi_workspace_check", C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    ("ndgi_debug_workspace_inject", C.c_int, [_vp, C.c_int, _vp, _i32, _vp]),
    ("ndgi_prepare_workspace_size", _sz, [_vp, C.c_int]),
    ("ndgi_prepare", C.c_int, [_vp, C.c_int, _vp, _sz, _vp]),
    ("ndgi_calibrate_fp8", C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    ("ndgi_prepare_fp8", C.c_int, [_vp, _vp, _vp, _sz, _vp]),
    ("ndgi_fp8_unpack", C.c_int, [_vp, _vp, _vp, _sz, _vp]),
    ("ndgi_decode_points", C.c_int, [_vp, C.c_int, _vp, _vp, _i64, _vp, _vp]),
    ("ndgi_decode_points_path", C.c_int32, [_vp, C.c_int, _i64]),
    ("ndgi_host_pipe_staging_size", _sz, [_i64]),
    ("ndgi_host_pipe_create", C.c_int, [_i64, _vp, _sz, _vp]),
    ("ndgi_decode_points_host", C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _i64, _vp, _vp]),
    ("ndgi_host_pipe_destroy", C.c_int, [_vp]),
    ("ndgi_debug_features", C.c_int, [_vp, _vp, _i64, _vp, _vp, _vp]),
    ("ndgi_debug_features_tc", C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
    ("ndgi_debug_features_cache", C.c_int, [_vp, _vp, _vp, _i64, _vp, _vp]),
    ("ndgi_pages_plan_create", C.c_int, [_vp, _vp, _i32, C.c_int, _i32, _i32, _vp, _i64, _i64, _vp]),
    ("ndgi_decode_pages", C.c_int, [_vp, _vp, _vp, _vp]),
    ("ndgi_pages_autotune", C.c_int, [_vp, _vp, _vp, _i32, _vp]),
    ("ndgi_pages_check", C.c_int, [_vp, _vp, _vp]),
    ("ndgi_pages_plan_destroy", C.c_int, [_vp]),
    ("ndgi_pages_plan_info", C.c_int, [_vp, _vp]),
    ("ndgi_pages_plan_set_shape", C.c_int, [_vp, _i32, _i32, _i32]),
    ("ndgi_pages_plan_set_debug", C.c_int, [_vp, _i32]),
    ("ndgi_pages_fp8_dump_size", _sz, [_vp]),
    ("ndgi_pages_plan_set_fp8_dump", C.c_int, [_vp, _i32, _vp]),
    ("ndgi_decode_pages_static", C.c_int, [_vp, _i32, _vp, _vp, _i32, _i32, _vp, _i64, _i64, _vp, _vp]),
    ("ndgi_bc_pack", C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _vp]),
    ("ndgi_bc7_encode", C.c_int, [_vp, _i32, _i32, _vp, _vp, _vp]),
    ("ndgi_bc7_decode", C.c_int, [_vp, _i32, _i32, _vp, _vp]),
    ("ndgi_bc4x4_to_rgba8", C.c_int, [_vp, _i32, _i32, _vp, _vp]),
    ("ndgi_debug_bc7_hw_decode", C.c_int, [_vp, _i32, _i32, _vp, _vp]),
    ("ndgi_bc_sim7_to_rgba8", C.c_int, [_vp, _vp, _vp, _i32, _i32, _vp, _vp]),
    ("ndgi_bc7_pack_sim", C.c_int, [_vp, _vp, _vp, C.c_int64, _vp, _vp]),
    ("ndgi_fit_forward", C.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("ndgi_fit_backward", C.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp]),
    ("ndgi_encode_fit_workspace_size", _sz, [_vp, _vp]),
    ("ndgi_encode_fit", C.c_int, [_vp, _vp, _vp, _i32, _vp, _sz, _vp, _vp]),
    ("ndgi_encode_fit_batch_workspace_size", _sz, [_vp, _i32, _vp]),
    ("ndgi_encode_fit_batch", C.c_int, [_vp, _i32, _vp, _vp, _i32, _vp, _sz, _vp, _vp]),
    ("ndgi_hybrid_workspace_size", _sz, [_vp, C.c_int]),
    ("ndgi_hybrid_prepare", C.c_int, [_vp, C.c_int, _vp, _vp]),
    ("ndgi_hybrid_decode_points", C.c_int, [_vp, C.c_int, _vp, _vp, _i64, _vp, _vp]),
    ("ndgi_hybrid_workspace_check", C.c_int, [_vp, C.c_int, _vp, _vp, _vp]),
    ("ndgi_hybrid_debug_inject", C.c_int, [_vp, C.c_int, _vp, _vp, _i32, _vp]),
    ("ndgi_hybrid_table_create", C.c_int, [_vp, _vp, _i32, C.c_int, _vp]),
    ("ndgi_hybrid_table_destroy", C.c_int, [_vp]),
    ("ndgi_hybrid_decode_pages", C.c_int, [_vp, _vp, _i32, _vp, _i64, _i64, C.c_int, _vp]),
    ("ndgi_hybrid_table_check", C.c_int, [_vp, _vp, _vp]),
    ("ndgi_hybrid_table_set_border", C.c_int, [_vp, _i32]),
    ("ndgi_debug_gelu", C.c_int, [_vp, _i64, _vp, _i32, _vp]),
    ("ndgi_model_bpp", C.c_double, [_vp, _i32, _i32, _i32]),
    ("ndgi_tile_metrics", C.c_int, [_vp, _vp, _vp, _i32, _i32, _i32, _i32, _i32, _vp, _vp, _vp]),
    ("ndgi_hybrid_fit_forward", C.c_int, [_vp, _vp, _i64, _i32, _vp, _vp]),
    ("ndgi_hybrid_fit_backward", C.c_int, [_vp, _vp, _i64, _i32, _vp, _vp, _vp]),
    ("ndgi_hybrid_encode_fit_workspace_size", _sz, [_vp, _vp]),
    ("ndgi_hybrid_encode_fit", C.c_int, [_vp, _vp, _i32, _vp, _vp, _i32, _vp, _sz, _vp, _vp]),
    ("ndgi_hybrid_encode_fit_batch_workspace_size", C.c_size_t, [_vp, _i32, _vp]),
    ("ndgi_hybrid_encode_fit_batch", C.c_int, [_vp, _i32, _vp, _i32, _vp, _vp, _i32, _vp, C.c_size_t, _vp, _vp]),
]

_lib = None


class NdgiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """The loaded libndgi.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libndgi.so is not built ({LIB_PATH}); run paper_2604_12625_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error():
    buf = C.create_string_buffer(1024)
    st = lib().ndgi_last_error(buf, len(buf))
    return st, buf.value.decode(errors="replace")


def check(status):
    if status != NDGI_OK:
        _, msg = last_error()
        raise NdgiError(status, msg)
    return status
