"""NDGI random-access neural lightmap decode for NVIDIA GB300 (sm_103a).

The compute path is libndgi.so (hand-written CUDA, C ABI in include/ndgi.h);
this package only marshals torch tensors into it.  The first call into the
library raises if it was not built (``paper_2604_12625_gb300.build.build()``):
there is no CPU fallback.
"""
from ._abi import NdgiError, lib  # noqa: F401
from .api import (  # noqa: F401
    FitState, HostPipe, Model, NdgiDecodeFunction, PagesPlan, fit_config, ndgi_decode_fit, ndgi_bc_pack, ndgi_check, ndgi_debug_features,
    ndgi_decode_pages, ndgi_decode_pages_static, ndgi_decode_points, ndgi_encode_fit, ndgi_encode_fit_workspace_size, ndgi_fit_backward,
    ndgi_fit_forward, ndgi_prepare, ndgi_prepare_workspace_size, ndgi_version, page_requests_to_device,
    ndgi_calibrate_fp8, ndgi_prepare_fp8, ndgi_fp8_unpack, ndgi_debug_features_tc, ndgi_workspace_check,
    ndgi_debug_workspace_inject, ndgi_debug_features_cache, ndgi_decode_points_path, HybridModel, HybridTable,
    ndgi_hybrid_workspace_size, ndgi_hybrid_prepare, ndgi_hybrid_decode_points, ndgi_hybrid_workspace_check,
    ndgi_hybrid_debug_inject, ndgi_model_bpp, hybrid_prepare_set, ndgi_debug_gelu,
    ndgi_tile_metrics, ndgi_bc7_encode, ndgi_bc7_decode, ndgi_bc4x4_to_rgba8, ndgi_debug_bc7_hw_decode, ndgi_bc_sim7_to_rgba8,
    ndgi_bc7_pack_sim,
    FitBatch, ndgi_encode_fit_batch, HybridFitState, ndgi_hybrid_fit_forward,
    ndgi_hybrid_fit_backward, ndgi_hybrid_encode_fit,
    HybridFitBatch, ndgi_hybrid_encode_fit_batch)

