"""The C-ABI library builds, loads on the CPU (no GPU calls) and exports every
entry point that include/ndgi.h declares; the binding's signature table
covers exactly that set."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "ndgi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return set(re.findall(r"^[A-Za-z_][\w\s\*]*?\b(ndgi_\w+)\s*\(", src, flags=re.M))


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_12625_gb300 import build
    return build.build()


def test_header_declares_the_core_calls():
    syms = declared_symbols()
    for name in ("ndgi_decode_points", "ndgi_decode_pages", "ndgi_bc_pack", "ndgi_encode_fit",
                 "ndgi_fit_forward", "ndgi_fit_backward", "ndgi_prepare", "ndgi_pages_plan_create"):
        assert name in syms


def test_library_exports_every_declared_symbol(libpath):
    L = ctypes.CDLL(libpath)
    missing = [s for s in sorted(declared_symbols()) if not hasattr(L, s)]
    assert not missing, missing


def test_binding_signature_table_matches_header(libpath):
    from paper_2604_12625_gb300 import _abi
    names = {n for n, _, _ in _abi.SIGNATURES}
    assert names == declared_symbols()


def test_host_side_argument_errors_without_gpu(libpath):
    # Host-side validation runs before any CUDA call: NULL model / plan.
    from paper_2604_12625_gb300 import _abi
    L = _abi.lib()
    assert L.ndgi_decode_points(None, 0, None, None, 0, None, None) == _abi.NDGI_ERR_INVALID_ARG
    assert L.ndgi_pages_plan_destroy(None) == _abi.NDGI_OK
    assert L.ndgi_bc_pack(None, None, None, 1, 4, 4, None, None) == _abi.NDGI_ERR_INVALID_ARG
    st, msg = _abi.last_error()
    assert st == _abi.NDGI_ERR_INVALID_ARG and "ndgi_bc_pack" in msg
    assert L.ndgi_version().startswith(b"ndgi")
    # host-buffer pipe: sizes and refusals before any CUDA call
    assert L.ndgi_host_pipe_staging_size(0) == 0
    assert L.ndgi_host_pipe_staging_size(1) == 3 * 2 * 256
    assert L.ndgi_host_pipe_staging_size(1 << 20) == 3 * 2 * (12 << 20)
    h = ctypes.c_void_p()
    assert L.ndgi_host_pipe_create(16, None, 0, ctypes.byref(h)) == _abi.NDGI_ERR_INVALID_ARG and not h.value
    assert L.ndgi_host_pipe_create(0, None, 0, ctypes.byref(h)) == _abi.NDGI_ERR_INVALID_ARG
    assert L.ndgi_host_pipe_destroy(None) == _abi.NDGI_OK
    assert L.ndgi_decode_points_host(None, None, 0, None, None, 1, None, None) == _abi.NDGI_ERR_INVALID_ARG
