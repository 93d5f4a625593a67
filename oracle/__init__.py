"""FP64 CPU oracle for the NDGI decode and fit (test infrastructure).

Only tests/, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never calls it, and it shares no code with that path: the
arithmetic lives in ``ndgi_oracle.c`` (plain C, FP64), this module only
marshals numpy arrays into it.

Reduced-precision parity is measured against the *stored* parameters: for an
FP16 or BF16 decode the MLP weights and biases are rounded to that format
(round to nearest even) and then evaluated exactly in FP64 here.  The FP8
(E4M3) page decode also quantises the activations at each layer input, with
the power-of-two scales described in ndgi_oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ndgi_oracle.c")
_LIB = os.path.join(_HERE, "libndgi_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the oracle with gcc (no fast-math, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Model(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("feat_w", C.c_int32), ("feat_h", C.c_int32),
                ("cs", C.c_int32), ("bc4", C.c_void_p), ("t_count", C.c_int32), ("ct", C.c_int32),
                ("temporal", C.c_void_p), ("hidden", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("address_mode", C.c_int32), ("key_t", C.c_void_p)]


class _PageReq(C.Structure):
    _fields_ = [("model", C.c_int32), ("x0", C.c_int32), ("y0", C.c_int32), ("w", C.c_int32),
                ("h", C.c_int32), ("t", C.c_float), ("dst_x", C.c_int32), ("dst_y", C.c_int32)]


class _FitParams(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("feat_w", C.c_int32), ("feat_h", C.c_int32),
                ("cs", C.c_int32), ("t_count", C.c_int32), ("ct", C.c_int32), ("hidden", C.c_int32),
                ("ea", C.c_void_p), ("eb", C.c_void_p), ("w", C.c_void_p), ("temporal", C.c_void_p),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("address_mode", C.c_int32), ("key_t", C.c_void_p)]


class _FitGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("ea", "eb", "w", "temporal", "w1", "b1", "w2", "b2", "w3", "b3")]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            vp, i32, i64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double
            L.om_bc4_p35.argtypes = [vp, C.c_int]
            L.om_bc4_p35.restype = C.c_int
            L.om_p35_value.argtypes = [C.c_int]
            L.om_p35_value.restype = f32
            L.om_features.argtypes = [vp, f64, f64, f64, vp, vp]
            L.om_features_batch.argtypes = [vp, vp, i64, vp, vp, C.c_int]
            L.om_mlp_batch.argtypes = [vp, vp, i64, vp]
            L.om_decode_points.argtypes = [vp, vp, i64, vp, C.c_int]
            L.om_decode_pages.argtypes = [vp, i32, vp, i32, vp, i64, i64, C.c_int]
            L.om_q255.argtypes = [f32]
            L.om_q7.argtypes = [f32]
            L.om_bc_pack.argtypes = [vp, vp, vp, i32, i32, i32, vp]
            L.om_fit_forward.argtypes = [vp, vp, i64, C.c_int, vp, vp]
            L.om_fit_loss.argtypes = [vp, vp, i64]
            L.om_fit_loss.restype = f64
            L.om_fit_backward.argtypes = [vp, vp, vp, i64, C.c_int, vp]
            L.om_fit_backward.restype = f64
            L.om_adam.argtypes = [vp, vp, vp, vp, i64, i32, f64, f64, f64, f64, i32]
            L.om_fit_draw.argtypes = [C.c_uint64, i64, i64, i64, i32, i32, vp, vp]
            L.om_temporal_weights.argtypes = [f64, i32, vp, vp, vp, vp]
            L.om_max_hidden.restype = C.c_int
            L.om_e4m3_batch.argtypes = [vp, i64, vp, vp]
            L.om_p2.argtypes = [f64]
            L.om_p2.restype = f64
            L.om_fp8_scales.argtypes = [vp, vp, vp]
            L.om_fp8_bias.argtypes = [vp, C.c_int, f64, vp, vp, vp]
            L.om_fp8_weights.argtypes = [vp, vp, vp, vp, vp]
            L.om_fp8_calibrate.argtypes = [vp, vp, i64, vp]
            L.om_decode_pages_fp8.argtypes = [vp, vp, vp, i32, vp, i64, C.c_int]
            L.om_gelu.argtypes = [f64]
            L.om_gelu.restype = f64
            L.om_hybrid_gamma.argtypes = [f64, vp]
            L.om_hybrid_decode_points.argtypes = [vp, vp, i64, vp, vp, C.c_int]
            L.om_hybrid_decode_pages.argtypes = [vp, i32, vp, i32, vp, i64, i64, i32, C.c_int]
            L.om_tile_metrics.argtypes = [vp, vp, vp, i32, i32, i32, i32, i32, vp, vp]
            L.om_hfit_forward.argtypes = [vp, vp, i64, C.c_int, vp, vp]
            L.om_hfit_backward.argtypes = [vp, vp, vp, vp, i64, C.c_int, vp]
            L.om_fit_noise.argtypes = [C.c_uint64, i64, i64, i64, f64, vp]
            L.om_hfit_backward.restype = f64
            L.om_bc7_decode_block.argtypes = [vp, vp]
            L.om_bc7_decode.argtypes = [vp, i32, i32, vp]
            L.om_bc7_candidate.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, vp]
            L.om_bc7_candidate.restype = i64
            L.om_bc7_encode_block.argtypes = [vp, vp]
            L.om_bc7_encode_block.restype = i64
            L.om_bc7_encode.argtypes = [vp, i32, i32, vp, C.c_int]
            L.om_bc7_encode.restype = i64
            L.om_bc7_subset.argtypes = [C.c_int, C.c_int, C.c_int]
            L.om_bc_sim7_rgba8.argtypes = [vp, vp, vp, i32, i32, vp]
            L.om_bc7_pack_sim.argtypes = [vp, vp, vp, i64, vp]
            L.om_bc7_anchor.argtypes = [C.c_int, C.c_int, C.c_int]
            L.om_splitmix64_next.argtypes = [C.c_uint64]
            L.om_splitmix64_next.restype = C.c_uint64
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------------
# Stored-parameter rounding (what a reduced-precision decode actually holds)
# --------------------------------------------------------------------------

def round_bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    b = x.view(np.uint32).astype(np.uint64)
    rounded = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    nan = np.isnan(x)
    out = rounded.astype(np.uint32).view(np.float32).copy()
    out[nan] = np.nan
    return out


def stored_weights(m, precision):
    """MLP weights/biases as the decode of `precision` stores them, in FP64."""
    keys = ("w1", "b1", "w2", "b2", "w3", "b3")
    if precision == "fp32":
        return {k: np.asarray(m[k], np.float32).astype(np.float64) for k in keys}
    if precision == "fp16":
        return {k: np.asarray(m[k], np.float32).astype(np.float16).astype(np.float64) for k in keys}
    if precision == "bf16":
        return {k: round_bf16(m[k]).astype(np.float64) for k in keys}
    raise ValueError(precision)


def _key_times(m):
    """Keyframe times of a model or fit dict (FP32 values as FP64), or None for uniform keyframes j/T."""
    k = m.get("key_t") if isinstance(m, dict) else None
    return None if k is None else _c(np.asarray(k, np.float32).astype(np.float64), np.float64)


class Model:
    """A decodable model (dict from synth.model) held in oracle form."""

    def __init__(self, m, precision="fp32"):
        self.src = m
        self.cs, self.ct, self.hidden = int(m["cs"]), int(m["ct"]), int(m["hidden"])
        assert self.hidden <= lib().om_max_hidden()
        self.bc4 = _c(m["bc4"], np.uint8)
        self.temporal = _c(np.asarray(m["temporal"]).astype(np.float64), np.float64)
        self.key_t = _key_times(m)
        w = stored_weights(m, precision)
        self.w = {k: _c(v, np.float64) for k, v in w.items()}
        self.s = _Model(int(m["lm_w"]), int(m["lm_h"]), int(m["feat_w"]), int(m["feat_h"]), self.cs,
                        _ptr(self.bc4), int(m["t_count"]), self.ct, _ptr(self.temporal), self.hidden,
                        _ptr(self.w["w1"]), _ptr(self.w["b1"]), _ptr(self.w["w2"]), _ptr(self.w["b2"]),
                        _ptr(self.w["w3"]), _ptr(self.w["b3"]), int(m.get("address_mode", 0)),
                        _ptr(self.key_t))


class _Hybrid(C.Structure):
    _fields_ = [("lm_w", C.c_int32), ("lm_h", C.c_int32), ("uv_w", C.c_int32), ("uv_h", C.c_int32),
                ("uv_bc4", C.c_void_p), ("vol_w", C.c_int32), ("vol_h", C.c_int32), ("vol_t", C.c_int32),
                ("vol_bc4", C.c_void_p), ("ut_w", C.c_int32), ("ut_t", C.c_int32), ("ut", C.c_void_p),
                ("vt_h", C.c_int32), ("vt_t", C.c_int32), ("vt", C.c_void_p), ("hidden", C.c_int32),
                ("w1", C.c_void_p), ("b1", C.c_void_p), ("w2", C.c_void_p), ("b2", C.c_void_p),
                ("w3", C.c_void_p), ("b3", C.c_void_p), ("address_mode", C.c_int32), ("feat_format", C.c_int32)]


class HybridModel:
    """A hybrid-feature-map model (dict from synth.hybrid_model) held in oracle form."""

    def __init__(self, m, precision="fp32"):
        self.src = m
        self.hidden = int(m["hidden"])
        assert self.hidden <= lib().om_max_hidden()
        self.fmt = int(m.get("feat_format", 0))
        uv, vol = ("uv_bc7", "vol_bc7") if self.fmt == 1 else ("uv_bc4", "vol_bc4")
        self.arr = {k: _c(m[src], np.uint8) for k, src in (("uv_bc4", uv), ("vol_bc4", vol), ("ut", "ut"),
                                                           ("vt", "vt"))}
        w = stored_weights(m, precision)
        self.w = {k: _c(v, np.float64) for k, v in w.items()}
        vol_t, vol_h, vol_w = (int(d) for d in m["vol_shape"])
        self.s = _Hybrid(int(m["lm_w"]), int(m["lm_h"]), int(m["uv_w"]), int(m["uv_h"]), _ptr(self.arr["uv_bc4"]),
                         vol_w, vol_h, vol_t, _ptr(self.arr["vol_bc4"]),
                         int(m["ut"].shape[1]), int(m["ut"].shape[0]), _ptr(self.arr["ut"]),
                         int(m["vt"].shape[1]), int(m["vt"].shape[0]), _ptr(self.arr["vt"]), self.hidden,
                         _ptr(self.w["w1"]), _ptr(self.w["b1"]), _ptr(self.w["w2"]), _ptr(self.w["b2"]),
                         _ptr(self.w["w3"]), _ptr(self.w["b3"]), int(m.get("address_mode", 0)), self.fmt)


def _hybrid(m, precision="fp32"):
    return m if isinstance(m, HybridModel) else HybridModel(m, precision)


def gelu(x):
    """GELU x Phi(x) of each value (FP64)."""
    f = lib().om_gelu
    return np.array([f(float(v)) for v in np.asarray(x, np.float64).reshape(-1)]).reshape(np.shape(x))


def hybrid_gamma(t):
    """The time code gamma(t) of Eq. 4, [4]."""
    g = np.zeros(4, np.float64)
    lib().om_hybrid_gamma(float(t), _ptr(g))
    return g


def hybrid_decode_points(m, uvt, precision="fp32", nthreads=None, features=False):
    """FP64 RGB [n][3] of the hybrid decoder at each (u, v, t); with features=True also the inputs [n][16]."""
    M = _hybrid(m, precision)
    q = _c(uvt, np.float32).reshape(-1, 3)
    y = np.zeros((q.shape[0], 3), np.float64)
    x = np.zeros((q.shape[0], 16), np.float64) if features else None
    lib().om_hybrid_decode_points(C.byref(M.s), _ptr(q), q.shape[0], _ptr(y), _ptr(x), nthreads or nthreads_default())
    return (y, x) if features else y


def hybrid_decode_pages(models, reqs, phys_w, phys_h, precision="fp32", nthreads=None, fill=np.nan, border=0):
    """FP64 RGBA physical texture [phys_h][phys_w][4] of hybrid-model page requests (with a mirrored tile border
    of `border` texels per edge); untouched texels = fill."""
    r = np.ascontiguousarray(reqs)
    out = np.full((phys_h, phys_w, 4), fill, np.float64)
    Ms = [_hybrid(m, precision) for m in models]
    arr = (_Hybrid * len(Ms))(*[M.s for M in Ms])
    lib().om_hybrid_decode_pages(arr, len(Ms), r.ctypes.data_as(C.c_void_p), len(r), _ptr(out), phys_w, phys_h,
                                 int(border), nthreads or nthreads_default())
    return out


def _model(m, precision="fp32"):
    return m if isinstance(m, Model) else Model(m, precision)


def nthreads_default():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def bc4_p35(block, p):
    """Palette numerator (value * 8925) of texel p of one 8-byte BC4 block."""
    b = _c(np.frombuffer(bytes(block), dtype=np.uint8), np.uint8)
    return int(lib().om_bc4_p35(_ptr(b), int(p)))


def p35_value(p35):
    return float(lib().om_p35_value(int(p35)))


def features(m, uvt, nthreads=None):
    """x = [v_s, v_t] [n][cs+ct] and tap numerators [n][4][cs]."""
    M = _model(m)
    q = _c(uvt, np.float32).reshape(-1, 3)
    n = q.shape[0]
    x = np.zeros((n, M.cs + M.ct), np.float64)
    p = np.zeros((n, 4, M.cs), np.int32)
    lib().om_features_batch(C.byref(M.s), _ptr(q), n, _ptr(x), _ptr(p), nthreads or nthreads_default())
    return x, p


def mlp(m, x, precision="fp32"):
    M = _model(m, precision)
    x = _c(x, np.float64)
    y = np.zeros((x.shape[0], 3), np.float64)
    lib().om_mlp_batch(C.byref(M.s), _ptr(x), x.shape[0], _ptr(y))
    return y


def decode_points(m, uvt, precision="fp32", nthreads=None):
    """FP64 RGB [n][3] of the decode at each (u, v, t)."""
    M = _model(m, precision)
    q = _c(uvt, np.float32).reshape(-1, 3)
    y = np.zeros((q.shape[0], 3), np.float64)
    lib().om_decode_points(C.byref(M.s), _ptr(q), q.shape[0], _ptr(y), nthreads or nthreads_default())
    return y


def decode_pages(models, reqs, phys_w, phys_h, precision="fp32", nthreads=None, fill=np.nan, act_max=None):
    """FP64 RGBA physical texture [phys_h][phys_w][4]; untouched texels = fill.

    precision "fp8": the E4M3 decode with scales from act_max ([n_models][3]
    calibration maxima; see fp8_scales), evaluated on the FP32 master weights.
    """
    r = np.ascontiguousarray(reqs)
    out = np.full((phys_h, phys_w, 4), fill, np.float64)
    if precision == "fp8":
        Ms = [_model(m, "fp32") for m in models]
        arr = (_Model * len(Ms))(*[M.s for M in Ms])
        am = _c(np.asarray(act_max, np.float64).reshape(len(Ms), 3), np.float64)
        lib().om_decode_pages_fp8(arr, _ptr(am), r.ctypes.data_as(C.c_void_p), len(r), _ptr(out), phys_w,
                                  nthreads or nthreads_default())
        return out
    Ms = [_model(m, precision) for m in models]
    arr = (_Model * len(Ms))(*[M.s for M in Ms])
    lib().om_decode_pages(arr, len(Ms), r.ctypes.data_as(C.c_void_p), len(r), _ptr(out), phys_w, phys_h,
                          nthreads or nthreads_default())
    return out


# --------------------------------------------------------------------------
# FP8 E4M3 (see ndgi_oracle.c for the scale reading)
# --------------------------------------------------------------------------

def e4m3(x):
    """Round to E4M3 (nearest, ties to even, saturating at +-448): (values, codes)."""
    x = _c(np.asarray(x, np.float64).reshape(-1), np.float64)
    y = np.zeros_like(x)
    codes = np.zeros(x.shape, np.int32)
    lib().om_e4m3_batch(_ptr(x), x.size, _ptr(y), _ptr(codes))
    return y, codes


def p2(y):
    """Smallest power of two P with y <= 448 P."""
    return float(lib().om_p2(float(y)))


def fp8_scales(m, act_max):
    """{a1, s1, a2, s2, a3, s3, out} of a model for calibration maxima (m1, m2, m3)."""
    M = _model(m, "fp32")
    am = _c(np.asarray(act_max, np.float64).reshape(3), np.float64)
    sc = np.zeros(7, np.float64)
    lib().om_fp8_scales(C.byref(M.s), _ptr(am), _ptr(sc))
    return dict(zip(("a1", "s1", "a2", "s2", "a3", "s3", "out"), sc.tolist()))


def fp8_weights(m, act_max):
    """Stored FP8 weights s_l e4m3(W_l / s_l) as FP64 arrays shaped like w1, w2, w3."""
    M = _model(m, "fp32")
    am = _c(np.asarray(act_max, np.float64).reshape(3), np.float64)
    sc = np.zeros(7, np.float64)
    lib().om_fp8_scales(C.byref(M.s), _ptr(am), _ptr(sc))
    out = {k: np.zeros(np.asarray(m[k]).shape, np.float64) for k in ("w1", "w2", "w3")}
    lib().om_fp8_weights(C.byref(M.s), _ptr(sc), _ptr(out["w1"]), _ptr(out["w2"]), _ptr(out["w3"]))
    return out


def fp8_bias(b, u):
    """Three-term E4M3 bias in units u: (terms [n][3], v, stored values)."""
    b = _c(np.asarray(b, np.float64).reshape(-1), np.float64)
    terms = np.zeros((b.size, 3), np.float64)
    stored = np.zeros(b.size, np.float64)
    v = C.c_double(0.0)
    lib().om_fp8_bias(_ptr(b), b.size, float(u), _ptr(terms), C.byref(v), _ptr(stored))
    return terms, v.value, stored


def fp8_calibrate(m, uvt):
    """Calibration maxima (max|x|, max relu(z1), max relu(z2)) of the FP64 decode at the queries."""
    M = _model(m, "fp32")
    q = _c(uvt, np.float32).reshape(-1, 3)
    am = np.zeros(3, np.float64)
    lib().om_fp8_calibrate(C.byref(M.s), _ptr(q), q.shape[0], _ptr(am))
    return am


def q255(e):
    return int(lib().om_q255(float(np.float32(e))))


def q7(w):
    return int(lib().om_q7(float(np.float32(w))))


def bc_pack(ea, eb, w):
    """BC4 blocks [bh][bw][cs][8] from endpoints [bh][bw][cs] and weights [bh][bw][cs][16]."""
    ea, eb, w = _c(ea, np.float32), _c(eb, np.float32), _c(w, np.float32)
    bh, bw, cs = ea.shape
    out = np.zeros((bh, bw, cs, 8), np.uint8)
    lib().om_bc_pack(_ptr(ea), _ptr(eb), _ptr(w), cs, bw * 4, bh * 4, _ptr(out))
    return out


# --------------------------------------------------------------------------
# Fit
# --------------------------------------------------------------------------

FIT_KEYS = ("ea", "eb", "w", "temporal", "w1", "b1", "w2", "b2", "w3", "b3")


class FitParams:
    def __init__(self, p, lm_w, lm_h):
        self.a = {k: _c(p[k], np.float32) for k in FIT_KEYS}
        bh, bw, cs = self.a["ea"].shape
        T, ct = self.a["temporal"].shape
        H = self.a["w2"].shape[0]
        self.dims = dict(lm_w=lm_w, lm_h=lm_h, feat_w=bw * 4, feat_h=bh * 4, cs=cs, t_count=T, ct=ct, hidden=H)
        self.key_t = _key_times(p)
        self.s = _FitParams(lm_w, lm_h, bw * 4, bh * 4, cs, T, ct, H,
                            *[_ptr(self.a[k]) for k in FIT_KEYS], int(p.get("address_mode", 0)), _ptr(self.key_t))


def fit_forward(params, uvt, lm_w, lm_h, relaxed=False, want_signs=False):
    """Straight-through (or relaxed) forward at the queries uvt [n][3] float32: rgb [n][3]."""
    P = params if isinstance(params, FitParams) else FitParams(params, lm_w, lm_h)
    s = _c(uvt, np.float32).reshape(-1, 3)
    y = np.zeros((s.shape[0], 3), np.float64)
    signs = np.zeros((s.shape[0], 2 * P.dims["hidden"]), np.uint8) if want_signs else None
    lib().om_fit_forward(C.byref(P.s), _ptr(s), s.shape[0], int(relaxed), _ptr(y), _ptr(signs))
    return (y, signs) if want_signs else y


def fit_loss(rgb, target):
    rgb, target = _c(rgb, np.float64), _c(target, np.float64)
    return float(lib().om_fit_loss(_ptr(rgb), _ptr(target), rgb.shape[0]))


def fit_backward(params, uvt, target, lm_w, lm_h, relaxed=False):
    """(loss, grads) at the queries uvt [n][3] float32, grads a dict of FP64 arrays shaped like the params."""
    P = params if isinstance(params, FitParams) else FitParams(params, lm_w, lm_h)
    s = _c(uvt, np.float32).reshape(-1, 3)
    t = _c(target, np.float64).reshape(-1, 3)
    g = {k: np.zeros(P.a[k].shape, np.float64) for k in FIT_KEYS}
    G = _FitGrads(*[_ptr(g[k]) for k in FIT_KEYS])
    loss = lib().om_fit_backward(C.byref(P.s), _ptr(s), _ptr(t), s.shape[0], int(relaxed), C.byref(G))
    return float(loss), g


def adam(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, project=False):
    """In-place Adam on float32 p with float64 moments m, v."""
    assert p.dtype == np.float32 and p.flags.c_contiguous
    g = _c(g, np.float64)
    lib().om_adam(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.size, int(step), lr, beta1, beta2, eps, int(project))


def fit_draw(seed, step, n, lm_w, lm_h, first=0):
    """The fit loop's samples of one step: (texel int32 [n][2], uvt float32 [n][3])."""
    texel = np.zeros((n, 2), np.int32)
    uvt = np.zeros((n, 3), np.float32)
    lib().om_fit_draw(C.c_uint64(seed), step, first, n, lm_w, lm_h, _ptr(texel), _ptr(uvt))
    return texel, uvt


def temporal_weights(t, t_count, key_t=None):
    """(j0, j1, alpha) of time t: keyframes at j / t_count or at the times key_t, periodic (the decode's
    temporal lerp)."""
    j0, j1, a = C.c_int32(0), C.c_int32(0), C.c_double(0.0)
    k = None if key_t is None else _c(np.asarray(key_t, np.float32).astype(np.float64), np.float64)
    lib().om_temporal_weights(float(t), int(t_count), _ptr(k), C.byref(j0), C.byref(j1), C.byref(a))
    return j0.value, j1.value, a.value


def fit_targets_at(targets, texel, uvt, key_t=None):
    """Target of each fit sample: the keyframe targets [T][H][W][3] at its texel, interpolated linearly in t
    between the two keyframes around it (the lightmap at time t is the interpolation of its keyframes,
    Eq. 2), in FP64."""
    T = targets.shape[0]
    out = np.zeros((texel.shape[0], 3), np.float64)
    for i in range(texel.shape[0]):
        j0, j1, a = temporal_weights(float(uvt[i, 2]), T, key_t)
        ix, iy = int(texel[i, 0]), int(texel[i, 1])
        out[i] = (1.0 - a) * targets[j0, iy, ix].astype(np.float64) + a * targets[j1, iy, ix].astype(np.float64)
    return out


def tile_metrics(pred, ref, mask=None, tile=128):
    """Per-tile (PSNR, SSIM) of lightmaps [n][h][w][c] (or [h][w][c]) under an optional mask [n][h][w]."""
    p = _c(pred, np.float64)
    q = _c(ref, np.float64)
    if p.ndim == 3:
        p, q = p[None], q[None]
        mask = None if mask is None else np.asarray(mask)[None]
    n, h, w, c = p.shape
    m = None if mask is None else _c(np.asarray(mask) != 0, np.uint8)
    ty, tx = (h + tile - 1) // tile, (w + tile - 1) // tile
    ps = np.zeros((n, ty, tx), np.float64)
    ss = np.zeros((n, ty, tx), np.float64)
    lib().om_tile_metrics(_ptr(p), _ptr(q), _ptr(m), n, h, w, c, tile, _ptr(ps), _ptr(ss))
    return ps, ss


# --------------------------------------------------------------------------
# Fit of the hybrid decoder
# --------------------------------------------------------------------------

HFIT_KEYS = ("uv_ea", "uv_eb", "uv_wt", "vol_ea", "vol_eb", "vol_wt", "ut", "vt", "w1", "b1", "w2", "b2", "w3", "b3")


class _HFitParams(C.Structure):
    _fields_ = [(k, C.c_int32) for k in ("lm_w", "lm_h", "uv_w", "uv_h", "vol_w", "vol_h", "vol_t", "ut_w", "ut_t",
                                         "vt_h", "vt_t", "hidden", "address_mode")] + \
               [(k, C.c_void_p) for k in HFIT_KEYS] + [("shared_w", C.c_int32)]


class _HFitGrads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in HFIT_KEYS]


class HFitParams:
    """Hybrid-fit parameters (dict from synth.hybrid_fit_init) in oracle form.  A weight tensor uv_wt of shape
    [uv_h/4][uv_w/4][16] (vol_wt [vol_t][..][16]) selects Eq. 7's weight per texel shared by the channels."""

    def __init__(self, p):
        self.a = {k: _c(p[k], np.float32) for k in HFIT_KEYS}
        vt_, vh, vw = (int(d) for d in p["vol_shape"])
        ut_t, ut_w, _ = self.a["ut"].shape
        vt_t, vt_h, _ = self.a["vt"].shape
        self.s = _HFitParams(int(p["lm_w"]), int(p["lm_h"]), int(p["uv_w"]), int(p["uv_h"]), vw, vh, vt_, ut_w, ut_t,
                             vt_h, vt_t, int(p["hidden"]), int(p.get("address_mode", 0)),
                             *[_ptr(self.a[k]) for k in HFIT_KEYS], int(self.a["uv_wt"].ndim == 3))


def fit_noise(seed, step, n, alpha, first=0):
    """The training-time quantisation noise [n][12] of the hybrid fit's samples first.. of one step."""
    out = np.zeros((n, 12), np.float64)
    lib().om_fit_noise(C.c_uint64(seed), int(step), int(first), int(n), float(alpha), _ptr(out))
    return out


def hfit_forward(p, uvt, relaxed=False, noise=None):
    """rgb [n][3] of the hybrid fit's straight-through (or relaxed) forward at queries uvt [n][3] (with the
    inputs' additive noise [n][12] when given)."""
    P = p if isinstance(p, HFitParams) else HFitParams(p)
    q = _c(uvt, np.float32).reshape(-1, 3)
    y = np.zeros((q.shape[0], 3), np.float64)
    nz = None if noise is None else _c(noise, np.float64)
    lib().om_hfit_forward(C.byref(P.s), _ptr(q), q.shape[0], int(relaxed), _ptr(nz), _ptr(y))
    return y


def hfit_backward(p, uvt, target, relaxed=False, noise=None):
    """(loss, gradients dict) of the MSE at queries uvt against target [n][3] (FP64)."""
    P = p if isinstance(p, HFitParams) else HFitParams(p)
    q = _c(uvt, np.float32).reshape(-1, 3)
    tg = _c(target, np.float64).reshape(-1, 3)
    g = {k: np.zeros(P.a[k].shape, np.float64) for k in HFIT_KEYS}
    G = _HFitGrads(*[_ptr(g[k]) for k in HFIT_KEYS])
    nz = None if noise is None else _c(noise, np.float64)
    loss = lib().om_hfit_backward(C.byref(P.s), _ptr(q), _ptr(tg), _ptr(nz), q.shape[0], int(relaxed), C.byref(G))
    return loss, g


# --------------------------------------------------------------------------
# BC7 blocks (the paper's storage format for F_uv and the F3D slices)
# --------------------------------------------------------------------------

def bc7_decode_block(blk):
    """RGBA8 [16][4] of one 16-byte BC7 block (texel p = 4 row + col)."""
    b = _c(np.asarray(blk, np.uint8).reshape(16), np.uint8)
    out = np.zeros((16, 4), np.uint8)
    lib().om_bc7_decode_block(_ptr(b), _ptr(out))
    return out


def bc7_decode(blocks, w, h):
    """RGBA8 image [h][w][4] of BC7 blocks [h/4][w/4][16]."""
    b = _c(blocks, np.uint8)
    out = np.zeros((h, w, 4), np.uint8)
    lib().om_bc7_decode(_ptr(b), int(w), int(h), _ptr(out))
    return out


def bc7_candidate(x, mode, part=0, rot=0, isb=0):
    """(block, squared error) of one encoder candidate for the block x [16][4] uint8."""
    xb = _c(np.asarray(x, np.uint8).reshape(16, 4), np.uint8)
    blk = np.zeros(16, np.uint8)
    err = lib().om_bc7_candidate(_ptr(xb), int(mode), int(part), int(rot), int(isb), _ptr(blk))
    return blk, int(err)


def bc7_encode_block(x):
    """(block, squared error) of the encoder on x [16][4] uint8."""
    xb = _c(np.asarray(x, np.uint8).reshape(16, 4), np.uint8)
    blk = np.zeros(16, np.uint8)
    err = lib().om_bc7_encode_block(_ptr(xb), _ptr(blk))
    return blk, int(err)


def bc7_encode(rgba, nthreads=None):
    """(blocks [h/4][w/4][16], total squared error) of the encoder on an RGBA8 image [h][w][4]."""
    x = _c(rgba, np.uint8)
    h, w, _ = x.shape
    out = np.zeros((h // 4, w // 4, 16), np.uint8)
    err = lib().om_bc7_encode(_ptr(x), int(w), int(h), _ptr(out), nthreads or nthreads_default())
    return out, int(err)


def bc7_subset(ns, part, p):
    return int(lib().om_bc7_subset(int(ns), int(part), int(p)))


def bc7_anchor(ns, part, s):
    return int(lib().om_bc7_anchor(int(ns), int(part), int(s)))


def bc_sim7_rgba8(ea, eb, w):
    """RGBA8 [h][w][4] of a shared-weight BC simulation: ea, eb [h/4][w/4][4], w [h/4][w/4][16] (float32)."""
    a, b, ww = _c(ea, np.float32), _c(eb, np.float32), _c(w, np.float32)
    bw = a.shape[-2]
    bh = a.size // (bw * 4)                 # leading axes (F3D slices) stacked along the height
    out = np.zeros((bh * 4, bw * 4, 4), np.uint8)
    lib().om_bc_sim7_rgba8(_ptr(a), _ptr(b), _ptr(ww), bw * 4, bh * 4, _ptr(out))
    return out


def bc7_pack_sim(ea, eb, w):
    """Exact BC7 mode-6 blocks [..][16] of a shared-weight BC simulation (ea, eb [..][4], w [..][16])."""
    a, b, ww = _c(ea, np.float32), _c(eb, np.float32), _c(w, np.float32)
    nb = a.size // 4
    out = np.zeros(a.shape[:-1] + (16,), np.uint8)
    lib().om_bc7_pack_sim(_ptr(a), _ptr(b), _ptr(ww), nb, _ptr(out))
    return out
