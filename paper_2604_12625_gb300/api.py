"""Python binding of libndgi.so: the entry points of include/ndgi.h under the
same names, taking torch CUDA tensors.  Argument marshalling only; every
step of the decode and the fit runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _abi as A
from ._abi import check, lib


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _need(t, dtype, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA tensor of {dtype}")
    return t


def _prec(p):
    return A.PRECISIONS[p] if isinstance(p, str) else int(p)


# ---------------------------------------------------------------------------
# Model
# ---------------------------------------------------------------------------
class Model:
    """A decodable model resident on the GPU plus its ndgi_model_desc.

    Tensors: bc4 uint8 [feat_h/4][feat_w/4][cs][8], temporal [T][ct] float32 or
    float16, MLP weights float32 [in][out].  Prepared tensor-core workspaces
    are kept per precision in ``self.ws``.
    """

    def __init__(self, lm_w, lm_h, bc4, temporal, w1, b1, w2, b2, w3, b3, address_mode=0, key_t=None):
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.bc4 = _need(bc4, torch.uint8, "bc4")
        bh, bw, cs, eight = bc4.shape
        assert eight == 8
        self.feat_w, self.feat_h, self.cs = bw * 4, bh * 4, cs
        if temporal.dtype not in (torch.float32, torch.float16):
            raise ValueError("temporal must be float32 or float16")
        self.temporal = _need(temporal, temporal.dtype, "temporal")
        self.t_count, self.ct = temporal.shape
        self.w = {k: _need(v, torch.float32, k) for k, v in
                  dict(w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3).items()}
        self.hidden = w2.shape[0]
        self.address_mode = int(address_mode)
        self.key_t = None if key_t is None else _need(key_t, torch.float32, "key_t")
        self.desc = A.ModelDesc(self.lm_w, self.lm_h, self.feat_w, self.feat_h, self.cs, self.bc4.data_ptr(),
                                self.t_count, self.ct, self.temporal.data_ptr(),
                                A.NDGI_FP16 if temporal.dtype == torch.float16 else A.NDGI_FP32, self.hidden,
                                *[self.w[k].data_ptr() for k in ("w1", "b1", "w2", "b2", "w3", "b3")],
                                self.address_mode, _p(self.key_t))
        self.ws = {}

    @classmethod
    def from_arrays(cls, m, device="cuda"):
        """From a dict of numpy arrays (the layout of synth.model)."""
        def t(a):
            return torch.from_numpy(np.ascontiguousarray(a)).to(device)
        key_t = m.get("key_t")
        return cls(m["lm_w"], m["lm_h"], t(m["bc4"]), t(m["temporal"]), t(m["w1"]), t(m["b1"]), t(m["w2"]),
                   t(m["b2"]), t(m["w3"]), t(m["b3"]), m.get("address_mode", 0),
                   None if key_t is None else t(np.asarray(key_t, np.float32)))

    def workspace(self, precision):
        precision = _prec(precision)
        if precision == A.NDGI_FP32:
            return None
        if precision not in self.ws:
            if precision == A.NDGI_FP8_E4M3:
                raise ValueError("the FP8 workspace needs calibration maxima: call ndgi_prepare_fp8 first")
            self.ws[precision] = ndgi_prepare(self, precision)
        return self.ws[precision]


def ndgi_workspace_check(model, precision, stream=None):
    """(status, error word) of the point decodes that used the model's prepared workspace; clears the word."""
    err = C.c_int32(0)
    st = lib().ndgi_workspace_check(C.byref(model.desc), _prec(precision), _p(model.workspace(precision)),
                                    C.byref(err), _stream(stream))
    return st, err.value


def ndgi_debug_workspace_inject(model, precision, flags, stream=None):
    """Test hook: flags = 1 makes point decodes with this workspace take their timeout path; 0 = normal."""
    check(lib().ndgi_debug_workspace_inject(C.byref(model.desc), _prec(precision), _p(model.workspace(precision)),
                                            int(flags), _stream(stream)))


def ndgi_version():
    return lib().ndgi_version().decode()


def ndgi_check(stream=None):
    return check(lib().ndgi_check(_stream(stream)))


def ndgi_prepare_workspace_size(model, precision):
    return int(lib().ndgi_prepare_workspace_size(C.byref(model.desc), _prec(precision)))


def ndgi_prepare(model, precision, ws=None, stream=None):
    """Packs the MLP for a tensor-core decode; returns the workspace tensor."""
    n = ndgi_prepare_workspace_size(model, precision)
    if ws is None:
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=model.bc4.device)
    check(lib().ndgi_prepare(C.byref(model.desc), _prec(precision), _p(ws), ws.numel(), _stream(stream)))
    return ws


def ndgi_calibrate_fp8(model, uvt, act_max=None, stream=None):
    """Maxima (|layer-1 input|, relu(z1), relu(z2)) of the FP32 decode at the queries: float32 [3] on the GPU."""
    uvt = _need(uvt, torch.float32, "uvt")
    if act_max is None:
        act_max = torch.empty(3, dtype=torch.float32, device=uvt.device)
    _need(act_max, torch.float32, "act_max")
    check(lib().ndgi_calibrate_fp8(C.byref(model.desc), _p(uvt), uvt.shape[0], _p(act_max), _stream(stream)))
    return act_max


def ndgi_prepare_fp8(model, act_max, ws=None, stream=None):
    """Packs the FP8 (E4M3) page-decode image from calibration maxima (3 values, any host or CUDA array);
    the workspace is kept as the model's FP8 workspace and returned."""
    am = torch.as_tensor(act_max, dtype=torch.float32).detach().cpu().numpy().reshape(3)
    arr = (C.c_float * 3)(*[float(x) for x in am])
    n = ndgi_prepare_workspace_size(model, A.NDGI_FP8_E4M3)
    if ws is None:
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=model.bc4.device)
    check(lib().ndgi_prepare_fp8(C.byref(model.desc), arr, _p(ws), ws.numel(), _stream(stream)))
    model.ws[A.NDGI_FP8_E4M3] = ws
    return ws


def ndgi_fp8_unpack(model, ws=None):
    """The stored FP8 parameters as float32 numpy arrays: scales, w1, w2, w3, b2, b3."""
    ws = ws if ws is not None else model.workspace(A.NDGI_FP8_E4M3)
    need = C.c_size_t(0)
    check(lib().ndgi_fp8_unpack(C.byref(model.desc), _p(ws), None, 0, C.byref(need)))
    out = np.zeros(need.value, np.float32)
    check(lib().ndgi_fp8_unpack(C.byref(model.desc), _p(ws), out.ctypes.data_as(C.c_void_p), out.size, None))
    H, cin = model.hidden, model.cs + model.ct
    head = out[:16]
    o = 16
    parts = {}
    for k, shape in (("w1", (cin, H)), ("w2", (H, H)), ("w3", (H, 3)), ("b2", (H,)), ("b3", (3,))):
        size = int(np.prod(shape))
        parts[k] = out[o:o + size].reshape(shape)
        o += size
    parts["scales"] = dict(zip(("a1", "a2", "a3", "out", "s1", "s2", "s3", "v2", "v3", "status"), head[:10].tolist()))
    return parts


def ndgi_decode_points(model, uvt, precision="fp32", ws=None, out=None, stream=None):
    """rgb [n][3] float32 of the decode at each (u, v, t) row of uvt."""
    uvt = _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=uvt.device)
    _need(out, torch.float32, "out")
    pr = _prec(precision)
    if ws is None and pr != A.NDGI_FP32:
        ws = model.workspace(pr)
    check(lib().ndgi_decode_points(C.byref(model.desc), pr, _p(ws), _p(uvt), n, _p(out), _stream(stream)))
    return out


class HostPipe:
    """ndgi_host_pipe_* wrapper: point decode from host (CPU) tensors with the
    copies in, the decode and the copies out overlapped chunk by chunk.  The
    pipe's device staging is a torch allocation made here, at creation."""

    def __init__(self, chunk=1 << 20, device=None):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.chunk = int(chunk)
        nbytes = int(lib().ndgi_host_pipe_staging_size(self.chunk))
        if nbytes == 0:
            raise ValueError("chunk must be >= 1")
        self.staging = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        h = C.c_void_p()
        with torch.cuda.device(dev):
            check(lib().ndgi_host_pipe_create(self.chunk, _p(self.staging), nbytes, C.byref(h)))
        self.handle = h

    def decode_points(self, model, uvt_host, precision="fp32", ws=None, out=None, stream=None):
        """rgb [n][3] float32 (host) of the decode at each (u, v, t) row of the host tensor uvt_host.
        Asynchronous on `stream`: synchronise it before reading `out`."""
        if uvt_host.is_cuda or uvt_host.dtype != torch.float32 or not uvt_host.is_contiguous():
            raise ValueError("uvt_host must be a contiguous float32 host tensor")
        n = uvt_host.shape[0]
        if out is None:
            out = torch.empty((n, 3), dtype=torch.float32, pin_memory=uvt_host.is_pinned())
        if out.is_cuda or out.dtype != torch.float32 or not out.is_contiguous() or out.shape[0] != n:
            raise ValueError("out must be a contiguous float32 host tensor [n][3]")
        pr = _prec(precision)
        if ws is None and pr != A.NDGI_FP32:
            ws = model.workspace(pr)
        check(lib().ndgi_decode_points_host(self.handle, C.byref(model.desc), pr, _p(ws), uvt_host.data_ptr(), n,
                                            out.data_ptr(), _stream(stream)))
        return out

    def close(self):
        if self.handle:
            check(lib().ndgi_host_pipe_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ndgi_debug_features(model, uvt, stream=None):
    """(x [n][cs+ct] float32, p35 [n][4][cs] int32) of the gather stage."""
    uvt = _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    x = torch.empty((n, model.cs + model.ct), dtype=torch.float32, device=uvt.device)
    p35 = torch.empty((n, 4, model.cs), dtype=torch.int32, device=uvt.device)
    check(lib().ndgi_debug_features(C.byref(model.desc), _p(uvt), n, _p(x), _p(p35), _stream(stream)))
    return x, p35


def ndgi_debug_features_tc(model, uvt, precision="fp16", stream=None):
    """x [n][cs+ct] float32 of the tensor-core point decode's gather (texel-sliced planes)."""
    uvt = _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    x = torch.empty((n, model.cs + model.ct), dtype=torch.float32, device=uvt.device)
    ws = model.workspace(precision)
    check(lib().ndgi_debug_features_tc(C.byref(model.desc), _p(ws), _p(uvt), n, _p(x), _stream(stream)))
    return x


def ndgi_debug_features_cache(model, uvt, precision="fp16", stream=None):
    """x [n][cs+ct] float32 of the cache path's gather (FP16 decoded-texel cache, half2 blend)."""
    uvt = _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    x = torch.empty((n, model.cs + model.ct), dtype=torch.float32, device=uvt.device)
    ws = model.workspace(precision)
    check(lib().ndgi_debug_features_cache(C.byref(model.desc), _p(ws), _p(uvt), n, _p(x), _stream(stream)))
    return x


def ndgi_decode_points_path(model, precision, n):
    """'direct', 'cache' (four-lane kernel) or 'cache_ws' (warp-specialised kernel): how a point decode of n
    queries gathers."""
    return ("direct", "cache", "cache_ws")[lib().ndgi_decode_points_path(C.byref(model.desc), _prec(precision),
                                                                        int(n))]


# ---------------------------------------------------------------------------
# Pages
# ---------------------------------------------------------------------------
PAGE_REQ_DTYPE = np.dtype([("model", "<i4"), ("x0", "<i4"), ("y0", "<i4"), ("w", "<i4"), ("h", "<i4"),
                           ("t", "<f4"), ("dst_x", "<i4"), ("dst_y", "<i4")])


def page_requests_to_device(reqs, device="cuda"):
    """Structured numpy array (PAGE_REQ_DTYPE) -> (int32 [n][8] CUDA tensor, n tensor)."""
    r = np.ascontiguousarray(reqs).view(np.int32).reshape(-1, 8)
    t = torch.from_numpy(r.copy()).to(device)
    n = torch.tensor([len(reqs)], dtype=torch.int32, device=device)
    return t, n


class PagesPlan:
    """ndgi_pages_plan_* wrapper.  `phys` is [phys_h][phys_w][4] float32 or float16."""

    def __init__(self, models, precision, max_reqs, phys):
        self.models = list(models)
        self.precision = _prec(precision)
        self.phys = phys
        if phys.dtype == torch.float32:
            fmt = A.NDGI_RGBA32F
        elif phys.dtype == torch.float16:
            fmt = A.NDGI_RGBA16F
        else:
            raise ValueError("phys must be float32, float16 or uint8 RGBA")
        assert phys.is_cuda and phys.is_contiguous() and phys.shape[-1] == 4
        descs = (A.ModelDesc * len(self.models))(*[m.desc for m in self.models])
        ws = [m.workspace(self.precision) for m in self.models]
        ws_arr = (C.c_void_p * len(ws))(*[w.data_ptr() if w is not None else None for w in ws])
        self._keep = (descs, ws_arr, ws)
        h = C.c_void_p()
        check(lib().ndgi_pages_plan_create(descs, ws_arr, len(self.models), self.precision, int(max_reqs), fmt,
                                           _p(phys), phys.shape[1], phys.shape[0], C.byref(h)))
        self.handle = h

    def decode(self, reqs, n_dev, stream=None):
        check(lib().ndgi_decode_pages(self.handle, _p(reqs), _p(n_dev), _stream(stream)))

    def autotune(self, reqs, n_dev, n_host, stream=None):
        check(lib().ndgi_pages_autotune(self.handle, _p(reqs), _p(n_dev), int(n_host), _stream(stream)))

    def info(self):
        """(precision, ctas_per_sm or grid, lanes, slots) of the current launch shape."""
        a = (C.c_int32 * 4)()
        check(lib().ndgi_pages_plan_info(self.handle, a))
        return tuple(a)

    def set_shape(self, ctas_per_sm, lanes, slots):
        check(lib().ndgi_pages_plan_set_shape(self.handle, int(ctas_per_sm), int(lanes), int(slots)))

    def check(self, stream=None):
        err = C.c_int32(0)
        st = lib().ndgi_pages_check(self.handle, C.byref(err), _stream(stream))
        return st, err.value

    def set_debug(self, flags):
        """Test hook: 1 = the tensor-core decodes take their timeout path before any MMA; 0 = normal."""
        check(lib().ndgi_pages_plan_set_debug(self.handle, int(flags)))

    def set_fp8_dump(self, item, dump=None):
        """Test hook: operands of one tile of request `item` into `dump` (uint8 CUDA tensor; None = off)."""
        check(lib().ndgi_pages_plan_set_fp8_dump(self.handle, int(item), _p(dump)))

    def fp8_dump_size(self):
        return int(lib().ndgi_pages_fp8_dump_size(self.handle))

    def close(self):
        if self.handle:
            check(lib().ndgi_pages_plan_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ndgi_decode_pages(plan, reqs, n_dev, stream=None):
    plan.decode(reqs, n_dev, stream)


def ndgi_decode_pages_static(models, reqs, n_dev, max_reqs, phys, device_error=None, stream=None):
    """FP32 page decode that allocates nothing on the device (library-held
    static scratch); for callers that cannot use cudaMalloc.  Same output as
    a PagesPlan with "fp32"."""
    fmt = A.NDGI_RGBA32F if phys.dtype == torch.float32 else A.NDGI_RGBA16F
    descs = (A.ModelDesc * len(models))(*[m.desc for m in models])
    check(lib().ndgi_decode_pages_static(descs, len(models), _p(reqs), _p(n_dev), int(max_reqs), fmt, _p(phys),
                                         phys.shape[1], phys.shape[0], _p(device_error), _stream(stream)))


# ---------------------------------------------------------------------------
# BC pack and fit
# ---------------------------------------------------------------------------
def ndgi_bc_pack(ea, eb, w, out=None, stream=None):
    """BC4 blocks uint8 [bh][bw][cs][8] from endpoints [bh][bw][cs] and weights [bh][bw][cs][16]."""
    _need(ea, torch.float32, "ea")
    _need(eb, torch.float32, "eb")
    _need(w, torch.float32, "w")
    bh, bw, cs = ea.shape
    if out is None:
        out = torch.empty((bh, bw, cs, 8), dtype=torch.uint8, device=ea.device)
    check(lib().ndgi_bc_pack(_p(ea), _p(eb), _p(w), cs, bw * 4, bh * 4, _p(out), _stream(stream)))
    return out


class FitState:
    """Trainable parameters of the fit (float32 CUDA tensors) and their struct."""

    def __init__(self, tensors, lm_w, lm_h, address_mode=0, key_t=None):
        self.t = {k: _need(tensors[k], torch.float32, k) for k in A.FIT_TENSORS}
        self.key_t = None if key_t is None else _need(key_t, torch.float32, "key_t")
        bh, bw, cs = self.t["ea"].shape
        T, ct = self.t["temporal"].shape
        H = self.t["w2"].shape[0]
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.dims = dict(feat_w=bw * 4, feat_h=bh * 4, cs=cs, t_count=T, ct=ct, hidden=H)
        self.params = A.FitParams(self.lm_w, self.lm_h, bw * 4, bh * 4, cs, T, ct, H,
                                  *[self.t[k].data_ptr() for k in A.FIT_TENSORS], int(address_mode),
                                  _p(self.key_t))
        self.address_mode = int(address_mode)

    @classmethod
    def from_arrays(cls, p, lm_w, lm_h, device="cuda"):
        key_t = p.get("key_t")
        return cls({k: torch.from_numpy(np.ascontiguousarray(p[k], np.float32)).to(device) for k in A.FIT_TENSORS},
                   lm_w, lm_h, p.get("address_mode", 0),
                   None if key_t is None else torch.from_numpy(np.ascontiguousarray(key_t, np.float32)).to(device))

    def zeros_like(self):
        return {k: torch.zeros_like(v) for k, v in self.t.items()}


def ndgi_fit_forward(state, uvt, relaxed=False, out=None, stream=None):
    """rgb [n][3] of the fit's straight-through (or relaxed) decode at queries uvt [n][3] float32 (u, v, t)."""
    _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=uvt.device)
    check(lib().ndgi_fit_forward(C.byref(state.params), _p(uvt), n, int(relaxed), _p(out), _stream(stream)))
    return out


def ndgi_fit_backward(state, uvt, grad_rgb, grads=None, relaxed=False, stream=None):
    """Adds dL/dparams at queries uvt [n][3] into `grads` (dict of tensors, created zeroed if None); returns it."""
    _need(uvt, torch.float32, "uvt")
    _need(grad_rgb, torch.float32, "grad_rgb")
    if grads is None:
        grads = state.zeros_like()
    g = A.FitGrads(*[grads[k].data_ptr() for k in A.FIT_TENSORS])
    check(lib().ndgi_fit_backward(C.byref(state.params), _p(uvt), uvt.shape[0], int(relaxed),
                                  _p(grad_rgb), C.byref(g), _stream(stream)))
    return grads


class NdgiDecodeFunction(torch.autograd.Function):
    """The fit's decode as a differentiable torch op: the straight-through
    BC4 forward of ndgi_fit_forward and the hand-written CUDA backward of
    ndgi_fit_backward (through the MLP, the temporal and bilinear sampling
    and the BC4 quantisation, treated as identity).  Inputs after the four
    settings and the keyframe times are the FIT_TENSORS in order; the queries
    carry no gradient."""

    @staticmethod
    def forward(ctx, uvt, relaxed, lm_w, lm_h, address_mode, key_t, *tensors):
        state = FitState(dict(zip(A.FIT_TENSORS, tensors)), lm_w, lm_h, address_mode, key_t)
        ctx.save_for_backward(uvt, *tensors)
        ctx.key_t = key_t
        ctx.settings = (bool(relaxed), int(lm_w), int(lm_h), int(address_mode))
        return ndgi_fit_forward(state, uvt, relaxed)

    @staticmethod
    def backward(ctx, grad_rgb):
        uvt, *tensors = ctx.saved_tensors
        relaxed, lm_w, lm_h, address_mode = ctx.settings
        state = FitState(dict(zip(A.FIT_TENSORS, tensors)), lm_w, lm_h, address_mode, ctx.key_t)
        grads = ndgi_fit_backward(state, uvt, grad_rgb.contiguous(), relaxed=relaxed)
        return (None, None, None, None, None, None) + tuple(grads[k] for k in A.FIT_TENSORS)


def ndgi_decode_fit(params, uvt, lm_w, lm_h, relaxed=False, address_mode=0, key_t=None):
    """rgb [n][3] of the fit's decode at arbitrary queries uvt [n][3] float32 (u, v, t), differentiable
    w.r.t. params (dict of float32 CUDA tensors keyed by FIT_TENSORS), through the temporal interpolation
    at fractional t as well as the MLP, the bilinear gather and the straight-through BC4 quantisation.
    key_t: keyframe times (float32 CUDA tensor [T]) or None for j / T."""
    return NdgiDecodeFunction.apply(uvt, relaxed, lm_w, lm_h, address_mode, key_t,
                                    *[params[k] for k in A.FIT_TENSORS])


def fit_config(steps, batch, lr=1e-2, beta1=0.9, beta2=0.999, eps=1e-8, freeze_steps=0, loss_every=0, seed=0,
               relaxed=False, noise_alpha=0.0):
    return A.FitConfig(int(steps), int(batch), float(lr), float(beta1), float(beta2), float(eps), int(freeze_steps),
                       int(loss_every), int(seed), int(relaxed), float(noise_alpha))


def ndgi_encode_fit_workspace_size(state, cfg):
    return int(lib().ndgi_encode_fit_workspace_size(C.byref(state.params), C.byref(cfg)))


def ndgi_encode_fit(state, targets, cfg, step_offset=0, ws=None, loss_log=None, stream=None):
    """Runs cfg.steps Adam steps in place on state's tensors.  targets: float16
    [T][lm_h][lm_w][3] CUDA.  Returns (ws, loss_log)."""
    _need(targets, torch.float16, "targets")
    if ws is None:
        ws = torch.empty(ndgi_encode_fit_workspace_size(state, cfg), dtype=torch.uint8, device=targets.device)
    if loss_log is None and cfg.loss_every > 0:
        loss_log = torch.zeros((cfg.steps + cfg.loss_every - 1) // cfg.loss_every, dtype=torch.float64,
                               device=targets.device)
    check(lib().ndgi_encode_fit(C.byref(state.params), _p(targets), C.byref(cfg), int(step_offset), _p(ws),
                                ws.numel(), _p(loss_log), _stream(stream)))
    return ws, loss_log


# ---------------------------------------------------------------------------
# Hybrid feature map decoder (the paper's full decoder)
# ---------------------------------------------------------------------------
class HybridModel:
    """A hybrid model resident on the GPU plus its ndgi_hybrid_desc.

    Tensors: uv_bc4 uint8 [uv_h/4][uv_w/4][4][8], vol_bc4 uint8
    [vol_t][vol_h/4][vol_w/4][4][8], ut uint8 [ut_t][ut_w][2], vt uint8
    [vt_t][vt_h][2], MLP weights float32 [in][out] (w1 [16][hidden]).
    Prepared tensor-core workspaces are kept per precision in ``self.ws``.
    """

    def __init__(self, lm_w, lm_h, uv_bc4, vol_bc4, ut, vt, w1, b1, w2, b2, w3, b3, address_mode=0):
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.uv_bc4 = _need(uv_bc4, torch.uint8, "uv_bc4")
        self.vol_bc4 = _need(vol_bc4, torch.uint8, "vol_bc4")
        self.ut = _need(ut, torch.uint8, "ut")
        self.vt = _need(vt, torch.uint8, "vt")
        # block format from the shape: four BC4 planes [..][4][8] or BC7 [..][16]
        self.feat_format = A.NDGI_FEAT_BC7 if uv_bc4.dim() == 3 else A.NDGI_FEAT_BC4X4
        if self.feat_format == A.NDGI_FEAT_BC7:
            bh, bw, sixteen = uv_bc4.shape
            vt_, vbh, vbw, sixteen2 = vol_bc4.shape
            assert sixteen == 16 and sixteen2 == 16
        else:
            bh, bw, four, eight = uv_bc4.shape
            assert four == 4 and eight == 8
            vt_, vbh, vbw, four, eight = vol_bc4.shape
            assert four == 4 and eight == 8
        self.w = {k: _need(v, torch.float32, k) for k, v in
                  dict(w1=w1, b1=b1, w2=w2, b2=b2, w3=w3, b3=b3).items()}
        self.hidden = w2.shape[0]
        self.address_mode = int(address_mode)
        self.desc = A.HybridDesc(self.lm_w, self.lm_h, bw * 4, bh * 4, uv_bc4.data_ptr(), vbw * 4, vbh * 4, vt_,
                                 vol_bc4.data_ptr(), ut.shape[1], ut.shape[0], ut.data_ptr(), vt.shape[1],
                                 vt.shape[0], vt.data_ptr(), self.hidden,
                                 *[self.w[k].data_ptr() for k in ("w1", "b1", "w2", "b2", "w3", "b3")],
                                 self.address_mode, self.feat_format)
        self.ws = {}

    @classmethod
    def from_arrays(cls, m, device="cuda"):
        """From a dict of numpy arrays (the layout of synth.hybrid_model)."""
        def t(a):
            return torch.from_numpy(np.ascontiguousarray(a)).to(device)
        uv, vol = ("uv_bc7", "vol_bc7") if m.get("feat_format", 0) == 1 else ("uv_bc4", "vol_bc4")
        return cls(m["lm_w"], m["lm_h"], t(m[uv]), t(m[vol]), t(m["ut"]), t(m["vt"]), t(m["w1"]),
                   t(m["b1"]), t(m["w2"]), t(m["b2"]), t(m["w3"]), t(m["b3"]), m.get("address_mode", 0))

    @classmethod
    def from_set(cls, s, device="cuda"):
        """All models of a stacked set (synth.hybrid_tile_set) as views into one device tensor per array."""
        uv, vol = ("uv_bc7", "vol_bc7") if s.get("feat_format", 0) == 1 else ("uv_bc4", "vol_bc4")
        keys = (uv, vol, "ut", "vt", "w1", "b1", "w2", "b2", "w3", "b3")
        big = {k: torch.from_numpy(np.ascontiguousarray(s[k])).to(device) for k in keys}
        return [cls(s["lm_w"], s["lm_h"], *[big[k][i] for k in keys], s.get("address_mode", 0))
                for i in range(int(s["n_tiles"]))]

    def workspace(self, precision):
        precision = _prec(precision)
        if precision == A.NDGI_FP32:
            return None
        if precision not in self.ws:
            self.ws[precision] = ndgi_hybrid_prepare(self, precision)
        return self.ws[precision]


def hybrid_prepare_set(models, precision, stream=None):
    """Prepares every model of a list into slices of one device workspace tensor (256-byte aligned)."""
    precision = _prec(precision)
    if precision == A.NDGI_FP32:
        return None
    n = ndgi_hybrid_workspace_size(models[0], precision)
    ws = torch.empty(n * len(models), dtype=torch.uint8, device=models[0].uv_bc4.device)
    for i, m in enumerate(models):
        m.ws[precision] = ndgi_hybrid_prepare(m, precision, ws[i * n:(i + 1) * n], stream)
    return ws


def ndgi_hybrid_workspace_size(model, precision):
    return int(lib().ndgi_hybrid_workspace_size(C.byref(model.desc), _prec(precision)))


def ndgi_hybrid_prepare(model, precision, ws=None, stream=None):
    """Packs the hybrid model's MLP for a tensor-core decode; returns the workspace tensor."""
    n = ndgi_hybrid_workspace_size(model, precision)
    if ws is None:
        ws = torch.empty(max(n, 256), dtype=torch.uint8, device=model.uv_bc4.device)
    check(lib().ndgi_hybrid_prepare(C.byref(model.desc), _prec(precision), _p(ws), _stream(stream)))
    return ws


def ndgi_hybrid_decode_points(model, uvt, precision="fp32", out=None, stream=None):
    """rgb [n][3] float32 of the hybrid decoder at queries uvt [n][3] float32."""
    _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=uvt.device)
    check(lib().ndgi_hybrid_decode_points(C.byref(model.desc), _prec(precision), _p(model.workspace(precision)),
                                          _p(uvt), n, _p(out), _stream(stream)))
    return out


def ndgi_hybrid_workspace_check(model, precision, stream=None):
    """(status, error word) of the hybrid point decodes that used the model's workspace; clears the word."""
    err = C.c_int32(0)
    st = lib().ndgi_hybrid_workspace_check(C.byref(model.desc), _prec(precision), _p(model.workspace(precision)),
                                           C.byref(err), _stream(stream))
    return st, err.value


def ndgi_hybrid_debug_inject(model=None, precision="fp16", table=None, flags=1, stream=None):
    """Test hook: flags = 1 makes the tensor-core decodes that use the model's workspace and/or the table take
    their timeout path before any MMA; 0 = normal."""
    desc = C.byref(model.desc) if model is not None else None
    ws = _p(model.workspace(precision)) if model is not None else None
    check(lib().ndgi_hybrid_debug_inject(desc, _prec(precision), ws, table.handle if table is not None else None,
                                         int(flags), _stream(stream)))


class HybridTable:
    """ndgi_hybrid_table_* wrapper: the device table of hybrid models of a page decode."""

    def __init__(self, models, precision):
        self.models = list(models)
        self.precision = _prec(precision)
        descs = (A.HybridDesc * len(self.models))(*[m.desc for m in self.models])
        ws = [m.workspace(self.precision) for m in self.models]
        ws_arr = (C.c_void_p * len(ws))(*[w.data_ptr() if w is not None else None for w in ws])
        self._keep = (descs, ws_arr, ws)
        h = C.c_void_p()
        check(lib().ndgi_hybrid_table_create(descs, ws_arr, len(self.models), self.precision, C.byref(h)))
        self.handle = h

    def decode(self, reqs, n, phys, stream=None):
        """Decodes n requests (int32 [n][8] CUDA tensor) into phys ([h][w][4] float32, float16 or uint8 UNORM)."""
        if phys.dtype == torch.float32:
            fmt = A.NDGI_RGBA32F
        elif phys.dtype == torch.float16:
            fmt = A.NDGI_RGBA16F
        elif phys.dtype == torch.uint8:
            fmt = A.NDGI_RGBA8
        else:
            raise ValueError("phys must be float32 or float16 RGBA")
        assert phys.is_cuda and phys.is_contiguous() and phys.shape[-1] == 4
        check(lib().ndgi_hybrid_decode_pages(self.handle, _p(reqs), int(n), _p(phys), phys.shape[1], phys.shape[0],
                                             fmt, _stream(stream)))

    def check(self, stream=None):
        err = C.c_int32(0)
        st = lib().ndgi_hybrid_table_check(self.handle, C.byref(err), _stream(stream))
        return st, err.value

    def set_border(self, border):
        """Mirrored tile border (texels per edge, 0..8) of later page decodes."""
        check(lib().ndgi_hybrid_table_set_border(self.handle, int(border)))

    def close(self):
        if self.handle:
            check(lib().ndgi_hybrid_table_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ndgi_model_bpp(desc, n_lightmaps, bc_bits_per_texel=8, mlp_bits=16):
    """Bits per lightmap texel of a hybrid model's storage (host only; desc an A.HybridDesc or HybridModel)."""
    d = desc.desc if isinstance(desc, HybridModel) else desc
    return float(lib().ndgi_model_bpp(C.byref(d), int(n_lightmaps), int(bc_bits_per_texel), int(mlp_bits)))


def ndgi_debug_gelu(x, fast=1, stream=None):
    """GELU of a float32 CUDA tensor: fast = 0 as the FP32 decodes evaluate it (erff), 1 the scalar erfc form,
    2 the packed-pair form the tensor-core epilogues use."""
    _need(x, torch.float32, "x")
    y = torch.empty_like(x)
    check(lib().ndgi_debug_gelu(_p(x), x.numel(), _p(y), int(fast), _stream(stream)))
    return y


def ndgi_tile_metrics(pred, ref, mask=None, tile=128, stream=None):
    """Per-tile (PSNR, SSIM) FP64 tensors [n][ceil(h/tile)][ceil(w/tile)] of float32 CUDA maps [n][h][w][c]
    (or [h][w][c]) under an optional uint8/bool mask [n][h][w]."""
    if pred.dim() == 3:
        pred, ref = pred[None], ref[None]
        mask = None if mask is None else mask[None]
    _need(pred, torch.float32, "pred")
    _need(ref, torch.float32, "ref")
    if mask is not None:
        mask = mask.to(torch.uint8).contiguous()
    n, h, w, c = pred.shape
    ty, tx = (h + tile - 1) // tile, (w + tile - 1) // tile
    ps = torch.empty((n, ty, tx), dtype=torch.float64, device=pred.device)
    ss = torch.empty_like(ps)
    check(lib().ndgi_tile_metrics(_p(pred), _p(ref), _p(mask), n, h, w, c, int(tile), _p(ps), _p(ss),
                                  _stream(stream)))
    return ps, ss


class FitBatch:
    """n_models fit parameter sets of one shape, stacked along a leading axis (float32 CUDA tensors
    [n_models][...] per FIT_TENSORS key), for ndgi_encode_fit_batch."""

    def __init__(self, tensors, lm_w, lm_h, address_mode=0, key_t=None):
        self.t = {k: _need(tensors[k], torch.float32, k) for k in A.FIT_TENSORS}
        self.n_models = int(self.t["ea"].shape[0])
        assert all(int(v.shape[0]) == self.n_models for v in self.t.values())
        self.key_t = None if key_t is None else _need(key_t, torch.float32, "key_t")
        _, bh, bw, cs = self.t["ea"].shape
        _, T, ct = self.t["temporal"].shape
        H = self.t["w2"].shape[1]
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.params = A.FitParams(self.lm_w, self.lm_h, bw * 4, bh * 4, cs, T, ct, H,
                                  *[self.t[k].data_ptr() for k in A.FIT_TENSORS], int(address_mode),
                                  _p(self.key_t))

    @classmethod
    def from_arrays(cls, ps, lm_w, lm_h, key_t=None, device="cuda"):
        """From a list of fit dicts (synth.fit_init)."""
        t = {k: torch.from_numpy(np.ascontiguousarray(np.stack([p[k] for p in ps]), np.float32)).to(device)
             for k in A.FIT_TENSORS}
        return cls(t, lm_w, lm_h, ps[0].get("address_mode", 0),
                   None if key_t is None else torch.from_numpy(np.asarray(key_t, np.float32)).to(device))

    def model(self, m):
        """Model m's tensors (views)."""
        return {k: v[m] for k, v in self.t.items()}


def ndgi_encode_fit_batch(batch, targets, cfg, step_offset=0, ws=None, loss_log=None, stream=None):
    """cfg.steps Adam steps of every model of a FitBatch in place.  targets: float16
    [n_models][T][lm_h][lm_w][3] CUDA.  Returns (ws, loss_log)."""
    _need(targets, torch.float16, "targets")
    n = int(lib().ndgi_encode_fit_batch_workspace_size(C.byref(batch.params), batch.n_models, C.byref(cfg)))
    if ws is None:
        ws = torch.empty(n, dtype=torch.uint8, device=targets.device)
    if loss_log is None and cfg.loss_every > 0:
        loss_log = torch.zeros((cfg.steps + cfg.loss_every - 1) // cfg.loss_every, dtype=torch.float64,
                               device=targets.device)
    check(lib().ndgi_encode_fit_batch(C.byref(batch.params), batch.n_models, _p(targets), C.byref(cfg),
                                      int(step_offset), _p(ws), ws.numel(), _p(loss_log), _stream(stream)))
    return ws, loss_log


# ---------------------------------------------------------------------------
# Fit of the hybrid decoder
# ---------------------------------------------------------------------------
def _hfit_params(t, lm_w, lm_h, address_mode, lead=0):
    """ndgi_hybrid_fit_params of one model's shape (tensor shapes read past `lead` leading axes)."""
    ubh, ubw = t["uv_ea"].shape[lead:lead + 2]
    vt_, vbh, vbw = t["vol_ea"].shape[lead:lead + 3]
    ut_t, ut_w = t["ut"].shape[lead:lead + 2]
    vt_t, vt_h = t["vt"].shape[lead:lead + 2]
    hidden = int(t["w2"].shape[lead])
    shared = t["uv_wt"].dim() - lead == 3       # [uv_h/4][uv_w/4][16]: Eq. 7's weight per texel
    return A.HybridFitParams(int(lm_w), int(lm_h), ubw * 4, ubh * 4, vbw * 4, vbh * 4, vt_, ut_w, ut_t, vt_h, vt_t,
                             hidden, int(address_mode), *[t[k].data_ptr() for k in A.HFIT_TENSORS],
                             int(shared)), hidden, shared


class HybridFitState:
    """Trainable parameters of a hybrid model (float32 CUDA tensors keyed by HFIT_TENSORS) and their struct."""

    def __init__(self, tensors, lm_w, lm_h, address_mode=0):
        self.t = {k: _need(tensors[k], torch.float32, k) for k in A.HFIT_TENSORS}
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.params, self.hidden, self.shared_w = _hfit_params(self.t, lm_w, lm_h, address_mode)

    @classmethod
    def from_arrays(cls, p, device="cuda"):
        """From a dict of numpy arrays (synth.hybrid_fit_init)."""
        return cls({k: torch.from_numpy(np.ascontiguousarray(p[k], np.float32)).to(device) for k in A.HFIT_TENSORS},
                   p["lm_w"], p["lm_h"], p.get("address_mode", 0))


class HybridFitBatch:
    """n_models hybrid models of one shape, each tensor stacked along a leading model axis."""

    def __init__(self, tensors, lm_w, lm_h, address_mode=0):
        self.t = {k: _need(tensors[k], torch.float32, k) for k in A.HFIT_TENSORS}
        self.n_models = int(self.t["w1"].shape[0])
        self.lm_w, self.lm_h = int(lm_w), int(lm_h)
        self.params, self.hidden, self.shared_w = _hfit_params(self.t, lm_w, lm_h, address_mode, lead=1)

    @classmethod
    def from_arrays(cls, ps, device="cuda"):
        """From a list of dicts of numpy arrays (synth.hybrid_fit_init), one per model."""
        return cls({k: torch.from_numpy(np.ascontiguousarray(np.stack([p[k] for p in ps]), np.float32)).to(device)
                    for k in A.HFIT_TENSORS}, ps[0]["lm_w"], ps[0]["lm_h"], ps[0].get("address_mode", 0))

    def model(self, i):
        """Model i's tensors (views)."""
        return {k: v[i] for k, v in self.t.items()}


def ndgi_hybrid_fit_forward(state, uvt, relaxed=False, out=None, stream=None):
    """rgb [n][3] of the hybrid fit's straight-through (or relaxed) forward at queries uvt [n][3] float32."""
    _need(uvt, torch.float32, "uvt")
    n = uvt.shape[0]
    if out is None:
        out = torch.empty((n, 3), dtype=torch.float32, device=uvt.device)
    check(lib().ndgi_hybrid_fit_forward(C.byref(state.params), _p(uvt), n, int(relaxed), _p(out), _stream(stream)))
    return out


def ndgi_hybrid_fit_backward(state, uvt, grad_rgb, grads=None, relaxed=False, stream=None):
    """Gradients (dict of float32 tensors) of the loss whose dL/drgb is grad_rgb [n][3]; accumulated into grads
    when given (zeroed buffers are allocated otherwise)."""
    _need(uvt, torch.float32, "uvt")
    _need(grad_rgb, torch.float32, "grad_rgb")
    if grads is None:
        grads = {k: torch.zeros_like(v) for k, v in state.t.items()}
    gs = A.HybridFitGrads((C.c_void_p * 14)(*[grads[k].data_ptr() for k in A.HFIT_TENSORS]))
    check(lib().ndgi_hybrid_fit_backward(C.byref(state.params), _p(uvt), uvt.shape[0], int(relaxed), _p(grad_rgb),
                                         C.byref(gs), _stream(stream)))
    return grads


def ndgi_hybrid_encode_fit(state, targets, cfg, key_t=None, step_offset=0, ws=None, loss_log=None, stream=None):
    """cfg.steps Adam steps of the hybrid fit in place on state's tensors.  targets: float16 [T][lm_h][lm_w][3]
    CUDA at the keyframe times key_t (float32 CUDA [T]) or j / T.  Returns (ws, loss_log)."""
    _need(targets, torch.float16, "targets")
    n = int(lib().ndgi_hybrid_encode_fit_workspace_size(C.byref(state.params), C.byref(cfg)))
    if ws is None:
        ws = torch.empty(n, dtype=torch.uint8, device=targets.device)
    if loss_log is None and cfg.loss_every > 0:
        loss_log = torch.zeros((cfg.steps + cfg.loss_every - 1) // cfg.loss_every, dtype=torch.float64,
                               device=targets.device)
    check(lib().ndgi_hybrid_encode_fit(C.byref(state.params), _p(targets), int(targets.shape[0]), _p(key_t),
                                       C.byref(cfg), int(step_offset), _p(ws), ws.numel(), _p(loss_log),
                                       _stream(stream)))
    return ws, loss_log


# --------------------------------------------------------------------------
# BC7 (the paper's block format for F_uv and F3D)
# --------------------------------------------------------------------------

def ndgi_bc7_encode(rgba, out=None, sq_err=None, stream=None):
    """BC7 blocks uint8 [h/4][w/4][16] of an RGBA8 image uint8 [h][w][4] (CUDA); sq_err (int64 [1], CUDA), when
    given, accumulates the total squared error."""
    _need(rgba, torch.uint8, "rgba")
    h, w, four = rgba.shape
    assert four == 4
    if out is None:
        out = torch.empty((h // 4, w // 4, 16), dtype=torch.uint8, device=rgba.device)
    check(lib().ndgi_bc7_encode(_p(rgba), w, h, _p(out), _p(sq_err), _stream(stream)))
    return out


def ndgi_bc7_decode(blocks, out=None, stream=None):
    """RGBA8 [h][w][4] of BC7 blocks uint8 [h/4][w/4][16] (CUDA)."""
    _need(blocks, torch.uint8, "blocks")
    bh, bw, sixteen = blocks.shape
    assert sixteen == 16
    if out is None:
        out = torch.empty((bh * 4, bw * 4, 4), dtype=torch.uint8, device=blocks.device)
    check(lib().ndgi_bc7_decode(_p(blocks), bw * 4, bh * 4, _p(out), _stream(stream)))
    return out


def ndgi_bc4x4_to_rgba8(bc4, out=None, stream=None):
    """RGBA8 [h][w][4] = round(255 P35 / 8925) of four BC4 planes uint8 [h/4][w/4][4][8] (CUDA)."""
    _need(bc4, torch.uint8, "bc4")
    bh, bw, four, eight = bc4.shape
    assert four == 4 and eight == 8
    if out is None:
        out = torch.empty((bh * 4, bw * 4, 4), dtype=torch.uint8, device=bc4.device)
    check(lib().ndgi_bc4x4_to_rgba8(_p(bc4), bw * 4, bh * 4, _p(out), _stream(stream)))
    return out


def ndgi_debug_bc7_hw_decode(blocks, stream=None):
    """RGBA8 [h][w][4] of BC7 blocks decoded by the GPU's texture unit (test reference)."""
    _need(blocks, torch.uint8, "blocks")
    bh, bw, sixteen = blocks.shape
    out = torch.empty((bh * 4, bw * 4, 4), dtype=torch.uint8, device=blocks.device)
    check(lib().ndgi_debug_bc7_hw_decode(_p(blocks), bw * 4, bh * 4, _p(out), _stream(stream)))
    return out


def ndgi_bc_sim7_to_rgba8(ea, eb, w, out=None, stream=None):
    """RGBA8 [h][w][4] of a shared-weight BC-simulated map: ea, eb float32 [..][h/4][w/4][4], w [..][h/4][w/4][16]
    (CUDA; leading axes, e.g. F3D slices, stacked along the height)."""
    for t, name in ((ea, "ea"), (eb, "eb"), (w, "w")):
        _need(t, torch.float32, name)
    bw = ea.shape[-2]
    bh = ea.numel() // (bw * 4)
    if out is None:
        out = torch.empty((bh * 4, bw * 4, 4), dtype=torch.uint8, device=ea.device)
    check(lib().ndgi_bc_sim7_to_rgba8(_p(ea), _p(eb), _p(w), bw * 4, bh * 4, _p(out), _stream(stream)))
    return out


def ndgi_bc7_pack_sim(ea, eb, w, out=None, stream=None):
    """Exact BC7 mode-6 blocks uint8 [..][16] of a shared-weight BC-simulated map (ea, eb [..][4], w [..][16])."""
    for t, name in ((ea, "ea"), (eb, "eb"), (w, "w")):
        _need(t, torch.float32, name)
    if out is None:
        out = torch.empty(tuple(ea.shape[:-1]) + (16,), dtype=torch.uint8, device=ea.device)
    check(lib().ndgi_bc7_pack_sim(_p(ea), _p(eb), _p(w), ea.numel() // 4, _p(out), _stream(stream)))
    return out


def ndgi_hybrid_encode_fit_batch(batch, targets, cfg, key_t=None, step_offset=0, ws=None, loss_log=None,
                                 stream=None):
    """cfg.steps Adam steps of every model of a HybridFitBatch in place, one launch per step.  targets: float16
    [n_models][T][lm_h][lm_w][3] CUDA at the keyframe times key_t (float32 CUDA [T]) or j / T.
    Returns (ws, loss_log)."""
    _need(targets, torch.float16, "targets")
    n = int(lib().ndgi_hybrid_encode_fit_batch_workspace_size(C.byref(batch.params), batch.n_models, C.byref(cfg)))
    if ws is None:
        ws = torch.empty(n, dtype=torch.uint8, device=targets.device)
    if loss_log is None and cfg.loss_every > 0:
        loss_log = torch.zeros((cfg.steps + cfg.loss_every - 1) // cfg.loss_every, dtype=torch.float64,
                               device=targets.device)
    check(lib().ndgi_hybrid_encode_fit_batch(C.byref(batch.params), batch.n_models, _p(targets),
                                             int(targets.shape[1]), _p(key_t), C.byref(cfg), int(step_offset),
                                             _p(ws), ws.numel(), _p(loss_log), _stream(stream)))
    return ws, loss_log
