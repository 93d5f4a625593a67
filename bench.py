"""Benchmark of the NDGI random-access decode on GB300.

Workload (one "step"): decode 2^24 random (u, v, t) queries of a 2048x2048
atlas whose model is 1024x1024x16 BC4 planes, a 24x8 FP16 temporal line and
a 24->64->64->3 ReLU MLP (the whole hot path: BC fetch + decode, bilinear,
temporal lerp, MLP).  The headline value is the tensor-core FP16 decode in
Gtexels/s; the FP32 CUDA-core decode is timed beside it, and both are
checked against the FP64 oracle on a seeded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: every rank decodes its own 2^24 queries (weak
scaling, replicas, no data-path collective); the time is the max over ranks.
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

N_QUERIES = 1 << 24
FLOP_PER_TEXEL = 2 * (24 * 64 + 64 * 64 + 64 * 3)          # 11,648 (unpadded MLP)
WORKLOAD = "points 2^24 random (u,v,t); atlas 2048^2, BC4 1024^2x16, temporal 24x8 fp16, MLP 24-64-64-3"
METRIC = "Gtexels/s decoded (BC fetch+temporal lerp+MLP), FP16-TC vs FP32 plain @err"


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of a smaller case
# of the same kernel, scaled to a full launch by the units processed.  Valid only while the kernel's sources are
# the ones captured: each kernel's own source set is hashed at run time and its figure drops to null once the code
# changes.
_COMMON_SOURCES = ("tc_engine.cuh", "gather.cuh", "bc4.cuh", "umma.cuh", "ndgi_internal.h", "tc_decode.h")
KERNEL_SOURCES = {
    "k_points_ws": ("tc_points.cu",) + _COMMON_SOURCES,
    "k_pages_tc": ("tc_decode.cu",) + _COMMON_SOURCES,
    "k_pages_ws": ("tc_decode.cu",) + _COMMON_SOURCES,
    "k_hybrid_pages_tc": ("hybrid.cu", "hybrid.h", "bc7.cuh") + _COMMON_SOURCES,
    "k_hybrid_pages_tc_bc7": ("hybrid.cu", "hybrid.h", "bc7.cuh") + _COMMON_SOURCES,
}
NCU_TRAFFIC = {
    "k_points_ws": {"src": "dc313c105005e444", "read": 134407936, "write": 81475584, "units": 1 << 23,
                    "profile": "profiles/k_points_ws_points_2048_atlas.md"},
    "k_pages_tc": {"src": "f7fc86e019b63f3e", "read": 19674624, "write": 75905280, "units": 1024 * 128 * 128,
                   "profile": "profiles/k_pages_tc_pages_8_lightmaps.md"},
    "k_pages_ws": {"src": "f7fc86e019b63f3e", "read": 19192576, "write": 76340736, "units": 1024 * 128 * 128,
                   "profile": "profiles/k_pages_ws_pages_8_lightmaps.md"},
    "k_hybrid_pages_tc": {"src": "fef791fc427035db", "read": 187109120, "write": 475889664, "units": 4096 * 128 * 128,
                          "profile": "profiles/k_hybrid_pages_tc_m64_4096_tiles.md"},
    "k_hybrid_pages_tc_bc7": {"src": "fef791fc427035db", "read": 116471296, "write": 475803392, "units": 4096 * 128 * 128,
                              "profile": "profiles/k_hybrid_pages_tc_bc7_m64_4096_tiles.md"},
}


def kernel_source_hash(kernel):
    """Hash of a kernel's source files' code (comments and blank space stripped, so a comment edit keeps the
    figure)."""
    import hashlib
    import re
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_2604_12625_gb300", "csrc", f)) as fh:
            code = fh.read()
        code = re.sub(r"/\*.*?\*/", " ", code, flags=re.S)
        code = re.sub(r"//[^\n]*", " ", code)
        h.update(" ".join(code.split()).encode())
    return h.hexdigest()[:16]


def traffic_for(kernel, units):
    """Scaled ncu DRAM bytes for one launch over `units` texels, or None if the kernel changed since capture."""
    rec = NCU_TRAFFIC.get(kernel)
    if rec is None or rec["src"] != kernel_source_hash(kernel):
        return None
    return (rec["read"] + rec["write"]) * units / rec["units"]


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


def two_term_roofline(units, flop_per_unit, bytes_total, seconds, peaks, peak_kind):
    """Roofline of a decode: t_roof = max(bytes / HBM bandwidth, FLOPs / tensor peak) (both measured peaks).

    Reports the dominant term as bound/achieved/peak and both terms' times beside frac = t_roof / t_measured.
    """
    t_tc = units * flop_per_unit / (peaks["bf16_tflops"] * 1e12)
    t_hbm = bytes_total / (peaks["hbm_gbs"] * 1e9)
    if t_tc >= t_hbm:
        roof = {"bound": "tensor", "achieved": units * flop_per_unit / seconds / 1e12, "peak": peaks["bf16_tflops"],
                "unit": "TFLOP/s", "peak_source": f"{peak_kind} bf16 burst (fp16 has the same dense rate)"}
    else:
        roof = {"bound": "hbm", "achieved": bytes_total / seconds / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "peak_source": f"{peak_kind} HBM copy bandwidth"}
    roof["frac"] = max(t_tc, t_hbm) / seconds
    roof["terms_us"] = {"tensor": t_tc * 1e6, "hbm": t_hbm * 1e6, "measured": seconds * 1e6}
    roof["algorithmic"] = {"flop_per_unit": flop_per_unit, "bytes": bytes_total}
    return roof


def page_frame_bytes(reqs, maps, out_bytes_per_texel=8, block_bytes=None):
    """Algorithmic bytes of a page frame: every output texel once, plus each distinct compressed block the
    requests' bilinear taps touch, once (cs planes x 8 bytes per 4x4 block)."""
    keys = []
    for r in reqs:
        m = maps[int(r["model"])]
        sx, sy = m["feat_w"] / m["lm_w"], m["feat_h"] / m["lm_h"]

        def span(o, n, s, f):
            lo = int(np.floor((o + 0.5) * s - 0.5))
            hi = int(np.floor((o + n - 0.5) * s - 0.5)) + 1
            return max(lo, 0) // 4, min(hi, f - 1) // 4

        bx0, bx1 = span(int(r["x0"]), int(r["w"]), sx, m["feat_w"])
        by0, by1 = span(int(r["y0"]), int(r["h"]), sy, m["feat_h"])
        by, bx = np.meshgrid(np.arange(by0, by1 + 1), np.arange(bx0, bx1 + 1), indexing="ij")
        keys.append((int(r["model"]) << 40) | (by.ravel().astype(np.int64) << 20) | bx.ravel().astype(np.int64))
    nblocks = int(np.unique(np.concatenate(keys)).size)
    cs = int(maps[0]["cs"])
    texels = int(np.sum(reqs["w"].astype(np.int64) * reqs["h"]))
    return texels * out_bytes_per_texel + nblocks * cs * 8


def fp32_alu_peak_tflops(sm_mhz, sms=152):
    # 128 FP32 lanes per SM, one FMA (2 FLOP) per lane per clock
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
            return
        t0 = time.time()
        while time.time() - t0 < 3.0:          # wait for the first sample so the region is covered
            self.f.flush()
            if os.path.getsize(self.f.name) > 0:
                break
            time.sleep(0.01)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.06)
        self.proc.terminate()
        self.proc.wait()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[4 + i].lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
                if any(r[2].replace(".", "").isdigit() for r in rows) else None}


def cpu_cores():
    return len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def time_oracle_one_core(m, q_all, target_s=3.0, min_n=1 << 11):
    """The FP64 oracle on a single host core (queries per second)."""
    import oracle
    n = min_n
    t0 = time.perf_counter()
    oracle.decode_points(m, q_all[:n], nthreads=1)
    dt = time.perf_counter() - t0
    n2 = int(min(q_all.shape[0], max(min_n, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.decode_points(m, q_all[:n2], nthreads=1)
    return n2 / (time.perf_counter() - t0)


def time_oracle(m, q_all, target_s, min_n=1 << 14):
    """Times the FP64 oracle on a bounded prefix of the queries sized for ~target_s seconds."""
    import oracle
    nt = cpu_cores()
    n = min_n
    t0 = time.perf_counter()
    oracle.decode_points(m, q_all[:n], nthreads=nt)
    dt = time.perf_counter() - t0
    n2 = int(min(q_all.shape[0], max(min_n, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.decode_points(m, q_all[:n2], nthreads=nt)
    dt = time.perf_counter() - t0
    return n2 / dt / 1e9, n2, dt, nt


def max_over_ranks(ms, dist, device):
    """The step time every rank reports: the maximum over ranks (weak scaling, replicas)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms_per_step):
    """Whole-job throughput in G units/s: the units all ranks processed over the slowest rank's step time."""
    return world * units_per_rank / (ms_per_step * 1e-3) / 1e9


def rank_query_seed(rank):
    """Each rank decodes its own queries (replicas, no data-path exchange)."""
    return 2 + 1000 * rank


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    m = synth.points_model_2048(2)
    q = synth.random_queries(2, N_QUERIES)
    import oracle
    nt = cpu_cores()
    # size each step so (warmup + steps) steps take about a minute in total
    probe = 1 << 14
    t0 = time.perf_counter()
    oracle.decode_points(m, q[:probe], nthreads=nt)
    per_q = (time.perf_counter() - t0) / probe
    total_steps = max(1, args.steps + args.warmup)
    per_step = int(np.clip(args.ref_seconds / total_steps / max(per_q, 1e-9), 1 << 12, N_QUERIES))
    for w in range(args.warmup):
        oracle.decode_points(m, q[:per_step], nthreads=nt)
    t0 = time.perf_counter()
    for k in range(args.steps):
        off = (k * per_step) % (N_QUERIES - per_step + 1)
        oracle.decode_points(m, q[off:off + per_step], nthreads=nt)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt / 1e9
    sample = f"{per_step} of the 2^24 queries per step (FP64 oracle, OpenMP over {nt} threads)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gtexels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "queries_per_step": per_step},
            "cpu_baseline": {"value": value, "unit": "Gtexels/s", "cores": nt, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "Gtexels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


PAGE_FLOP_PER_TEXEL = 2 * (16 * 64 + 64 * 64 + 64 * 3)   # 10,624: temporal term folded per page
PAGES_WORKLOAD = ("pages: 8 lightmaps (2x 512^2, 1024^2, 2048^2, 4096^2), BC4 half-res x16, temporal 24x8 fp16, "
                  "MLP 24-64-64-3; 4096 Zipf(1.1) requests of 128^2 per frame, own t each; RGBA16F 8192^2 texture")


def check_status(ndgi, model=None, precision=None):
    """'ok', or the library's report of a CUDA error or, for a tensor-core point decode, of a device-side
    failure latched in the model's workspace (e.g. a timed-out barrier wait)."""
    try:
        ndgi.ndgi_check()
        if model is not None and precision in ("fp16", "bf16"):
            st, word = ndgi.ndgi_workspace_check(model, precision)
            if st != 0:
                return f"workspace error word 0x{word:x} (status {st})"
        return "ok"
    except Exception as ex:  # reported in the JSON line, never hidden
        return str(ex)[:200]


def page_kernel(plan_shape):
    """Name of the tensor-core page kernel a plan shape (precision, ctas/SM, lanes, slots) runs."""
    return "k_pages_ws" if tuple(plan_shape)[2:] == (8, 1) else "k_pages_tc"


def bench_pages(args, ndgi, torch, peaks, peak_kind, timed, rank, check_err=True):
    """Virtual-texture page decode: one step = one frame of 4096 page requests."""
    maps = synth.page_models(4)
    models = [ndgi.Model.from_arrays(m) for m in maps]
    reqs = synth.zipf_page_requests(4, synth.PAGE_LIGHTMAP_SIZES, args.page_requests, page=128, slots_x=64)
    r_dev, n_dev = ndgi.page_requests_to_device(reqs)
    phys = torch.empty((8192, 8192, 4), dtype=torch.float16, device="cuda")
    texels = int(len(reqs)) * 128 * 128
    out = {}
    for prec in ("fp16", "fp32"):
        plan = ndgi.PagesPlan(models, prec, len(reqs), phys)
        if prec != "fp32" and args.page_shape:
            plan.set_shape(1, *args.page_shape)
        else:
            plan.autotune(r_dev, n_dev, len(reqs))
        steps = args.steps if prec == "fp16" else max(3, min(args.steps, 10))
        ms, clocks = timed(lambda: plan.decode(r_dev, n_dev), steps, args.warmup, sample_clocks=(prec == "fp16"))
        st, err_word = plan.check()
        entry = {"value": job_value(texels, args.world, ms / steps), "unit": "Gtexels/s", "ms_per_frame": ms / steps,
                 "device_error_word": err_word, "device_check": check_status(ndgi), "plan_shape": plan.info()}
        if prec == "fp16":
            entry["clocks"] = clocks
            scratch = torch.empty(1 << 28, dtype=torch.float32, device="cuda")   # 1 GiB, written before each frame
            med = args.per_step_median(lambda: plan.decode(r_dev, n_dev), 20, flush=lambda: scratch.fill_(1.0))
            entry["cold_l2"] = {"ms_per_frame_median_of_20": med, "value": job_value(texels, args.world, med),
                                "unit": "Gtexels/s", "flush": "1 GiB scratch write before each frame"}
            entry["warm_ms_per_frame_median_of_20"] = args.per_step_median(lambda: plan.decode(r_dev, n_dev), 20)
            del scratch
        if check_err and rank == 0:
            import oracle
            pick = np.random.default_rng(5).choice(len(reqs), 12, replace=False)
            sub = reqs[pick]
            got = phys.float().cpu().numpy()
            ref = oracle.decode_pages(maps, sub, 8192, 8192, precision="fp16" if prec == "fp16" else "fp32",
                                      fill=0.0)
            worst = 0.0
            for q in sub:
                sl = (slice(q["dst_y"], q["dst_y"] + 128), slice(q["dst_x"], q["dst_x"] + 128))
                a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
                worst = max(worst, float(np.abs(a - b).max() / (b.max() - b.min())))
            entry["max_err_over_page_range"] = worst
            entry["err_sample"] = "12 seeded requests, per-page range; RGBA16F storage rounding included"
        out[prec] = entry
        plan.close()
    kernel_s = out["fp16"]["ms_per_frame"] * 1e-3
    kernel = page_kernel(out["fp16"]["plan_shape"])
    traffic = traffic_for(kernel, texels)
    out["roofline"] = two_term_roofline(texels, PAGE_FLOP_PER_TEXEL, page_frame_bytes(reqs, maps), kernel_s,
                                        peaks, peak_kind)
    out["roofline"].update({"traffic": traffic, "kernel": kernel, "flop_per_texel": PAGE_FLOP_PER_TEXEL})
    if traffic is not None:
        out["roofline"]["traffic_note"] = ("ncu DRAM bytes of a 1024-request frame scaled by texels; output lines "
                                           "still dirty in L2 at kernel end are not counted")
    out["workload"] = PAGES_WORKLOAD.replace("4096 Zipf", f"{args.page_requests} Zipf")
    out["texels_per_frame"] = texels
    return out


FIT_WORKLOAD = ("fit: 1024^2 x T=24 FP16 keyframe targets (32 Gaussians x sun term + 0.05), straight-through BC4 "
                "512^2x16 features, temporal 24x8, MLP 24-64-64-3, Adam lr 1e-2, 2^20 samples/step of (texel, t) "
                "with t ~ U[0,1) (temporal lerp differentiated; targets interpolated between keyframes), 2000 steps "
                "(last 200 freeze the features)")


_C3_TARGETS = []


def c3_targets():
    """The fit workload's keyframe targets (generated once per run)."""
    if not _C3_TARGETS:
        _C3_TARGETS.append(synth.fit_targets(3, 1024, 1024, 24))
    return _C3_TARGETS[0]


def bench_fit(args, ndgi, torch):
    """Differentiation: the full 2000-step fit, timed end to end on the device."""
    targets = c3_targets()
    p = synth.fit_init(3, 512, 512, 16, 24, 8, 64)
    st = ndgi.FitState.from_arrays(p, 1024, 1024)
    tg = torch.from_numpy(targets).cuda()
    batch, steps = 1 << 20, args.fit_steps
    # warm-up (graph capture, kernel load) on a throw-away copy of the parameters
    warm = ndgi.FitState({k: v.clone() for k, v in st.t.items()}, 1024, 1024)
    ndgi.ndgi_encode_fit(warm, tg, ndgi.fit_config(steps=3, batch=batch, seed=1))
    torch.cuda.synchronize()
    cfg = ndgi.fit_config(steps=steps, batch=batch, lr=1e-2, freeze_steps=steps // 10,
                          loss_every=max(1, min(100, steps // 4)), seed=7)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, log = ndgi.ndgi_encode_fit(st, tg, cfg)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    log = log.cpu().numpy()
    rng = float(targets.max()) - float(targets.min())
    return {"workload": FIT_WORKLOAD.replace("2000 steps", f"{steps} steps"), "steps": steps, "batch": batch, "seconds": ms / 1e3,
            "ms_per_step": ms / steps, "samples_per_s": steps * batch / (ms / 1e3),
            "loss_first": float(log[0]), "loss_last": float(log[-1]),
            "loss_every": cfg.loss_every, "loss_log": [float(x) for x in log],
            "psnr_db_last": float(10 * np.log10(rng * rng / max(log[-1], 1e-30))),
            "scope": "one rank (under torchrun every rank fits its own replica; no gradient exchange)",
            "device_check": check_status(ndgi)}


FIT_BATCH_WORKLOAD = ("per-tile fit: the fit workload's 1024^2 x T=24 targets cut into 256 tiles of 64^2, one model "
                      "per tile (BC4 32^2x16, temporal 24x8, MLP 24-64-64-3), all 256 fitted in one launch per "
                      "step, 2^12 samples per model and step (2^20 in all), Adam lr 1e-2, 500 steps")


def bench_fit_batch(args, ndgi, torch):
    """Batched per-tile fit: 256 tile models side by side (ndgi_encode_fit_batch)."""
    tiles, side, T = 16, 64, 24
    full = c3_targets()
    tg = full.reshape(T, tiles, side, tiles, side, 3).transpose(1, 3, 0, 2, 4, 5).reshape(tiles * tiles, T, side,
                                                                                         side, 3)
    tg = torch.from_numpy(np.ascontiguousarray(tg)).cuda()
    ps = [synth.fit_init(300 + i, 32, 32, 16, T, 8, 64) for i in range(tiles * tiles)]
    steps = max(10, min(500, args.fit_steps // 4))
    warm = ndgi.FitBatch.from_arrays(ps[:2], side, side)
    ndgi.ndgi_encode_fit_batch(warm, tg[:2].contiguous(), ndgi.fit_config(steps=2, batch=1 << 12, seed=1))
    fb = ndgi.FitBatch.from_arrays(ps, side, side)
    cfg = ndgi.fit_config(steps=steps, batch=1 << 12, lr=1e-2, freeze_steps=steps // 10,
                          loss_every=max(1, steps // 5), seed=8)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, log = ndgi.ndgi_encode_fit_batch(fb, tg, cfg)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    log = log.cpu().numpy()
    rng = float(full.max()) - float(full.min())
    return {"workload": FIT_BATCH_WORKLOAD.replace("500 steps", f"{steps} steps"), "models": tiles * tiles,
            "steps": steps, "ms_per_step": ms / steps, "samples_per_s": steps * (1 << 12) * tiles * tiles / (ms / 1e3),
            "loss_first": float(log[0]), "loss_last": float(log[-1]),
            "psnr_db_last": float(10 * np.log10(rng * rng / max(log[-1], 1e-30))), "device_check": check_status(ndgi)}


HYBRID_FIT_WORKLOAD = ("hybrid fit: one M.64 tile model (F_uv 128^2x4 and F3D 32^2x12x4 as BC endpoints + weights "
                       "under the straight-through BC simulation: four BC4 planes with a weight per channel, or "
                       "Eq. 7's weight per texel shared by the channels read as BC7's single-subset interpolation; "
                       "F_ut/F_vt 64x24x2, GELU MLP 16-64-64-3) against the top-left 128^2 crop of the fit "
                       "workload's 24 keyframe targets; 1000 Adam steps of 2^16 samples at t ~ U[0,1) (targets "
                       "interpolated between keyframes); then the maps quantised to 8 bits and BC7-compressed, "
                       "F_ut/F_vt to UNORM8, and every keyframe decoded (FP32) and scored")


def _bc7_export(ndgi, torch, uv8, vol8, vol_t, vol_side):
    """BC7 blocks of the 8-bit maps (F3D slices stacked along the height), their squared error and encode time."""
    sq = torch.zeros(2, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    uv7 = ndgi.ndgi_bc7_encode(uv8, sq_err=sq[0:1])
    vol7 = ndgi.ndgi_bc7_encode(vol8, sq_err=sq[1:2]).reshape(vol_t, vol_side // 4, vol_side // 4, 16).contiguous()
    e1.record(stream)
    e1.synchronize()
    n = uv8.numel() + vol8.numel()
    return uv7, vol7, float(np.sqrt(float(sq.sum().item()) / n)), e0.elapsed_time(e1), n // 64


def bench_hybrid_fit(args, ndgi, torch):
    """The hybrid decoder's fit (ndgi_hybrid_encode_fit) with both BC simulations, then the paper's export (8-bit
    maps BC7-compressed) decoded at every keyframe."""
    T, side = 24, 128
    tg = torch.from_numpy(np.ascontiguousarray(c3_targets()[:, :side, :side])).cuda()
    ref = tg.float()
    rng = float(ref.max() - ref.min())
    vol_side, vol_t, hidden = 32, 12, 64
    steps = max(20, min(1000, args.fit_steps // 2))
    batch = 1 << 16
    keys = np.arange(T, dtype=np.float32) / T
    q = torch.from_numpy(synth.texel_queries(side, side, keys)).cuda().reshape(-1, 3)
    mlp = ("w1", "b1", "w2", "b2", "w3", "b3")

    def psnr(hm):
        rgb = ndgi.ndgi_hybrid_decode_points(hm, q, "fp32").reshape(T, side, side, 3)
        return float(10 * np.log10(rng * rng / max(float(((rgb - ref) ** 2).mean()), 1e-30)))

    out = {"workload": HYBRID_FIT_WORKLOAD.replace("1000 Adam", f"{steps} Adam"), "steps": steps}
    for name, shared, noise in (("bc4x4", False, 0.0), ("eq7_shared_weight", True, 0.0),
                                ("eq7_shared_weight_noise", True, 1.0 / 256)):
        p = synth.hybrid_fit_init(21, side, side, side, side, vol_side, vol_side, vol_t, 64, 24, 64, 24, hidden,
                                  shared_w=shared)
        warm = ndgi.HybridFitState.from_arrays(p)
        ndgi.ndgi_hybrid_encode_fit(warm, tg, ndgi.fit_config(steps=2, batch=batch, seed=1))
        st = ndgi.HybridFitState.from_arrays(p)
        cfg = ndgi.fit_config(steps=steps, batch=batch, lr=1e-2, freeze_steps=steps // 10,
                              loss_every=max(1, steps // 5), seed=22, noise_alpha=noise)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, log = ndgi.ndgi_hybrid_encode_fit(st, tg, cfg)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        log = log.cpu().numpy()
        t = st.t
        ut = torch.round(t["ut"] * 255).to(torch.uint8)
        vt = torch.round(t["vt"] * 255).to(torch.uint8)
        entry = {"noise_alpha": noise, "ms_per_step": ms / steps, "samples_per_s": steps * batch / (ms / 1e3),
                 "loss_first": float(log[0]), "loss_last": float(log[-1]),
                 "psnr_db_fit": float(10 * np.log10(rng * rng / max(log[-1], 1e-30)))}
        if shared:
            # exact: the maps are mode-6 blocks
            hm6 = ndgi.HybridModel(side, side, ndgi.ndgi_bc7_pack_sim(t["uv_ea"], t["uv_eb"], t["uv_wt"]),
                                   ndgi.ndgi_bc7_pack_sim(t["vol_ea"], t["vol_eb"], t["vol_wt"]), ut, vt,
                                   *[t[k] for k in mlp])
            entry["psnr_db_mode6_pack_decode"] = psnr(hm6)
            entry["bpp_bc7"] = ndgi.ndgi_model_bpp(hm6, 1, 0, 16)
            uv8 = ndgi.ndgi_bc_sim7_to_rgba8(t["uv_ea"], t["uv_eb"], t["uv_wt"])
            vol8 = ndgi.ndgi_bc_sim7_to_rgba8(t["vol_ea"], t["vol_eb"], t["vol_wt"])
            export = "the shared-weight simulation's 8-bit texels (ndgi_bc_sim7_to_rgba8), then ndgi_bc7_encode"
        else:
            uv = ndgi.ndgi_bc_pack(t["uv_ea"], t["uv_eb"], t["uv_wt"])
            vol = torch.stack([ndgi.ndgi_bc_pack(t["vol_ea"][k].contiguous(), t["vol_eb"][k].contiguous(),
                                                 t["vol_wt"][k].contiguous()) for k in range(vol_t)]).contiguous()
            hm = ndgi.HybridModel(side, side, uv, vol, ut, vt, *[t[k] for k in mlp])
            entry["psnr_db_bc4x4_decode"] = psnr(hm)
            entry["bpp_bc4x4"] = ndgi.ndgi_model_bpp(hm, 1, 0, 16)
            uv8 = ndgi.ndgi_bc4x4_to_rgba8(uv)
            vol8 = torch.cat([ndgi.ndgi_bc4x4_to_rgba8(vol[k].contiguous()) for k in range(vol_t)], 0)
            export = "BC4-simulated values rounded to 8 bits (ndgi_bc4x4_to_rgba8), then ndgi_bc7_encode"
        uv7, vol7, rms, enc_ms, nblk = _bc7_export(ndgi, torch, uv8, vol8, vol_t, vol_side)
        hm7 = ndgi.HybridModel(side, side, uv7, vol7, ut, vt, *[t[k] for k in mlp])
        entry["bc7_export"] = {"psnr_db_decode": psnr(hm7), "bpp": ndgi.ndgi_model_bpp(hm7, 1, 0, 16),
                               "rms_8bit_levels": rms, "encode_ms": enc_ms,
                               "encode_blocks_per_s": nblk / (enc_ms / 1e3), "export": export}
        out[name] = entry
    out["device_check"] = check_status(ndgi)
    return out


HYBRID_FIT_BATCH_WORKLOAD = ("batched hybrid fit: the fit workload's 1024^2 x 24 keyframe targets cut into 64 tiles "
                             "of 128^2, one M.64 model per tile (Eq. 7 shared-weight BC7 mode-6 simulation, noise "
                             "1/256), all 64 fitted in one launch per step, 2^13 samples per model and step, 300 "
                             "Adam steps; then every tile packed exactly to BC7, F_ut/F_vt to UNORM8, and the whole "
                             "1024^2 lightmap decoded (FP32 page decode, one 128^2 page per tile) at every keyframe")


def bench_hybrid_fit_batch(args, ndgi, torch):
    """Per-tile hybrid models fitted side by side (ndgi_hybrid_encode_fit_batch), then the lightmap decoded from
    their exact BC7 packs."""
    T, side, tiles = 24, 128, 8
    full = c3_targets()
    tg = full.reshape(T, tiles, side, tiles, side, 3).transpose(1, 3, 0, 2, 4, 5).reshape(tiles * tiles, T, side,
                                                                                         side, 3)
    tg = torch.from_numpy(np.ascontiguousarray(tg)).cuda()
    ps = [synth.hybrid_fit_init(500 + i, side, side, side, side, 32, 32, 12, 64, 24, 64, 24, 64, shared_w=True)
          for i in range(tiles * tiles)]
    steps = max(10, min(300, args.fit_steps // 6))
    batch = 1 << 13
    warm = ndgi.HybridFitBatch.from_arrays(ps[:2])
    ndgi.ndgi_hybrid_encode_fit_batch(warm, tg[:2].contiguous(), ndgi.fit_config(steps=2, batch=batch, seed=1))
    fb = ndgi.HybridFitBatch.from_arrays(ps)
    cfg = ndgi.fit_config(steps=steps, batch=batch, lr=1e-2, freeze_steps=steps // 10, loss_every=max(1, steps // 5),
                          seed=23, noise_alpha=1.0 / 256)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    _, log = ndgi.ndgi_hybrid_encode_fit_batch(fb, tg, cfg)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    log = log.cpu().numpy()
    t = fb.t
    uv = ndgi.ndgi_bc7_pack_sim(t["uv_ea"], t["uv_eb"], t["uv_wt"])
    vol = ndgi.ndgi_bc7_pack_sim(t["vol_ea"], t["vol_eb"], t["vol_wt"])
    ut = torch.round(t["ut"] * 255).to(torch.uint8)
    vt = torch.round(t["vt"] * 255).to(torch.uint8)
    models = [ndgi.HybridModel(side, side, uv[i], vol[i], ut[i], vt[i],
                               *[t[k][i] for k in ("w1", "b1", "w2", "b2", "w3", "b3")]) for i in range(tiles * tiles)]
    table = ndgi.HybridTable(models, "fp32")
    phys = torch.zeros((tiles * side, tiles * side, 4), dtype=torch.float32, device="cuda")
    mse = 0.0
    for j in range(T):
        reqs = np.zeros(tiles * tiles, dtype=synth.PAGE_REQ_DTYPE)
        for i in range(tiles * tiles):
            reqs[i] = (i, 0, 0, side, side, np.float32(j / T), (i % tiles) * side, (i // tiles) * side)
        r, _ = ndgi.page_requests_to_device(reqs)
        table.decode(r, len(reqs), phys)
        mse += float(((phys[..., :3] - torch.from_numpy(full[j]).cuda().float()) ** 2).mean()) / T
    table.close()
    rng = float(full.max()) - float(full.min())
    return {"workload": HYBRID_FIT_BATCH_WORKLOAD.replace("300 Adam", f"{steps} Adam"), "models": tiles * tiles,
            "steps": steps, "ms_per_step": ms / steps, "samples_per_s": steps * batch * tiles * tiles / (ms / 1e3),
            "loss_first": float(log[0]), "loss_last": float(log[-1]),
            "psnr_db_fit": float(10 * np.log10(rng * rng / max(log[-1], 1e-30))),
            "psnr_db_bc7_decode_1024": float(10 * np.log10(rng * rng / max(mse, 1e-30))),
            "bpp_bc7_per_tile": ndgi.ndgi_model_bpp(models[0], 1, 0, 16), "device_check": check_status(ndgi)}


QUALITY_WORKLOAD = ("quality: 256^2 lightmap, 26 non-uniform keyframes (24 hourly + 2 around a light switch at "
                    "t = 0.73; a lamp on for 0.73 <= t < 0.9), UV-chart mask (~70% valid); BC4 128^2x16, temporal "
                    "26x8, MLP 24-64-64-3; 1500 Adam steps of 2^18 samples, with BC simulation (STE) and without it "
                    "(relaxed, then packed to BC4); every keyframe decoded (FP32) and scored with the tiled "
                    "mask-aware PSNR/SSIM (128^2 tiles, per-tile range)")


def bench_quality(args, ndgi, torch):
    """The BC-simulation ablation on switch-event targets, scored with the paper's tiled mask-aware metrics."""
    W = H = 256
    keys = synth.switch_key_times()
    T = len(keys)
    targets = synth.fit_targets_at_times(11, W, H, keys)
    mask = synth.lightmap_mask(12, W, H)
    tg = torch.from_numpy(targets).cuda()
    ref = tg.float().contiguous()
    mk = torch.from_numpy(np.repeat(mask[None], T, 0)).cuda()
    key_dev = torch.from_numpy(keys).cuda()
    q = torch.from_numpy(synth.texel_queries(W, H, keys)).cuda()     # [T][H][W] texel centres at each keyframe
    steps = max(20, min(1500, args.fit_steps))
    out = {"workload": QUALITY_WORKLOAD.replace("1500 Adam", f"{steps} Adam"), "key_t": [float(k) for k in keys]}
    for name, relaxed in (("bc_simulation", False), ("without_bc_simulation", True)):
        p = synth.fit_init(13, 128, 128, 16, T, 8, 64)
        st = ndgi.FitState.from_arrays(p, W, H)
        st = ndgi.FitState(st.t, W, H, 0, key_dev)
        cfg = ndgi.fit_config(steps=steps, batch=1 << 18, lr=1e-2, freeze_steps=steps // 10, seed=14, relaxed=relaxed)
        ndgi.ndgi_encode_fit(st, tg, cfg)
        bc4 = ndgi.ndgi_bc_pack(st.t["ea"], st.t["eb"], st.t["w"])
        model = ndgi.Model(W, H, bc4, st.t["temporal"], *[st.t[k] for k in ("w1", "b1", "w2", "b2", "w3", "b3")],
                           0, key_dev)
        rgb = ndgi.ndgi_decode_points(model, q, "fp32").reshape(T, H, W, 3)
        ps, ss = ndgi.ndgi_tile_metrics(rgb, ref, mk, tile=128)
        ps, ss = ps.cpu().numpy(), ss.cpu().numpy()
        ok_p, ok_s = np.isfinite(ps), np.isfinite(ss)
        near = [int(np.searchsorted(keys, 0.73)) - 1, int(np.searchsorted(keys, 0.73))]
        out[name] = {"psnr_db": float(ps[ok_p].mean()), "ssim": float(ss[ok_s].mean()),
                     "psnr_db_switch_keyframes": float(ps[near][np.isfinite(ps[near])].mean()),
                     "tiles": int(ok_p.sum())}
    out["psnr_drop_without_bc_simulation_db"] = out["bc_simulation"]["psnr_db"] - \
        out["without_bc_simulation"]["psnr_db"]
    out["device_check"] = check_status(ndgi)
    return out


SCALE_WORKLOAD = ("scale: 16384^2 atlas (268M texels) decoded at one t per frame as 128^2 pages; BC4 8192^2x16 "
                  "(512 MiB), temporal 48x16 fp16, MLP 32-64-64-3 in FP16, FP8 E4M3 (per-layer power-of-two "
                  "scales) and FP32; RGBA16F 16384^2 texture")


def bench_scale(args, ndgi, torch, peaks, peak_kind, timed, rank):
    m = synth.model(5, 16384, 16384, 8192, 8192, 16, 48, 16, 64, temporal_dtype="f16")
    model = ndgi.Model.from_arrays(m)
    n_side = 128
    reqs = np.zeros(n_side * n_side, dtype=synth.PAGE_REQ_DTYPE)
    for i in range(n_side * n_side):
        x0, y0 = (i % n_side) * 128, (i // n_side) * 128
        reqs[i] = (0, x0, y0, 128, 128, np.float32(0.37), x0, y0)
    r_dev, n_dev = ndgi.page_requests_to_device(reqs)
    phys = torch.empty((16384, 16384, 4), dtype=torch.float16, device="cuda")
    texels = 16384 * 16384
    out = {"workload": SCALE_WORKLOAD, "texels_per_frame": texels}
    act_max = None
    for prec in ("fp16", "fp8", "fp32"):
        if prec == "fp8":
            # per-layer FP8 scales from the library's own FP32 calibration pass over 2^16 seeded queries
            cal = torch.from_numpy(synth.random_queries(7, 1 << 16)).cuda()
            act_max = ndgi.ndgi_calibrate_fp8(model, cal).cpu().numpy().astype(np.float64)
            ndgi.ndgi_prepare_fp8(model, act_max)
        plan = ndgi.PagesPlan([model], prec, len(reqs), phys)
        if prec != "fp32" and args.page_shape:
            plan.set_shape(1, *args.page_shape)
        elif prec != "fp32":
            plan.autotune(r_dev, n_dev, len(reqs))
        steps = max(3, min(args.steps, 10)) if prec != "fp32" else 3
        ms, _ = timed(lambda: plan.decode(r_dev, n_dev), steps, 2)
        entry = {"value": job_value(texels, args.world, ms / steps), "unit": "Gtexels/s", "ms_per_frame": ms / steps,
                 "device_check": check_status(ndgi), "plan_shape": plan.info()}
        if rank == 0:
            import oracle
            pick = np.random.default_rng(6).choice(len(reqs), 3, replace=False)
            sub = reqs[pick]
            got = phys.float().cpu().numpy()
            refs = {"oracle": oracle.decode_pages([m], sub, 16384, 16384, precision=prec, fill=0.0,
                                                  act_max=None if act_max is None else act_max[None])}
            if prec == "fp8":
                refs["fp32_master"] = oracle.decode_pages([m], sub, 16384, 16384, precision="fp32", fill=0.0)
            for key, ref in refs.items():
                worst = rms = 0.0
                for q in sub:
                    sl = (slice(q["dst_y"], q["dst_y"] + 128), slice(q["dst_x"], q["dst_x"] + 128))
                    a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
                    rng_ = b.max() - b.min()
                    worst = max(worst, float(np.abs(a - b).max() / rng_))
                    rms = max(rms, float(np.sqrt(((a - b) ** 2).mean()) / rng_))
                name = "max_err_over_page_range" if key == "oracle" else "vs_fp32_master_max_err"
                entry[name] = worst
                entry[name.replace("max_err", "rms_err")] = rms
            if prec == "fp8":
                entry["act_max"] = act_max.tolist()
                entry["err_note"] = ("oracle = the FP8 decode with the same scales (E4M3 rounding of activations "
                                     "computed in different arithmetic may flip); fp32_master = the unquantised model")
        out[prec] = entry
        plan.close()
    out["roofline"] = two_term_roofline(texels, PAGE_FLOP_PER_TEXEL, page_frame_bytes(reqs, [m]),
                                        out["fp16"]["ms_per_frame"] * 1e-3, peaks, peak_kind)
    out["roofline"]["kernel"] = page_kernel(out["fp16"]["plan_shape"])
    del phys
    torch.cuda.empty_cache()
    return out


HYBRID_WORKLOAD = ("hybrid pages: 4096 tile models of the paper's M.64 profile (F_uv 128^2x4 and F3D 32^2x12x4 as "
                   "BC4 planes, F_ut/F_vt 64x24x2 UNORM8, gamma(t), MLP 16-64-64-3 GELU), one frame = 4096 whole "
                   "128^2 tile pages, each its own uniform tile and t ~ U[0,1); RGBA16F 8192^2 texture")
HYBRID_FLOP_PER_TEXEL = 2 * (16 * 64 + 64 * 64 + 64 * 3)   # 10,624


def hybrid_frame_bytes(n_req, n_models_touched, model_bytes, out_bytes_per_texel=8):
    """Algorithmic DRAM bytes of one hybrid frame: each touched model once plus the output texels."""
    return n_models_touched * model_bytes + n_req * 128 * 128 * out_bytes_per_texel


def bench_hybrid(args, ndgi, torch, peaks, peak_kind, timed, rank):
    """The paper's full decoder over per-tile models: one step = one frame of 4096 tile pages."""
    s = synth.hybrid_tile_set(90, 4096, "M.64")
    models = ndgi.HybridModel.from_set(s)
    reqs = synth.hybrid_tile_requests(91, 4096, 4096, slots_x=64)
    r_dev, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.empty((8192, 8192, 4), dtype=torch.float16, device="cuda")
    texels = len(reqs) * 128 * 128
    out = {"workload": HYBRID_WORKLOAD, "texels_per_frame": texels}
    for prec in ("fp16", "fp32"):
        ndgi.hybrid_prepare_set(models, prec)
        table = ndgi.HybridTable(models, prec)
        steps = max(3, min(args.steps, 20)) if prec == "fp16" else 3
        ms, clocks = timed(lambda: table.decode(r_dev, len(reqs), phys), steps, 2, sample_clocks=(prec == "fp16"))
        st, word = table.check()
        entry = {"value": job_value(texels, args.world, ms / steps), "unit": "Gtexels/s", "ms_per_frame": ms / steps,
                 "device_error_word": word, "device_check": "ok" if st == 0 else f"status {st}"}
        if prec == "fp16":
            entry["clocks"] = clocks
        if rank == 0:
            import oracle
            pick = np.random.default_rng(93).choice(len(reqs), 4, replace=False)
            used = sorted(set(int(reqs[i]["model"]) for i in pick))
            remap = {mi: k for k, mi in enumerate(used)}
            sub = reqs[pick].copy()
            sub["model"] = [remap[int(mi)] for mi in sub["model"]]
            ref = oracle.hybrid_decode_pages([synth.hybrid_tile_of(s, mi) for mi in used], sub, 8192, 8192,
                                             precision=prec, fill=0.0)
            got = phys.float().cpu().numpy()
            worst = 0.0
            for q in sub:
                sl = (slice(q["dst_y"], q["dst_y"] + 128), slice(q["dst_x"], q["dst_x"] + 128))
                a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
                worst = max(worst, float(np.abs(a - b).max() / (b.max() - b.min())))
            entry["max_err_over_page_range"] = worst
            entry["err_sample"] = "4 seeded requests, per-page range; RGBA16F storage rounding included"
        out[prec] = entry
        table.close()
    m0 = s
    model_bytes = sum(int(np.prod(m0[k].shape[1:])) * m0[k].itemsize for k in ("uv_bc4", "vol_bc4", "ut", "vt")) + \
        sum(int(np.prod(m0[k].shape[1:])) * 2 for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    touched = len(set(int(x) for x in reqs["model"]))
    out["roofline"] = two_term_roofline(texels, HYBRID_FLOP_PER_TEXEL, hybrid_frame_bytes(len(reqs), touched,
                                        model_bytes), out["fp16"]["ms_per_frame"] * 1e-3, peaks, peak_kind)
    out["roofline"].update({"kernel": "k_hybrid_pages_tc", "flop_per_texel": HYBRID_FLOP_PER_TEXEL,
                            "models_touched": touched, "traffic": traffic_for("k_hybrid_pages_tc", texels)})
    out["vs_fp32_plain"] = out["fp16"]["value"] / out["fp32"]["value"]
    # the same frame with the paper's BC7 maps (random blocks, every mode equally likely), FP16 tensor cores
    s7 = synth.hybrid_tile_set(94, 4096, "M.64", feat_format=1)
    models7 = ndgi.HybridModel.from_set(s7)
    ndgi.hybrid_prepare_set(models7, "fp16")
    table = ndgi.HybridTable(models7, "fp16")
    steps = max(3, min(args.steps, 20))
    ms, _ = timed(lambda: table.decode(r_dev, len(reqs), phys), steps, 2)
    st, word = table.check()
    entry = {"value": job_value(texels, args.world, ms / steps), "unit": "Gtexels/s", "ms_per_frame": ms / steps,
             "device_error_word": word, "device_check": "ok" if st == 0 else f"status {st}",
             "maps": "F_uv 128^2 and F3D 32^2x12 as BC7 (16 B per 4x4 block, modes uniform)"}
    if rank == 0:
        import oracle
        pick = np.random.default_rng(95).choice(len(reqs), 4, replace=False)
        used = sorted(set(int(reqs[i]["model"]) for i in pick))
        remap = {mi: k for k, mi in enumerate(used)}
        sub = reqs[pick].copy()
        sub["model"] = [remap[int(mi)] for mi in sub["model"]]
        ref = oracle.hybrid_decode_pages([synth.hybrid_tile_of(s7, mi) for mi in used], sub, 8192, 8192,
                                         precision="fp16", fill=0.0)
        got = phys.float().cpu().numpy()
        worst = 0.0
        for q in sub:
            sl = (slice(q["dst_y"], q["dst_y"] + 128), slice(q["dst_x"], q["dst_x"] + 128))
            a, b = got[sl][..., :3].astype(np.float64), ref[sl][..., :3]
            worst = max(worst, float(np.abs(a - b).max() / (b.max() - b.min())))
        entry["max_err_over_page_range"] = worst
    bytes7 = sum(int(np.prod(s7[k].shape[1:])) * s7[k].itemsize for k in ("uv_bc7", "vol_bc7", "ut", "vt")) + \
        sum(int(np.prod(s7[k].shape[1:])) * 2 for k in ("w1", "b1", "w2", "b2", "w3", "b3"))
    entry["roofline"] = two_term_roofline(texels, HYBRID_FLOP_PER_TEXEL, hybrid_frame_bytes(len(reqs), touched,
                                          bytes7), ms / steps * 1e-3, peaks, peak_kind)
    entry["roofline"].update({"kernel": "k_hybrid_pages_tc (BC7 instantiation)",
                              "traffic": traffic_for("k_hybrid_pages_tc_bc7", texels)})
    out["fp16_bc7"] = entry
    # the paper's full configuration: BC7 maps in, the 8-bit 4-channel physical texture out
    phys8 = torch.empty((8192, 8192, 4), dtype=torch.uint8, device="cuda")
    ms8, _ = timed(lambda: table.decode(r_dev, len(reqs), phys8), steps, 2)
    st8, word8 = table.check()
    e8 = {"value": job_value(texels, args.world, ms8 / steps), "unit": "Gtexels/s", "ms_per_frame": ms8 / steps,
          "device_check": "ok" if st8 == 0 else f"status {st8}", "output": "RGBA8 UNORM 8192^2 (4 B per texel)"}
    e8["roofline"] = two_term_roofline(texels, HYBRID_FLOP_PER_TEXEL,
                                       hybrid_frame_bytes(len(reqs), touched, bytes7, out_bytes_per_texel=4),
                                       ms8 / steps * 1e-3, peaks, peak_kind)
    out["fp16_bc7_rgba8"] = e8
    del phys8
    table.close()
    del models7, s7
    del phys
    torch.cuda.empty_cache()
    return out


# The paper's decompression table: a 1024^2 lightmap decoded in 0.201 / 0.203 / 0.314 ms (L / M / M.64) on an
# RTX 4060 (context: other hardware)
PAPER_DECODE_MS = {"L": 0.201, "M": 0.203, "M.64": 0.314}


def bench_hybrid_profiles(args, ndgi, torch, timed):
    """The paper's decompression measurement: one 1024^2 lightmap (8 x 8 tiles of 128^2, one model per tile) of
    each profile decoded per frame, submitted as 256 pages of 64^2, FP16 tensor cores, RGBA16F."""
    out = {"workload": "1024^2 lightmap = 8x8 tile models of 128^2 (F_uv 128^2x4, F_ut/F_vt 64x24x2, F3D RxRx12x4), "
                       "decoded at one t per frame as 256 pages of 64^2; FP16 tensor cores; RGBA16F 1024^2"}
    reqs = np.zeros(256, dtype=synth.PAGE_REQ_DTYPE)
    for i in range(256):
        tx, ty, qx, qy = (i // 4) % 8, (i // 4) // 8, (i % 4) % 2, (i % 4) // 2
        reqs[i] = (ty * 8 + tx, 64 * qx, 64 * qy, 64, 64, np.float32(0.37), 128 * tx + 64 * qx, 128 * ty + 64 * qy)
    r_dev, _ = ndgi.page_requests_to_device(reqs)
    phys = torch.empty((1024, 1024, 4), dtype=torch.float16, device="cuda")
    for prof in ("L", "M", "H", "M.64"):
        s_ = synth.hybrid_tile_set(400, 64, prof)
        models = ndgi.HybridModel.from_set(s_)
        ndgi.hybrid_prepare_set(models, "fp16")
        table = ndgi.HybridTable(models, "fp16")
        steps = max(10, min(args.steps, 100))
        ms, _ = timed(lambda: table.decode(r_dev, len(reqs), phys), steps, 3)
        st, word = table.check()
        out[prof] = {"ms_per_frame": ms / steps, "gtexels_s": (1 << 20) / (ms / steps * 1e-3) / 1e9,
                     "paper_rtx4060_ms": PAPER_DECODE_MS.get(prof), "device_check": "ok" if st == 0 else f"status {st}"}
        table.close()
    del phys
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="auto", choices=["auto", "fp16", "bf16", "fp32"])
    ap.add_argument("--no-pages", action="store_true", help="skip the page-decode measurement")
    ap.add_argument("--no-extra", action="store_true", help="skip the fit and scale measurements")
    ap.add_argument("--no-scale", action="store_true", help="skip the 16384^2 scale frame")
    ap.add_argument("--no-hybrid", action="store_true", help="skip the hybrid-decoder page frame")
    ap.add_argument("--fit-steps", type=int, default=2000, help="fit steps (2000 = the fit workload)")
    ap.add_argument("--queries-log2", type=int, default=24,
                    help="point queries per step = 2^this (24 = the headline workload; smaller for profiling)")
    ap.add_argument("--ref-seconds", type=float, default=60.0,
                    help="reference arm: seconds of oracle work over the warm-up and timed steps")
    ap.add_argument("--page-requests", type=int, default=4096,
                    help="page requests per frame (4096 = the page workload; smaller for profiling)")
    ap.add_argument("--e2e-chunk", type=int, default=1 << 20,
                    help="queries per chunk of the host-buffer decode in the e2e measurement")
    ap.add_argument("--page-shape", default=None,
                    help="lanes,slots of the tensor-core page kernel instead of the autotuner's pick "
                         "(4,1 / 2,2 / 8,1; for profiling one kernel)")
    args = ap.parse_args()
    args.page_shape = tuple(int(x) for x in args.page_shape.split(",")) if args.page_shape else None
    args.warmup = max(args.warmup, 3)
    nq = 1 << args.queries_log2
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    args.world = world
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_2604_12625_gb300 import build as _b
    _b.build()
    import paper_2604_12625_gb300 as ndgi

    peaks, peak_kind = load_peaks()
    m = synth.points_model_2048(2)
    q = synth.random_queries(rank_query_seed(rank), nq)
    model = ndgi.Model.from_arrays(m)
    uvt = torch.from_numpy(q).cuda()
    out = torch.empty((nq, 3), dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    tc = ndgi.ndgi_prepare_workspace_size(model, "fp16") > 0
    prec = args.precision if args.precision != "auto" else ("fp16" if tc else "fp32")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def timed(fn, steps, warmup, sample_clocks=False):
        for _ in range(warmup):
            fn()
        barrier()
        sampler = ClockSampler(local) if sample_clocks else None
        if sampler:
            sampler.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        barrier()
        clocks = sampler.stop() if sampler else None
        ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
        return ms, clocks

    def per_step_median(fn, k, flush=None):
        """Median of k individually timed steps (events around each); flush() runs before each, untimed."""
        times = []
        for _ in range(k):
            if flush is not None:
                flush()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        return float(np.median(times))

    args.per_step_median = per_step_median
    ws = model.workspace(prec)

    def step_main():
        ndgi.ndgi_decode_points(model, uvt, prec, ws=ws, out=out)

    def step_fp32():
        ndgi.ndgi_decode_points(model, uvt, "fp32", out=out)

    ms_main, clocks = timed(step_main, args.steps, args.warmup, sample_clocks=True)
    ms_median = per_step_median(step_main, 20)
    ms_step = ms_main / args.steps
    device_check = {"points": check_status(ndgi, model, prec)}
    value = job_value(nq, world, ms_step)

    # FP32 plain decode beside it (fewer steps: it is ~10x slower)
    k32 = max(3, min(args.steps, 20))
    ms32, _ = timed(step_fp32, k32, 3)
    fp32_gt = job_value(nq, world, ms32 / k32)

    # Accuracy on a seeded sample, against the FP64 oracle (rank 0)
    errs = {}
    if rank == 0:
        import oracle
        idx = np.random.default_rng(0).choice(nq, 1 << 14, replace=False)
        idx_t = torch.from_numpy(idx).cuda()
        for p in sorted({prec, "fp32"}):
            ndgi.ndgi_decode_points(model, uvt, p, ws=model.workspace(p), out=out)
            got = out[idx_t].cpu().numpy().astype(np.float64)
            ref = oracle.decode_points(m, q[idx], precision=p if p in ("fp16", "bf16") else "fp32")
            errs[p] = float(np.abs(got - ref).max() / (ref.max() - ref.min()))

    # End to end through the public API with host buffers: the host-buffer
    # decode (ndgi_decode_points_host) copies the step's pinned queries in,
    # decodes and copies the results out, chunk by chunk with the three stages
    # overlapped, all inside the timed region.
    q_host = torch.from_numpy(q).pin_memory()
    out_host = torch.empty((nq, 3), dtype=torch.float32).pin_memory()
    pipe = ndgi.HostPipe(chunk=args.e2e_chunk)

    def step_e2e():
        pipe.decode_points(model, q_host, prec, ws=ws, out=out_host)

    ke = max(3, min(args.steps, 20))
    ms_e2e, _ = timed(step_e2e, ke, 3)
    e2e_val = job_value(nq, world, ms_e2e / ke)
    step_main()   # the device decode of the same queries: the pipe's result must equal it
    torch.cuda.synchronize()
    e2e_ok = bool(torch.equal(out_host, out.cpu()))
    pipe.close()

    pages = None
    if not args.no_pages:
        pages = bench_pages(args, ndgi, torch, peaks, peak_kind, timed, rank)
    fit = scale = hybrid = quality = fit_batch = hybrid_fit = hybrid_fit_batch = None
    if not args.no_extra:
        if not args.no_scale:
            scale = bench_scale(args, ndgi, torch, peaks, peak_kind, timed, rank)
        fit = bench_fit(args, ndgi, torch)
        if not args.no_hybrid:
            hybrid = bench_hybrid(args, ndgi, torch, peaks, peak_kind, timed, rank)
        quality = bench_quality(args, ndgi, torch)
        if not args.no_hybrid:
            hybrid["profiles_1024"] = bench_hybrid_profiles(args, ndgi, torch, timed)
        fit_batch = bench_fit_batch(args, ndgi, torch)
        if not args.no_hybrid:
            hybrid_fit = bench_hybrid_fit(args, ndgi, torch)
            hybrid_fit_batch = bench_hybrid_fit_batch(args, ndgi, torch)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    sm_mhz = (clocks or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    kernel_s = ms_step * 1e-3
    if prec == "fp32":
        peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0), torch.cuda.get_device_properties(local).multi_processor_count)
        roof = {"bound": "alu", "achieved": nq * FLOP_PER_TEXEL / kernel_s / 1e12, "peak": peak,
                "unit": "TFLOP/s", "peak_source": "derived: SMs x 128 FP32 lanes x 2 FLOP x max SM clock"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        # bytes: 24 B of query I/O per query plus the compressed feature map once
        roof = two_term_roofline(nq, FLOP_PER_TEXEL, nq * 24 + m["bc4"].nbytes, kernel_s, peaks, peak_kind)
    path = ndgi.ndgi_decode_points_path(model, prec, nq) if prec != "fp32" else "direct"
    roof["kernel"] = ("k_points_f32" if prec == "fp32" else
                      {"direct": "k_points_tc", "cache": "k_points_tc", "cache_ws": "k_points_ws"}[path])
    roof["gather"] = path
    roof["traffic"] = traffic_for(roof["kernel"], nq)
    if roof["traffic"] is not None:
        roof["traffic_note"] = (f"ncu DRAM bytes of a 2^23-query launch scaled x{nq / (1 << 23):g}; output lines "
                                "still dirty in L2 at kernel end are not counted; algorithmic "
                                f"{(nq * 24 + (8 << 20)) / 1e6:.0f} MB")

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        gt, n_s, dt, nt = time_oracle(m, q, 12.0)
        one = time_oracle_one_core(m, q)
        cpu = {"value": gt, "unit": "Gtexels/s", "cores": nt, "kind": "oracle",
               "sample": f"first {n_s} of the 2^{args.queries_log2} queries, FP64 oracle ({dt:.1f} s)",
               "per_core_gtexels_s": one / 1e9, "cpu_model": cpu_model()}

    line = {
        "metric": METRIC, "value": value, "unit": "Gtexels/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp16": "f16", "bf16": "bf16", "fp32": "f32"}[prec], "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("2^24", f"2^{args.queries_log2}"), "queries_per_rank": nq, "precision": prec,
                   "l2": f"inputs larger than L2: {nq * 12 / 1e6:.0f} MB of queries + {nq * 12 / 1e6:.0f} MB of "
                         "output per step; the 8 MiB feature map stays L2-resident as in a steady frame"},
        "device_check": device_check, "max_err_over_range": errs, "fp32_plain": {"value": fp32_gt, "unit": "Gtexels/s",
                                                  "err": errs.get("fp32")},
        "roofline": roof, "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "Gtexels/s", "h2d_bytes_per_step": nq * 12,
                "d2h_bytes_per_step": nq * 12, "api": "ndgi_decode_points_host (pinned host buffers)",
                "pipeline": f"chunks of {args.e2e_chunk} queries; copy-in, decode and copy-out overlapped on three "
                            "streams", "matches_device_decode": e2e_ok},
        "ms_per_step_median_of_20": ms_median,
        "gpu_launches": args.steps * (2 if path in ("cache", "cache_ws") else 1),
        "gpu_launches_per_step": ("k_feature_cache + " + roof["kernel"]) if path in ("cache", "cache_ws")
                                 else roof["kernel"],
        "clocks": clocks,
        "fit": fit, "fit_batch": fit_batch, "hybrid_fit": hybrid_fit, "hybrid_fit_batch": hybrid_fit_batch, "scale": scale, "hybrid": hybrid, "quality": quality, "pages": pages,
    }
    if hybrid is not None:
        h16, hr = hybrid["fp16"], hybrid["roofline"]
        line["hybrid_m64_fp16"] = {
            "value": h16["value"], "unit": "Gtexels/s", "ms_per_frame": h16["ms_per_frame"], "frac": hr["frac"],
            "bound": hr["bound"], "max_err_over_page_range": h16.get("max_err_over_page_range"),
            "vs_fp32_plain": hybrid["vs_fp32_plain"], "device_check": h16["device_check"],
            "bc7_value": hybrid["fp16_bc7"]["value"], "bc7_rgba8_value": hybrid["fp16_bc7_rgba8"]["value"]}
    if pages is not None:
        # the batched page decode (the configuration the >= 60 % roofline target is stated on), in brief, last
        p16, rf = pages["fp16"], pages["roofline"]
        line["pages_c4_fp16"] = {
            "value": p16["value"], "unit": "Gtexels/s", "ms_per_frame": p16["ms_per_frame"],
            "frac": rf["frac"], "bound": rf["bound"], "kernel": rf["kernel"], "plan_shape": p16["plan_shape"],
            "max_err_over_page_range": p16.get("max_err_over_page_range"),
            "vs_fp32_plain": p16["value"] / pages["fp32"]["value"], "device_check": p16["device_check"]}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
