#!/usr/bin/env python3
"""Benchmark of the MSDA hot path on GB300.

One step = one training pass of the operator over one frame of the
outside-in 64-camera workload: msda_forward (BF16 features and weights, FP32
accumulation and output) followed by msda_backward (deterministic mode, or
the atomic one with --atomic: FP32 gradients for the features, locations and
weights).  Shapes: B=1, 64 cameras,
maps 68x120, 34x60, 17x30, 9x15 (1080p at strides 8..64), C=256, G=8,
A=900 anchors, P=13 keypoints, 40% of (anchor, camera) pairs out of view.
Inputs are synthetic and seeded (paper_2601_10819_gb300.inputs, workload 2).

Printed: one JSON line with the metric (us/frame, lower is better), the
Gsamples/s throughput, a roofline entry for the dominant kernel, the
end-to-end number through the public API with host buffers, the FP64 CPU
oracle timed on a bounded sample, the SM clocks seen during the timed
region, and (N = 1) the other forms of the path timed in the same run.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank processes its own frame (weak scaling,
no collective on the data path); the step time is the max over ranks.  With
--split cameras the ranks share one frame by camera instead (strong
scaling, one NCCL sum all-reduce of the partial output per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

METRIC = "MSDA fwd+bwd µs/frame @64 cams bf16; Gsamples/s; % gather roofline"
UNIT = "µs/frame"
WORKLOAD = ("outside-in-64cam fwd+bwd: B1 Ncam64 maps 68x120/34x60/17x30/9x15 C256 G8 A900 P13, "
            "40% of (anchor,camera) pairs out of view, BF16 feat+weights, FP32 accumulate/out/grads")
# Other workloads the step can run on (diagnostics and profiles; the benchmark line is the default one):
# name -> (workload index, feature dtype, weight dtype, description)
WORKLOADS = {
    "outside-in-64cam": (2, None, None, WORKLOAD),
    "train-16cam": (3, None, None, "train-16cam fwd+bwd: B4 Ncam16 maps 64x176/32x88/16x44/8x22 C256 G8 A900 P13, "
                                   "BF16 feat, FP32 weights/accumulate/out/grads"),
    "sparse4d-6cam-bf16": (1, "bf16", "bf16", "sparse4d-6cam fwd+bwd: B1 Ncam6 maps 64x176/32x88/16x44/8x22 C256 G8 "
                                              "A900 P13, BF16 feat+weights, FP32 accumulate"),
}
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "dram_traffic.json")
FALLBACK_HBM_GBS = 6800.0


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--copy-streams", type=int, default=1, help="streams per copy direction in the end-to-end run")
    ap.add_argument("--cpu-sample-anchors", type=int, default=300)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--atomic", action="store_true",
                    help="time the atomic backward (FP32 vector reductions) instead of the deterministic one")
    ap.add_argument("--deterministic", action="store_true",
                    help="the deterministic backward (the default; kept for older command lines)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other timed forms (6-camera forwards, standalone forward, the other backward "
                         "mode, batched serving)")
    ap.add_argument("--clear", default="forward", choices=["forward", "side", "inline"],
                    help="atomic backward: clear the feature gradient inside the forward kernel "
                         "(msda_forward_train), on a side stream during the forward (side), or with a memset "
                         "inside msda_backward (inline)")
    ap.add_argument("--no-tune", action="store_true", help="use the built-in launch mappings")
    ap.add_argument("--extras", action="store_true",
                    help="also time the fused occlusion-aware forward, the keypoint prologue and the half2 forward")
    ap.add_argument("--workload", default="outside-in-64cam", choices=sorted(WORKLOADS),
                    help="workload of the timed step (the benchmark line is quoted on outside-in-64cam)")
    ap.add_argument("--configs", action="store_true",
                    help="also time the 6-camera (FP32, BF16) and 16-camera training workloads")
    ap.add_argument("--with-batched", action="store_true",
                    help="also time the 16-scene batched serving workload (per-scene p50/p99)")
    ap.add_argument("--split", default="replicas", choices=["replicas", "cameras"],
                    help="N > 1: every rank runs its own frame (replicas, weak scaling) or the ranks split one "
                         "frame's cameras and sum the partial outputs with one NCCL all-reduce (cameras, strong "
                         "scaling)")
    return ap.parse_args(argv)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(values, device):
    """Element-wise max of per-rank timings (the job is as slow as its slowest rank)."""
    t = torch.tensor(list(values), dtype=torch.float64, device=device)
    if torch.distributed.is_available() and torch.distributed.is_initialized() and \
            torch.distributed.get_world_size() > 1:
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return t.tolist()


def split_shard(tensors, rank, world):
    """Camera split: this rank's cameras and its shard of the frame (maps re-packed, location and weight
    slices of its cameras)."""
    from paper_2601_10819_gb300 import shard
    cams = shard.split_cameras(tensors[1].shape[0], world)[rank]
    return cams, shard.shard_problem(*tensors, cams)


def split_step(sub, grad_out, forward, backward, group=None):
    """One step of the camera split on this rank: the shard's partial output, completed by one sum all-reduce
    over the ranks (the frame's output on every rank), then the shard's gradients for the full grad_out."""
    from paper_2601_10819_gb300 import shard
    out = forward(*sub)
    shard.reduce_partials(out, group)
    return out, backward(*sub, grad_out)


def backward_launches(det, zeroed=False):
    """Kernels msda_backward enqueues on the benchmark frame: atomic: the scatter kernel (and a memset unless
    the forward cleared grad_feat); deterministic: the cell-binned plan, location transpose, binning and reduce,
    dloc/dw, and the one-thread launcher that issues the corner-slot form from the device only when the
    cell-binned plan has cleared its flag (it does not on this frame)."""
    return 6 if det else (1 if zeroed else 2)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def load_traffic(kernel_key):
    """DRAM bytes per launch from a committed ncu capture, if it matches the current source."""
    try:
        with open(TRAFFIC_FILE) as f:
            d = json.load(f)
        e = d[kernel_key]
        if e["source_sha"] != source_sha(e["sources"]):
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.lines = []
        self.proc = None
        try:
            bus = torch.cuda.get_device_properties(device_index).pci_bus_id
            sel = ["-i", f"{int(torch.cuda.get_device_properties(device_index).pci_domain_id):08X}:"
                         f"{int(bus):02X}:{int(torch.cuda.get_device_properties(device_index).pci_device_id):02X}.0"]
        except Exception:
            sel = []
        self.cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100"] + sel

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for _, _, r in rows:
            for n, flag in zip(names, r[1:]):
                if flag.lower() in ("active", "1", "yes"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def l2_rates(dev, stream, tries=5):
    """L2 rates measured live (best of `tries` runs of ~0.3 ms each, 64 MB L2-resident buffers): random
    512-byte row gathers (the operator's corner loads) and random 1 KB FP32 vector reductions (the atomic
    backward's scatter), in GB/s."""
    from paper_2601_10819_gb300 import msda
    nsm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, reps, rows = nsm * 4, 16, 64
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def best(fn, nbytes):
        fn()
        rate = 0.0
        for _ in range(tries):
            e0.record(stream)
            fn()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            rate = max(rate, nbytes / (e0.elapsed_time(e1) * 1e-3) / 1e9)
        return rate

    buf = torch.empty(64 << 20, dtype=torch.uint8, device=dev).random_()
    gather = best(lambda: msda.probe_read(buf, reps, blocks, rows), blocks * 16 * reps * rows * 512)
    del buf
    red_buf = torch.zeros(16 << 20, dtype=torch.float32, device=dev)
    red = best(lambda: msda.probe_reduce(red_buf, reps // 4, blocks, rows), blocks * 16 * (reps // 4) * rows * 1024)
    del red_buf
    return gather, red


def _oracle_calls(sub, nthreads):
    """Seconds of one oracle call each on `sub`: forward on `nthreads` threads, backward, forward on one thread."""
    import oracle
    args = [oracle._f64(t) if i in (0, 3, 4) else oracle._i32(t) for i, t in enumerate(sub.tensors())]
    go = oracle._f64(sub.grad_out)
    t0 = time.perf_counter()
    oracle.forward(*args, nthreads=nthreads)
    t1 = time.perf_counter()
    oracle.backward(*args, go)
    t2 = time.perf_counter()
    oracle.forward(*args, nthreads=1)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2


def oracle_times(pr, sample_anchors):
    """Seconds per frame of the FP64 oracle, extrapolated from a sample of the first `sample_anchors` anchors:
    forward on all host threads and on one, backward on one.  A call costs a fixed part (the backward allocates and
    clears the FP64 feature gradient, whatever the anchor count) plus a part per anchor, so each call is also timed
    on one anchor and a frame's time is fixed + (sample - fixed) * (A - 1) / (sample anchors - 1)."""
    import oracle
    oracle.build()
    nthreads = oracle.max_threads()
    A, B = pr.sampling_location.shape[1], pr.feat.shape[0]
    na = max(2, min(sample_anchors, A))
    one = _oracle_calls(pr.anchors(range(1)), nthreads)
    big = _oracle_calls(pr.anchors(range(na)), nthreads)
    frame = [(t1 + (tn - t1) * (A - 1) / (na - 1)) / B for t1, tn in zip(one, big)]
    return {"fwd_all": frame[0], "bwd_1": frame[1], "fwd_1": frame[2], "raw": big[:2], "fixed": one[:2],
            "threads": nthreads, "anchors": na}


def cpu_baseline(pr, sample_anchors, others=False):
    """The FP64 oracle (as it stands) on the first `sample_anchors` anchors of the frame; with `others`, also on
    samples of the 6-camera and 16-camera workloads."""
    t = oracle_times(pr, sample_anchors)
    A = pr.sampling_location.shape[1]
    per_frame_s = t["fwd_all"] + t["bwd_1"]
    res = {"value": per_frame_s * 1e6, "unit": UNIT, "cores": t["threads"], "kind": "oracle",
           "sample": f"{t['anchors']} of {A} anchors of one frame (fwd on {t['threads']} OpenMP threads, bwd "
                     f"single-threaded): fwd {t['raw'][0]:.2f} s + bwd {t['raw'][1]:.2f} s, of which fwd "
                     f"{t['fixed'][0]:.2f} s + bwd {t['fixed'][1]:.2f} s is the per-call cost (timed on one anchor); "
                     f"the per-anchor part scaled to {A} anchors",
           "fwd_us_per_frame_all_cores": t["fwd_all"] * 1e6,
           "fwd_us_per_frame_1_core": t["fwd_1"] * 1e6,
           "bwd_us_per_frame_1_core": t["bwd_1"] * 1e6,
           "host": host_info()}
    if others:
        from paper_2601_10819_gb300 import inputs
        res["other_workloads"] = {}
        for name, idx, kw, n in (("sparse4d-6cam-fp32", 1, {"feat_dtype": "f32", "w_dtype": "f32"}, 300),
                                 ("train-16cam-b4", 3, {}, 100)):
            o = oracle_times(inputs.make_workload(idx, **kw), n)
            res["other_workloads"][name] = {"fwd_us_per_frame_all_cores": o["fwd_all"] * 1e6,
                                            "fwd_us_per_frame_1_core": o["fwd_1"] * 1e6,
                                            "bwd_us_per_frame_1_core": o["bwd_1"] * 1e6,
                                            "sample_anchors": o["anchors"]}
    return res


def host_info():
    """CPU model, logical CPUs and the CPUs this process may run on."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    try:
        affinity = len(os.sched_getaffinity(0))
    except AttributeError:
        affinity = os.cpu_count()
    return {"cpu": model, "machine": platform.machine(), "nproc": os.cpu_count(), "affinity": affinity}


def batched_serving(dev, stream, tune_it=True, reps=20):
    """16 uneven scenes in one persistent launch replayed from a CUDA graph: per-scene latency."""
    from paper_2601_10819_gb300 import inputs, msda, tune
    scenes = [s.to(dev) for s in inputs.make_workload(4, with_grad=False)]
    cfg = tune.tune_batched(scenes) if tune_it else dict(vec=0, warps=0, bps=0)
    plan = msda.plan_batched(scenes, warps=cfg["warps"] or None, blocks_per_sm=cfg["bps"] or None, vec=cfg["vec"])
    plan.run()
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream(dev)
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.run()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize(dev)
    lat, total = [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for _ in range(reps):
        e0.record(stream)
        g.replay()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        t = plan.done_ns.cpu().double()
        lat.extend(((t[1:] - t[0]) / 1e3).tolist())
        total.append(e0.elapsed_time(e1) * 1e3)
    lat.sort()
    nominal = sum(int(np.prod(sc.weights.shape[:5])) for sc in scenes)
    return {"scenes": len(scenes), "cameras": sum(sc.spatial_shape.shape[0] for sc in scenes),
            "anchors": plan.total, "tuning": cfg,
            "us_per_batch_median": statistics.median(total),
            "scene_latency_us_p50": lat[len(lat) // 2], "scene_latency_us_p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
            "gsamples_per_s": nominal / (statistics.median(total) * 1e-6) / 1e9}


def extras(pr, dev, ft, reps=20):
    """Timings (us) of the other forms of the path on the benchmark frame."""
    from paper_2601_10819_gb300 import inputs, msda
    d = pr.to(dev)
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    out = torch.empty(d.grad_out.shape, device=dev)
    vis = inputs.make_visibility(pr, 2).to(dev)
    geo = [t.to(dev) for t in inputs.make_scene_geometry(2, B=1, A=pr.weights.shape[1], P=pr.weights.shape[2],
                                                         ncam=pr.weights.shape[3])]
    loc = torch.empty_like(d.sampling_location)
    f16 = (d.feat.half(), d.weights.half())

    def tm(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            fn()
        e1.record()
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps * 1e3

    kw = dict(warps=ft["warps"] or None, vec=ft["vec"])
    return {
        "forward_us": tm(lambda: msda.forward(*T, out=out, workspace=None, **kw)),
        "forward_fused_occlusion_aware_us": tm(lambda: msda.forward_oae(*T, vis, out=out, **kw)),
        "keypoint_prologue_us": tm(lambda: msda.keypoints(*geo, out=loc)),
        "forward_fp16_fp32acc_us": tm(lambda: msda.forward(f16[0], d.spatial_shape, d.scale_start_index,
                                                           d.sampling_location, f16[1], out=out, workspace=None, **kw)),
        "forward_fp16_half2acc_us": tm(lambda: msda.forward(f16[0], d.spatial_shape, d.scale_start_index,
                                                            d.sampling_location, f16[1], out=out, workspace=None,
                                                            variant=3, **kw)),
    }


def other_forms(dev, stream, pr, cnt, det_step, l2_gbs, l2_red_gbs, hbm_peak, tune_it=True, reps=20):
    """The other forms of the path timed in the same run as the step, each with its gather-roof fraction:
    the 6-camera Sparse4D forward in FP32 and BF16, the benchmark frame's standalone forward (no gradient
    clearing), the backward mode the step does not use, and the 16-scene batched serving launch."""
    from paper_2601_10819_gb300 import inputs, msda, roofline, tune

    def tm(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps * 1e3

    def fwd_roof(c):
        return max(c.fwd_hbm_bytes / (hbm_peak * 1e9), c.fwd_l2_gather_bytes / (l2_gbs * 1e9)) * 1e6

    res = {}
    for name, fdt in (("sparse4d-6cam fwd fp32", "f32"), ("sparse4d-6cam fwd bf16", "bf16")):
        p1 = inputs.make_workload(1, feat_dtype=fdt, w_dtype=fdt, with_grad=False)
        c1 = roofline.count(p1)
        d = p1.to(dev)
        T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
        out = torch.empty(d.weights.shape[0], d.weights.shape[1], d.feat.shape[2], device=dev)
        ft = tune.tune_forward(T, out) if tune_it else dict(vec=0, warps=0, workspace=False)
        us = tm(lambda: msda.forward(*T, out=out, warps=ft["warps"] or None, vec=ft["vec"]))
        res[name] = {"us_per_frame": us, "gsamples_per_s": c1.nominal_samples / (us * 1e-6) / 1e9,
                     "gather_roof_us": fwd_roof(c1), "gather_roof_frac": fwd_roof(c1) / us, "tuning": ft}
        del d, out
    d = pr.to(dev)
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    B, sum_hw, C = d.feat.shape
    out = torch.empty(d.grad_out.shape, device=dev)
    ft = tune.tune_forward(T, out) if tune_it else dict(vec=0, warps=0, workspace=False)
    us = tm(lambda: msda.forward(*T, out=out, warps=ft["warps"] or None, vec=ft["vec"]))
    res["outside-in-64cam fwd standalone"] = {
        "us_per_frame": us / B, "gsamples_per_s": cnt.nominal_samples / (us * 1e-6) / 1e9,
        "gather_roof_us": fwd_roof(cnt), "gather_roof_frac": fwd_roof(cnt) / us}
    det = not det_step
    grads = (torch.empty(B, sum_hw, C, device=dev), torch.empty(d.sampling_location.shape, device=dev),
             torch.empty(d.weights.shape, device=dev))
    K, S = d.weights.shape[3], d.weights.shape[4]
    A, P, G = d.weights.shape[1], d.weights.shape[2], d.weights.shape[5]
    ws = torch.empty(max(16, msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, det)), dtype=torch.uint8,
                     device=dev)
    us = tm(lambda: msda.backward(*T, d.grad_out, deterministic=det, workspace=ws, grads=grads))
    red = cnt.bwd_l2_bytes - cnt.fwd_l2_gather_bytes
    t_hbm = cnt.bwd_hbm_bytes / (hbm_peak * 1e9) * 1e6
    if det:  # gathers: corner rows and, per in-bound corner, its anchor's grad_out row (no L2 reductions)
        roof = max(t_hbm, (cnt.fwd_l2_gather_bytes + red) / (l2_gbs * 1e9) * 1e6)
    else:
        roof = max(t_hbm, cnt.fwd_l2_gather_bytes / (l2_gbs * 1e9) * 1e6, red / (l2_red_gbs * 1e9) * 1e6)
    res["outside-in-64cam bwd " + ("deterministic" if det else "atomic (with its clearing of grad_feat)")] = {
        "us_per_frame": us / B, "roof_us": roof, "roof_frac": roof / us}
    del d, out, grads, ws
    res["batched-serving fwd"] = batched_serving(dev, stream, tune_it=tune_it, reps=reps)
    return res


def other_configs(dev, l2_gbs, l2_red_gbs, hbm_peak, reps=20):
    """Forward and atomic backward timings of the non-headline workloads, each with its roofline: the
    forward against max(HBM, L2 gathers), the backward against max(HBM, L2 gathers, L2 FP32 reductions).

    A frame is one batch element; a backward timing includes clearing the feature gradient.
    """
    from paper_2601_10819_gb300 import inputs, msda, roofline
    res = {}
    for name, idx, fdt, wdt in (("sparse4d-6cam-fp32", 1, "f32", "f32"), ("sparse4d-6cam-bf16", 1, "bf16", "bf16"),
                                ("train-16cam-b4", 3, None, None)):
        pr = inputs.make_workload(idx, feat_dtype=fdt, w_dtype=wdt)
        cnt = roofline.count(pr)
        d = pr.to(dev)
        T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
        B, sum_hw, C = d.feat.shape
        out = torch.empty(d.grad_out.shape, device=dev)
        grads = (torch.empty(B, sum_hw, C, device=dev), torch.empty(d.sampling_location.shape, device=dev),
                 torch.empty(d.weights.shape, device=dev))
        ws = torch.empty(msda.backward_workspace_size(B, sum_hw, C, *d.weights.shape[3:5], d.weights.shape[1],
                                                      d.weights.shape[2], d.weights.shape[5], False),
                         dtype=torch.uint8, device=dev)

        def tm(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                fn()
            e1.record()
            torch.cuda.synchronize(dev)
            return e0.elapsed_time(e1) / reps * 1e3

        f_us = tm(lambda: msda.forward(*T, out=out))
        f_staged_us = tm(lambda: msda.forward(*T, out=out, workspace="auto"))
        b_us = tm(lambda: msda.backward(*T, d.grad_out, workspace=ws, grads=grads))
        roof_f = max(cnt.fwd_hbm_bytes / (hbm_peak * 1e9), cnt.fwd_l2_gather_bytes / (l2_gbs * 1e9)) * 1e6
        roof_b = max(cnt.bwd_hbm_bytes / (hbm_peak * 1e9), cnt.fwd_l2_gather_bytes / (l2_gbs * 1e9),
                     (cnt.bwd_l2_bytes - cnt.fwd_l2_gather_bytes) / (l2_red_gbs * 1e9)) * 1e6
        res[name] = {"frames": B, "fwd_us_per_frame": f_us / B, "fwd_staged_us_per_frame": f_staged_us / B,
                     "bwd_us_per_frame": b_us / B,
                     "fwd_gsamples_per_s": cnt.nominal_samples / (f_us * 1e-6) / 1e9,
                     "fwd_gather_roof_frac": roof_f / f_us, "bwd_gather_roof_frac": roof_b / b_us}
        del d, out, grads
    return res


def run_camera_split(args, rank, world, local):
    """--split cameras: the ranks share one frame by camera (Sec. 3.2: the operator is a sum over cameras).
    Rank r holds only its cameras' maps and their location and weight slices; a step is the shard's forward,
    one NCCL sum all-reduce of the FP32 partial output [B, A, C], and the shard's backward for the full
    grad_out.  The job processes B frames per step whatever N is (strong scaling)."""
    from paper_2601_10819_gb300 import build as msda_build
    from paper_2601_10819_gb300 import inputs, msda, shard, tune

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        msda_build.build()
    if world > 1:
        torch.distributed.barrier()
    msda.load()
    wl_idx, wl_f, wl_w, wl_desc = WORKLOADS[args.workload]
    pr = inputs.make_workload(wl_idx, **({"feat_dtype": wl_f, "w_dtype": wl_w} if wl_f else {}))
    cams, sub = split_shard(pr.tensors(), rank, world)
    sub = tuple(t.to(dev) for t in sub)
    go = pr.grad_out.to(dev)
    B, A, C = go.shape
    det = not args.atomic
    sum_hw, K, S, P, G = sub[0].shape[1], sub[3].shape[3], sub[4].shape[4], sub[4].shape[2], sub[4].shape[5]
    out_buf = torch.empty(B, A, C, device=dev)
    grads = (torch.empty(B, sum_hw, C, device=dev), torch.empty(sub[3].shape, device=dev),
             torch.empty(sub[4].shape, device=dev))
    ws = torch.empty(max(16, msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, det)), dtype=torch.uint8,
                     device=dev)
    if args.no_tune:
        ft, bt = dict(vec=0, warps=0), dict(vec=0, warps=0)
    else:  # the shard's own launch mappings (untimed)
        ft = tune.tune_forward(sub, out_buf)
        bt = tune.tune_backward(sub, go, grads, deterministic=det, workspace=ws)

    def fwd(*t):
        return msda.forward(*t, out=out_buf, warps=ft["warps"] or None, vec=ft["vec"])

    def bwd(*t):
        return msda.backward(*t, deterministic=det, workspace=ws, grads=grads, warps=bt["warps"] or None,
                             vec=bt["vec"])

    for _ in range(args.warmup):
        split_step(sub, go, fwd, bwd)
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            e = evs[i]
            e[0].record(stream)
            out = fwd(*sub)
            e[1].record(stream)
            shard.reduce_partials(out)
            e[2].record(stream)
            bwd(*sub, go)
            e[3].record(stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(end)
    fwd_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    ar_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    bwd_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / args.steps
    total_ms, fwd_ms, ar_ms, bwd_ms = max_over_ranks([total_ms, fwd_ms, ar_ms, bwd_ms], dev)
    if msda.device_status() != 0:
        raise RuntimeError("device status set during the timed region")
    per_rank = [len(c) for c in shard.split_cameras(pr.spatial_shape.shape[0], world)]
    ms_per_step = total_ms / args.steps
    line = {
        "metric": METRIC, "value": ms_per_step * 1e3 / B, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "strong",
        "vs_baseline": None, "dtype": "bf16", "accumulate": "f32", "data": "synthetic",
        "config": {"workload": wl_desc, "frames_per_step": B,
                   "parallelism": f"camera split x{world}: rank r owns cameras split_cameras(Ncam, {world})[r] "
                                  f"with their maps; one NCCL sum all-reduce of out [B, A, C] FP32 per step",
                   "cameras_per_rank": per_rank, "backward": "deterministic" if det else "atomic",
                   "l2": "inputs larger than L2 on one GPU; no flush"},
        "fwd_us": fwd_ms * 1e3, "allreduce_us": ar_ms * 1e3, "bwd_us": bwd_ms * 1e3,
        "allreduce_bytes_per_step": B * A * C * 4 if world > 1 else 0,
        "e2e": None,  # the end-to-end number is measured by the default (replica) mode
        "gpu_launches": (1 + backward_launches(det)) * args.steps,
        "clocks": clk.summary(),
        "gpu": torch.cuda.get_device_name(dev),
    }
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle, timed on the host cores."""
    if rank != 0:
        return 0
    from paper_2601_10819_gb300 import inputs
    import oracle
    oracle.build()
    wl_idx, wl_f, wl_w, wl_desc = WORKLOADS[args.workload]
    pr = inputs.make_workload(wl_idx, **({"feat_dtype": wl_f, "w_dtype": wl_w} if wl_f else {}))
    A = pr.sampling_location.shape[1]
    nthreads = oracle.max_threads()
    feat = oracle._f64(pr.feat)
    shape, start = oracle._i32(pr.spatial_shape), oracle._i32(pr.scale_start_index)
    def step(idx):
        sub = pr.anchors(idx)
        loc, w, go = oracle._f64(sub.sampling_location), oracle._f64(sub.weights), oracle._f64(sub.grad_out)
        t0 = time.perf_counter()
        oracle.forward(feat, shape, start, loc, w, nthreads=nthreads)
        oracle.backward(feat, shape, start, loc, w, go)
        return time.perf_counter() - t0

    # a call costs a fixed part (the backward allocates and clears the FP64 feature gradient) plus a part per
    # anchor: the fixed part is timed on one anchor, and each step's anchor sample is sized so that the whole run
    # stays within about three minutes (at least 8 anchors a step)
    fixed = min(step([0]), step([1 % A]))
    budget_s = 180.0
    per_anchor_s = 0.02
    na = int(max(8, min(A, (budget_s / max(1, args.steps + args.warmup) - fixed) / per_anchor_s)))
    na = min(na, A)
    times, raw = [], []
    for it in range(args.warmup + args.steps):
        a0 = (it * na) % A
        dt = step([(a0 + j) % A for j in range(na)])
        if it >= args.warmup:
            times.append(dt if na == A else fixed + (dt - fixed) * (A - 1) / (na - 1))
            raw.append(dt)
    v = statistics.mean(times) * 1e6
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": v / 1e3, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl_desc, "parallelism": "host cores"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": nthreads, "kind": "oracle",
                             "sample": f"{na} anchors of {A} per step (forward on {nthreads} threads, backward "
                                       f"single-threaded); a frame = the per-call cost ({fixed:.2f} s, timed on one "
                                       f"anchor) + the sample's per-anchor part scaled to {A} anchors"},
            # value and ms_per_step are a frame's time extrapolated from the anchor sample, not the wall time of
            # a step; measured_ms_per_step is the sample's own time
            "extrapolated": na < A, "frame_scale": A / na, "per_call_s": fixed,
            "measured_ms_per_step": statistics.mean(raw) * 1e3,
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.split == "cameras":
        return run_camera_split(args, rank, world, local)

    from paper_2601_10819_gb300 import build as msda_build
    from paper_2601_10819_gb300 import inputs, msda, roofline, tune

    if not torch.cuda.is_available():
        raise RuntimeError("bench.py needs a CUDA GPU")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        msda_build.build()
    if world > 1:
        torch.distributed.barrier()
    msda.load()

    wl_idx, wl_f, wl_w, wl_desc = WORKLOADS[args.workload]
    pr = inputs.make_workload(wl_idx, **({"feat_dtype": wl_f, "w_dtype": wl_w} if wl_f else {}))
    cnt = roofline.count(pr)
    d = pr.to(dev)
    B, sum_hw, C = d.feat.shape
    _, A, P, K, _ = d.sampling_location.shape
    S, G = d.weights.shape[4], d.weights.shape[5]
    out = torch.empty(B, A, C, device=dev)
    gf = torch.empty(B, sum_hw, C, device=dev)
    gl = torch.empty(B, A, P, K, 2, device=dev)
    gw = torch.empty(B, A, P, K, S, G, device=dev)
    det = not args.atomic
    ws = None
    need = msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, det)
    if need:
        ws = torch.empty(need, dtype=torch.uint8, device=dev)
    tensors = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    fws = torch.empty(msda.forward_workspace_size(B, sum_hw, C, K, S, A, P, G), dtype=torch.uint8, device=dev)
    if args.no_tune:
        ft, bt = dict(vec=0, warps=0, workspace=False), dict(vec=0, warps=0)
    else:  # autotuned launch mappings (cached per GPU model and shape); untimed
        ft = tune.tune_forward(tensors, out, workspace=fws)
        bt = tune.tune_backward(tensors, d.grad_out, (gf, gl, gw), deterministic=det, workspace=ws)
    fwd_ws = fws if ft["workspace"] else None
    side_clear = not det and args.clear == "side"
    fwd_clear = not det and args.clear == "forward"
    side = torch.cuda.Stream(dev)  # clears the feature gradient while the forward runs (--clear side)
    main = torch.cuda.current_stream(dev)

    def fwd(tens=None, outs=None):
        o, g = (out, gf) if outs is None else (outs[0], outs[1])
        if side_clear:
            side.wait_stream(main)  # the previous backward is done with grad_feat
            with torch.cuda.stream(side):
                g.zero_()
        if fwd_clear:
            msda.forward_train(*(tens or tensors), g, out=o, warps=ft["warps"] or None, vec=ft["vec"])
        else:
            msda.forward(*(tens or tensors), out=o, workspace=fwd_ws, warps=ft["warps"] or None, vec=ft["vec"])

    def bwd(tens=None, go=None, outs=None):
        if side_clear:
            main.wait_stream(side)
        msda.backward(*(tens or tensors), d.grad_out if go is None else go, deterministic=det, workspace=ws,
                      grads=(gf, gl, gw) if outs is None else tuple(outs[1:]), warps=bt["warps"] or None,
                      vec=bt["vec"], grad_feat_zeroed=side_clear or fwd_clear)

    stream = torch.cuda.current_stream(dev)
    for _ in range(args.warmup):
        fwd()
        bwd()
    torch.cuda.synchronize(dev)
    if msda.device_status() != 0:
        raise RuntimeError("device status set during warm-up")

    l2_gather_gbs, l2_red_gbs = l2_rates(dev, stream)

    # timed region: exactly K steps, per-call events on the launching stream
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True),
            torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        start.record(stream)
        for i in range(args.steps):
            evs[i][0].record(stream)
            fwd()
            evs[i][1].record(stream)
            bwd()
            evs[i][2].record(stream)
        end.record(stream)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    total_ms = start.elapsed_time(end)
    fwd_ms = sum(a.elapsed_time(b) for a, b, _ in evs) / args.steps
    bwd_ms = sum(b.elapsed_time(c) for _, b, c in evs) / args.steps
    step_us = sorted(a.elapsed_time(c) * 1e3 for a, _, c in evs)
    total_ms, fwd_ms, bwd_ms = max_over_ranks([total_ms, fwd_ms, bwd_ms], dev)
    ms_per_step = total_ms / args.steps
    if msda.device_status() != 0:
        raise RuntimeError("device status set during the timed region")

    # End to end through the public API with host buffers (pinned): every step copies its inputs host->device,
    # runs the forward and backward, and reads its result back device->host.  The result is `out`, the
    # forward's output: the gradients are consumed on the device by the layers upstream of the operator (a
    # second run also copies all three gradients back, for hosts that want them).  Consecutive steps overlap on
    # three streams (copy-in, compute, copy-out) with two buffer sets, as an input pipeline would; the timed
    # steps start from an empty pipeline, so their count amortises one fill.
    h_in = [x.cpu().pin_memory() for x in (pr.feat, pr.sampling_location, pr.weights, pr.grad_out)]
    h2d = sum(x.numel() * x.element_size() for x in h_in)
    slots = []
    for _ in range(2):
        d_in = [torch.empty_like(x, device=dev) for x in h_in]
        d_out = [torch.empty_like(x) for x in (out, gf, gl, gw)]
        slots.append((d_in, d_out, [torch.empty(x.shape, dtype=x.dtype).pin_memory() for x in d_out]))
    nsplit = max(1, args.copy_streams)
    s_in = [torch.cuda.Stream(dev) for _ in range(nsplit)]
    s_out = [torch.cuda.Stream(dev) for _ in range(nsplit)]
    ev_in, ev_comp, ev_out = ([[torch.cuda.Event() for _ in range(nsplit)] for _ in range(2)] for _ in range(3))

    def split_copy(dsts, srcs, streams, wait, done):
        # every tensor cut into len(streams) contiguous pieces, piece q on stream q
        for q, st in enumerate(streams):
            st.wait_event(wait)
            with torch.cuda.stream(st):
                for dd, ss in zip(dsts, srcs):
                    n = dd.numel()
                    lo, hi = n * q // len(streams), n * (q + 1) // len(streams)
                    if hi > lo:
                        dd.view(-1)[lo:hi].copy_(ss.view(-1)[lo:hi], non_blocking=True)
            done[q].record(st)

    def run_e2e(sel, nsteps):
        """ms per step of the pipelined end-to-end step reading back outputs `sel` (of out, gf, gl, gw), the
        bytes it reads back, and the ms of the same copies alone (both directions at once)."""
        def e2e_step(i):
            j = i % 2
            d_in, d_out, h_out = slots[j]
            # copy-in waits until the compute that last read this slot's inputs is done
            split_copy(d_in, h_in, s_in, ev_comp[j][0], ev_in[j])
            for e in ev_in[j]:
                main.wait_event(e)
            for e in ev_out[j]:
                main.wait_event(e)  # this slot's outputs have been copied out
            tens = (d_in[0], d.spatial_shape, d.scale_start_index, d_in[1], d_in[2])
            fwd(tens, d_out)
            bwd(tens, d_in[3], d_out)
            ev_comp[j][0].record(main)
            split_copy([h_out[q] for q in sel], [d_out[q] for q in sel], s_out, ev_comp[j][0], ev_out[j])

        for i in range(2):
            e2e_step(i)
        torch.cuda.synchronize(dev)
        runs = []
        for _ in range(3):  # three passes of nsteps, each from an empty pipeline; the median is reported
            if world > 1:
                torch.distributed.barrier()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(main)
            for i in range(nsteps):
                e2e_step(i)
            for st in s_out:
                main.wait_stream(st)
            s1.record(main)
            torch.cuda.synchronize(dev)
            runs.append(s0.elapsed_time(s1) / nsteps)
        e2e_ms = max_over_ranks([sorted(runs)[1]], dev)[0]

        # the same copies alone (one step's inputs in and outputs out, both directions at once): the floor of
        # the end-to-end step on this host link
        def copies_only():
            s_in[0].wait_stream(main)
            s_out[0].wait_stream(main)
            with torch.cuda.stream(s_in[0]):
                for dd, ss in zip(slots[0][0], h_in):
                    dd.copy_(ss, non_blocking=True)
            with torch.cuda.stream(s_out[0]):
                for q in sel:
                    slots[1][2][q].copy_(slots[1][1][q], non_blocking=True)
            main.wait_stream(s_in[0])
            main.wait_stream(s_out[0])

        copies_only()
        torch.cuda.synchronize(dev)
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(main)
        for _ in range(3):
            copies_only()
        c1.record(main)
        torch.cuda.synchronize(dev)
        copy_ms = max_over_ranks([c0.elapsed_time(c1) / 3], dev)[0]
        return e2e_ms, sum(slots[0][2][q].numel() * slots[0][2][q].element_size() for q in sel), copy_ms

    e2e_ms, d2h, copy_ms = run_e2e((0,), args.e2e_steps)
    e2e_all_ms, d2h_all, copy_all_ms = run_e2e((0, 1, 2, 3), max(3, args.e2e_steps // 2))

    hbm_peak, peak_src = peaks()
    feat_mb = d.feat.numel() * d.feat.element_size() / 1e6
    gf_mb = gf.numel() * 4 / 1e6
    l2_mb = getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 126 << 20) / 1e6
    l2_note = (f"inputs larger than L2 (feat {feat_mb:.0f} MB, grad_feat {gf_mb:.0f} MB per step, L2 {l2_mb:.0f} MB); "
               f"no flush" if feat_mb + gf_mb > 2 * l2_mb else
               f"inputs fit in L2 (feat {feat_mb:.0f} MB, grad_feat {gf_mb:.0f} MB): warm-cache timing")
    frames = world * B
    us_per_frame = ms_per_step * 1e3 / frames
    # dominant call and its roofline (algorithmic HBM bytes / measured duration)
    if bwd_ms >= fwd_ms:
        dom, dom_ms, dom_bytes = "msda_backward", bwd_ms, cnt.bwd_hbm_bytes
        traffic = load_traffic("msda_backward_det" if det else "msda_backward_atomic")
    else:
        dom, dom_ms, dom_bytes = "msda_forward", fwd_ms, cnt.fwd_hbm_bytes
        traffic = load_traffic("msda_forward")
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9
    t_hbm_fwd = cnt.fwd_hbm_bytes / (hbm_peak * 1e9) * 1e6
    t_l2_fwd = cnt.fwd_l2_gather_bytes / (l2_gather_gbs * 1e9) * 1e6
    t_hbm_bwd = cnt.bwd_hbm_bytes / (hbm_peak * 1e9) * 1e6
    red_bytes = cnt.bwd_l2_bytes - cnt.fwd_l2_gather_bytes
    if det:
        # the deterministic backward reduces nothing in L2: it gathers the corner rows (dloc, dw) and, per
        # in-bound corner, its anchor's FP32 grad_out row (the same bytes the atomic form reduces)
        bwd_gather_bytes = cnt.fwd_l2_gather_bytes + red_bytes
        t_red_bwd = 0.0
    else:
        bwd_gather_bytes = cnt.fwd_l2_gather_bytes
        t_red_bwd = red_bytes / (l2_red_gbs * 1e9) * 1e6
    t_gather_bwd = bwd_gather_bytes / (l2_gather_gbs * 1e9) * 1e6
    t_roof_bwd = max(t_hbm_bwd, t_gather_bwd, t_red_bwd)
    line = {
        "metric": METRIC, "value": us_per_frame, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16", "accumulate": "f32", "data": "synthetic",
        "config": {"workload": wl_desc, "frames_per_step_per_gpu": B, "parallelism": f"replicas x{world}",
                   "backward": "deterministic" if det else "atomic",
                   "grad_feat_clear": None if det else {
                       "forward": "inside the forward kernel (msda_forward_train)",
                       "side": "torch fill on a side stream during the forward",
                       "inline": "memset inside msda_backward"}[args.clear],
                   "l2": l2_note},
        "gsamples_per_s": cnt.nominal_samples * frames / (ms_per_step * 1e-3) / 1e9,
        "inview_gsamples_per_s": cnt.inview_samples * frames / (ms_per_step * 1e-3) / 1e9,
        "fwd_us": fwd_ms * 1e3, "bwd_us": bwd_ms * 1e3,
        "step_us_p50": step_us[len(step_us) // 2], "step_us_p99": step_us[min(len(step_us) - 1, int(0.99 * len(step_us)))],
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic, "peak_source": peak_src,
                     "algorithmic_bytes": dom_bytes,
                     # the resource that actually binds the dominant call, measured live in this run
                     "binding": ({"resource": "L2 FP32 vector reductions (msda_probe_reduce)",
                                  "achieved": red_bytes / (bwd_ms * 1e-3) / 1e9, "peak": l2_red_gbs, "unit": "GB/s",
                                  "frac": t_red_bwd / (bwd_ms * 1e3)} if dom == "msda_backward" and not det else
                                 {"resource": "L2 random-row gathers (msda_probe_read): corner rows and grad_out rows",
                                  "achieved": bwd_gather_bytes / (bwd_ms * 1e-3) / 1e9, "peak": l2_gather_gbs,
                                  "unit": "GB/s", "frac": t_gather_bwd / (bwd_ms * 1e3)} if dom == "msda_backward" else
                                 {"resource": "L2 random-row gathers (msda_probe_read)",
                                  "achieved": cnt.fwd_l2_gather_bytes / (fwd_ms * 1e-3) / 1e9, "peak": l2_gather_gbs,
                                  "unit": "GB/s", "frac": t_l2_fwd / (fwd_ms * 1e3)} if dom == "msda_forward" else
                                 None)},
        "gather_roofline": {
            "l2_gather_gbs_measured": l2_gather_gbs,
            "l2_reduce_gbs_measured": l2_red_gbs,
            "fwd": {"t_hbm_us": t_hbm_fwd, "t_l2_us": t_l2_fwd, "t_roof_us": max(t_hbm_fwd, t_l2_fwd),
                    "t_us": fwd_ms * 1e3, "frac": max(t_hbm_fwd, t_l2_fwd) / (fwd_ms * 1e3)},
            "bwd": {"t_hbm_us": t_hbm_bwd, "t_l2_gather_us": t_gather_bwd, "t_l2_reduce_us": t_red_bwd,
                    "t_roof_us": t_roof_bwd, "t_us": bwd_ms * 1e3, "frac": t_roof_bwd / (bwd_ms * 1e3)}},
        "counts": cnt.as_dict(),
        "e2e": {"value": e2e_ms * 1e3 / B, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": args.e2e_steps,
                "reads_back": "out (the forward's result); the gradients stay on the device for the layers upstream",
                "pipeline": f"copy-in, compute and copy-out of consecutive steps overlap (2 buffer sets; each "
                            f"direction's copies cut over {nsplit} streams); the median of three passes of "
                            f"{args.e2e_steps} steps, each timed from an empty pipeline",
                "copy_floor": {"value": copy_ms * 1e3 / B, "unit": UNIT, "frac": copy_ms / e2e_ms,
                               "what": "the step's host<->device copies alone, both directions at once"},
                "with_gradients_to_host": {
                    "value": e2e_all_ms * 1e3 / B, "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h_all, "steps": max(3, args.e2e_steps // 2),
                    "reads_back": "out, grad_feat, grad_loc, grad_weights",
                    "copy_floor": {"value": copy_all_ms * 1e3 / B, "unit": UNIT, "frac": copy_all_ms / e2e_all_ms}}},
        "gpu_launches": ((2 if fwd_ws is not None and not fwd_clear else 1) + backward_launches(det, fwd_clear))
                        * args.steps,
        "tuning": {"forward": ft, "backward": bt},
        "clocks": clk.summary(),
        "gpu": torch.cuda.get_device_name(dev),
    }
    if rank == 0 and world == 1 and not args.no_forms:
        line["forms"] = other_forms(dev, stream, pr, cnt, det, l2_gather_gbs, l2_red_gbs, hbm_peak,
                                    tune_it=not args.no_tune)
    if args.with_batched and "forms" not in line:
        line["batched_serving"] = batched_serving(dev, stream, tune_it=not args.no_tune)
    if args.extras:
        line["extras"] = extras(pr, dev, ft)
    if args.configs:
        line["other_workloads"] = other_configs(dev, l2_gather_gbs, l2_red_gbs, hbm_peak)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(pr, args.cpu_sample_anchors, others=args.configs)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
