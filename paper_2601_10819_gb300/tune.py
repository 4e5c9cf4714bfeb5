"""Autotuner for the MSDA launch mappings.

For one problem signature (shapes, dtypes, GPU name) it times every
candidate mapping of the forward, the backward and the batched forward with
CUDA events and keeps the fastest.  Results are cached as JSON (path from
``MSDA_TUNE_CACHE``, default ``~/.cache/msda_gb300/tune.json``), so a
signature is searched once per GPU model; signatures measured on GB300 ship
with the package (``tuned_gb300.json``) and are used when the cache has no
entry.  Every candidate computes the same
operator; the mappings differ only in how lanes, warps and blocks are laid
out (and therefore in the order of FP32 sums).
"""
from __future__ import annotations

import json
import os
import threading
from typing import Dict, Optional

import torch

from . import msda

_lock = threading.Lock()

FWD_CANDIDATES = [dict(vec=v, warps=w, workspace=False) for v in (1, 2, 4) for w in (2, 4, 8)] + \
                 [dict(vec=0, warps=0, workspace=True)]
BWD_CANDIDATES = [dict(vec=v, warps=w) for v in (1, 2, 4) for w in (2, 4, 8)]
BATCHED_CANDIDATES = [dict(vec=v, warps=w, bps=b) for v in (1, 2, 4) for w in (2, 4, 8) for b in (0, 4, 8)]


def cache_path() -> str:
    return os.environ.get("MSDA_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "msda_gb300",
                                                          "tune.json"))


SHIPPED = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")


def _load() -> Dict:
    d = {}
    for path in (SHIPPED, cache_path()):
        try:
            with open(path) as f:
                d.update(json.load(f))
        except Exception:
            pass
    return d


def _store(d: Dict):
    path = cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(d, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only loses the cache


def signature(kind: str, tensors, extra: str = "") -> str:
    feat, shape, start, loc, w = tensors
    B, sum_hw, C = feat.shape
    _, A, P, K, _ = loc.shape
    S, G = w.shape[4], w.shape[5]
    dev = torch.cuda.get_device_name(feat.device)
    return (f"{dev}|{kind}|B{B} hw{sum_hw} C{C} K{K} S{S} A{A} P{P} G{G} "
            f"{str(feat.dtype).split('.')[-1]}/{str(w.dtype).split('.')[-1]}{extra}")


def _time(fn, reps: int = 5) -> float:
    fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _best(kind: str, sig: str, candidates, run, force: bool) -> Dict:
    with _lock:
        cache = _load()
        if not force and sig in cache:
            return cache[sig]["best"]
    results = []
    for cand in candidates:
        try:
            t = _time(lambda: run(cand))
        except msda.MSDAError:
            continue
        results.append((t, cand))
    if not results:
        raise RuntimeError(f"no valid {kind} mapping")
    results.sort(key=lambda x: x[0])
    best = dict(results[0][1])
    with _lock:
        try:
            with open(cache_path()) as f:
                cache = json.load(f)
        except Exception:
            cache = {}
        cache[sig] = {"best": best, "ms": results[0][0],
                      "all": [{"ms": t, **c} for t, c in results]}
        _store(cache)
    return best


def tune_forward(tensors, out: torch.Tensor, workspace: Optional[torch.Tensor] = None, force: bool = False) -> Dict:
    """Fastest forward mapping for these tensors: {vec, warps, workspace}."""
    sig = signature("fwd", tensors)

    def run(c):
        msda.forward(*tensors, out=out, workspace=workspace if c["workspace"] else None,
                     warps=c["warps"] or None, vec=c["vec"])

    cands = FWD_CANDIDATES if workspace is not None else [c for c in FWD_CANDIDATES if not c["workspace"]]
    return _best("forward", sig, cands, run, force)


def tune_backward(tensors, grad_out, grads, deterministic: bool = False, workspace=None, force: bool = False) -> Dict:
    """Fastest backward mapping for these tensors: {vec, warps}."""
    sig = signature("bwd-det" if deterministic else "bwd", tensors)

    def run(c):
        msda.backward(*tensors, grad_out, deterministic=deterministic, workspace=workspace, grads=grads,
                      warps=c["warps"], vec=c["vec"])

    return _best("backward", sig, BWD_CANDIDATES, run, force)


def tune_batched(scenes, force: bool = False) -> Dict:
    """Fastest persistent-launch mapping for a list of scenes: {vec, warps, bps}."""
    s0 = scenes[0]
    extra = f" scenes{len(scenes)} A{sum(s.sampling_location.shape[1] for s in scenes)}" \
            f" K{sum(s.sampling_location.shape[3] for s in scenes)}"
    sig = signature("batched", s0.tensors(), extra)
    plans = {}

    def run(c):
        key = (c["vec"], c["warps"], c["bps"])
        if key not in plans:
            plans[key] = msda.plan_batched(scenes, warps=c["warps"], blocks_per_sm=c["bps"] or None, vec=c["vec"])
        plans[key].run()

    return _best("batched", sig, BATCHED_CANDIDATES, run, force)


def main():
    """Search the benchmark workloads on this GPU and write a tuning table."""
    import argparse
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=SHIPPED)
    args = ap.parse_args()
    from . import inputs
    os.environ["MSDA_TUNE_CACHE"] = args.out + ".search.json"
    dev = torch.device("cuda")
    pr = inputs.make_workload(2).to(dev)
    T = pr.tensors()
    B, sum_hw, C = pr.feat.shape
    _, A, P, K, _ = pr.sampling_location.shape
    S, G = pr.weights.shape[4:]
    out = torch.empty(B, A, C, device=dev)
    fws = torch.empty(msda.forward_workspace_size(B, sum_hw, C, K, S, A, P, G), dtype=torch.uint8, device=dev)
    grads = (torch.zeros(B, sum_hw, C, device=dev), torch.empty(B, A, P, K, 2, device=dev),
             torch.empty(B, A, P, K, S, G, device=dev))
    ws = torch.empty(msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, False), dtype=torch.uint8, device=dev)
    tune_forward(T, out, workspace=fws, force=True)
    tune_backward(T, pr.grad_out, grads, workspace=ws, force=True)
    dws = torch.empty(msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, True), dtype=torch.uint8, device=dev)
    tune_backward(T, pr.grad_out, grads, deterministic=True, workspace=dws, force=True)
    scenes = [s.to(dev) for s in inputs.make_workload(4, with_grad=False)]
    tune_batched(scenes, force=True)
    with open(os.environ["MSDA_TUNE_CACHE"]) as f:
        found = json.load(f)
    table = {k: {"best": v["best"], "ms": round(v["ms"], 4)} for k, v in found.items()}
    with open(args.out, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    print(json.dumps(table, indent=1))


if __name__ == "__main__":
    main()
