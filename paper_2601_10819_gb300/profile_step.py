"""Run the operator's training step a fixed number of times, for a profiler.

    python -m paper_2601_10819_gb300.profile_step --workload outside-in-64cam --steps 3 --warps 8 --vec 2
    python -m paper_2601_10819_gb300.profile_step --workload outside-in-64cam --ncam 32 --steps 2   # half the maps

Each step is one msda_forward and one msda_backward (deterministic by default, ``--atomic`` for the
atomic mode; ``--forward-only`` drops the backward) on a seeded synthetic workload, with an explicit launch
mapping and preallocated outputs and workspace, so every step launches the same kernels in the same order
and a profiler can pick a launch by its kernel name and index.  Nothing is tuned or timed here.
"""
from __future__ import annotations

import argparse
import sys

import torch

from . import inputs, msda

# name -> (workload index, feature dtype, weight dtype)
WORKLOADS = {
    "outside-in-64cam": (2, None, None),
    "train-16cam": (3, None, None),
    "sparse4d-6cam": (1, None, None),
    "sparse4d-6cam-bf16": (1, "bf16", "bf16"),
}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--workload", default="outside-in-64cam", choices=sorted(WORKLOADS))
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warps", type=int, default=8, help="warps per block (forward and backward)")
    ap.add_argument("--vec", type=int, default=2, help="16-byte vectors per lane")
    ap.add_argument("--ncam", type=int, default=None, help="fewer cameras (64- and 16-camera workloads)")
    ap.add_argument("--batch", type=int, default=None, help="fewer frames (16-camera workload)")
    ap.add_argument("--atomic", action="store_true", help="atomic backward instead of the deterministic one")
    ap.add_argument("--forward-only", action="store_true")
    args = ap.parse_args(argv)

    idx, fdt, wdt = WORKLOADS[args.workload]
    pr = inputs.make_workload(idx, feat_dtype=fdt, w_dtype=wdt, with_grad=not args.forward_only, ncam=args.ncam,
                              batch=args.batch).to("cuda")
    T = pr.tensors()
    B, sum_hw, C = pr.feat.shape
    _, A, P, K, _ = pr.sampling_location.shape
    S, G = pr.weights.shape[4], pr.weights.shape[5]
    det = not args.atomic
    out = torch.empty(B, A, C, device="cuda")
    if not args.forward_only:
        ws = torch.empty(max(msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, det), 16), dtype=torch.uint8,
                         device="cuda")
        grads = (torch.empty(B, sum_hw, C, device="cuda"), torch.empty(B, A, P, K, 2, device="cuda"),
                 torch.empty(B, A, P, K, S, G, device="cuda"))
    for _ in range(args.steps):
        msda.forward(*T, out=out, warps=args.warps, vec=args.vec)
        if not args.forward_only:
            msda.backward(*T, pr.grad_out, deterministic=det, workspace=ws, grads=grads, warps=args.warps,
                          vec=args.vec)
    torch.cuda.synchronize()
    status = msda.device_status()
    print(f"{args.workload} (B={B}, {K} cameras): {args.steps} steps, device status {status}")
    return 0 if status == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
