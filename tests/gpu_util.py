"""Helpers shared by the GPU parity tests (oracle runs, error metrics)."""
import os

import numpy as np
import torch

import oracle
from paper_2601_10819_gb300 import build as msda_build
from paper_2601_10819_gb300 import msda

# Tolerances: max-abs error over max-abs reference, per output tensor.
TOL_FP32 = 1e-5      # FP32 features and weights
TOL_LOWP_OUT = 1e-2  # BF16/FP16 features (both sides see the same rounded inputs)
TOL_LOWP_GRAD = 2e-2

NTHREADS = max(1, min(32, os.cpu_count() or 1))


def ensure_lib():
    msda_build.build()
    return msda.load()


def relerr(y, r) -> float:
    y = np.asarray(y, dtype=np.float64)
    r = np.asarray(r, dtype=np.float64)
    den = np.abs(r).max() if r.size else 0.0
    if den == 0.0:
        return float(np.abs(y).max()) if y.size else 0.0
    return float(np.abs(y - r).max() / den)


def to_dev(pr, device="cuda"):
    return pr.to(device)


def gpu_forward(pr, **kw):  # kw: out_dtype, workspace, warps, variant, vec
    d = pr.to("cuda")
    out = msda.forward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights, **kw)
    torch.cuda.synchronize()
    return out


def oracle_forward(pr):
    return oracle.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, pr.weights,
                          nthreads=NTHREADS)


def oracle_backward(pr):
    return oracle.backward(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, pr.weights,
                           pr.grad_out)


def is_lowp(pr):
    return pr.feat.dtype != torch.float32 or pr.weights.dtype != torch.float32
