"""Algorithmic byte counts of the MSDA kernels, computed exactly from the inputs.

Used by bench.py to turn kernel times into roofline fractions.  The counts
are the minimum traffic of the operator, independent of how a kernel is
written:

forward
  HBM:  every feature row touched by at least one in-bound corner (read
        once) + all sampling locations (needed to decide visibility) + the
        weights of in-view point-scales (G values each) + the output.
  L2:   gathered corner bytes = C * sizeof(feat) per in-bound corner (what
        the SMs pull through L2 when nothing is reused on chip).
backward (atomic or deterministic)
  HBM:  the forward's feature, location and weight reads + grad_out + one
        write of grad_feat (all rows: untouched rows are zero) + grad_loc +
        grad_weights.
  L2:   the corner gathers again + C * 4 bytes of FP32 gradient per
        in-bound corner (the scatter).
A point-scale is in view when its bilinear footprint overlaps the map
(x = u*W - 0.5 in (-1, W), y = v*H - 0.5 in (-1, H)).
"""
from __future__ import annotations

from dataclasses import dataclass, asdict

import numpy as np
import torch


@dataclass
class Counts:
    nominal_samples: int      # B*A*P*Ncam*Nscale
    inview_samples: int       # point-scales whose footprint overlaps the map
    inbound_corners: int
    touched_rows: int
    total_rows: int
    fwd_hbm_bytes: int
    fwd_l2_gather_bytes: int
    bwd_hbm_bytes: int
    bwd_l2_bytes: int

    def as_dict(self):
        return asdict(self)


def count(pr, grad_dtype_bytes: int = 4) -> Counts:
    feat, shape, start, loc, w = pr.tensors()
    B, sum_hw, C = feat.shape
    _, A, P, K, _ = loc.shape
    S = shape.shape[1]
    G = w.shape[-1]
    fe = feat.element_size()
    we = w.element_size()
    u = loc[..., 0].double().numpy()   # [B, A, P, K]
    v = loc[..., 1].double().numpy()
    shp = shape.numpy()
    st = start.numpy()
    touched = np.zeros((B, sum_hw), dtype=bool)
    inview = 0
    corners = 0
    for k in range(K):
        for s in range(S):
            H, W = int(shp[k, s, 0]), int(shp[k, s, 1])
            x = u[..., k] * W - 0.5
            y = v[..., k] * H - 0.5
            ok = (x > -1) & (x < W) & (y > -1) & (y < H)
            inview += int(ok.sum())
            xs = np.floor(np.where(ok, x, 0)).astype(np.int64)
            ys = np.floor(np.where(ok, y, 0)).astype(np.int64)
            for dy in (0, 1):
                for dx in (0, 1):
                    i, j = ys + dy, xs + dx
                    m = ok & (i >= 0) & (i < H) & (j >= 0) & (j < W)
                    corners += int(m.sum())
                    b_idx = np.broadcast_to(np.arange(B)[:, None, None], m.shape)[m]
                    rows = int(st[k, s]) + i[m] * W + j[m]
                    touched[b_idx, rows] = True
    n_touched = int(touched.sum())
    nominal = B * A * P * K * S
    loc_bytes = B * A * P * K * 2 * 4
    w_inview = inview * G * we
    out_bytes = B * A * C * 4
    fwd_hbm = n_touched * C * fe + loc_bytes + w_inview + out_bytes
    fwd_l2 = corners * C * fe
    bwd_hbm = (n_touched * C * fe + loc_bytes + w_inview + out_bytes      # inputs + grad_out
               + B * sum_hw * C * grad_dtype_bytes                        # grad_feat written once
               + loc_bytes + nominal * G * 4)                             # grad_loc, grad_weights
    bwd_l2 = corners * C * fe + corners * C * grad_dtype_bytes
    return Counts(nominal, inview, corners, n_touched, B * sum_hw, fwd_hbm, fwd_l2, bwd_hbm, bwd_l2)
