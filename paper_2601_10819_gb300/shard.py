"""Camera sharding of one MSDA problem across ranks.

The operator is a sum over cameras (Sec. 3.2 and 5.3 of the paper), so a
problem splits exactly by camera: rank r takes a subset of the cameras
(their feature maps, and the location and weight slices of those cameras),
computes a partial output [B, A, C] in FP32, and one sum all-reduce of the
partial outputs gives the full result.  The backward needs grad_out on every
rank; the feature, location and weight gradients of a camera stay on the
rank that owns it.

This module holds only the host-side slicing and the reduction; each rank
computes its shard with ``msda.forward`` / ``msda.backward``.
"""
from __future__ import annotations

from typing import List, Sequence, Tuple

import torch


def split_cameras(ncam: int, world: int) -> List[List[int]]:
    """Contiguous, balanced camera subsets, one per rank (some may be empty)."""
    base, extra = divmod(ncam, world)
    out, k = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(list(range(k, k + n)))
        k += n
    return out


def shard_problem(feat, spatial_shape, scale_start_index, sampling_location, weights,
                  cams: Sequence[int]) -> Tuple[torch.Tensor, ...]:
    """The sub-problem of cameras `cams`, with its maps re-packed densely.

    Returns (feat, spatial_shape, scale_start_index, sampling_location, weights)
    of the shard; the feature rows of every map of the shard are copied into
    a new [B, sum_hw_shard, C] tensor in camera-major, scale-major order.
    """
    cams = list(cams)
    shape = spatial_shape[cams].contiguous()
    start = scale_start_index[cams]
    rows, new_start, off = [], torch.zeros_like(shape[..., 0]), 0
    for i in range(len(cams)):
        for s in range(shape.shape[1]):
            h, w = int(shape[i, s, 0]), int(shape[i, s, 1])
            st = int(start[i, s])
            rows.append(torch.arange(st, st + h * w, device=feat.device))
            new_start[i, s] = off
            off += h * w
    idx = torch.cat(rows) if rows else torch.zeros(0, dtype=torch.long, device=feat.device)
    sub_feat = feat[:, idx].contiguous()
    loc = sampling_location[:, :, :, cams].contiguous()
    w = weights[:, :, :, cams].contiguous()
    return sub_feat, shape, new_start.to(torch.int32).contiguous(), loc, w


def reduce_partials(out: torch.Tensor, group=None) -> torch.Tensor:
    """Sum the ranks' partial outputs in place (one all-reduce)."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(out, op=dist.ReduceOp.SUM, group=group)
    return out
