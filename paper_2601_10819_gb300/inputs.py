"""Seeded synthetic inputs for Multi-Scale Deformable Aggregation.

This module only draws random tensors; it holds none of the operator's
arithmetic, so both the CUDA path and the FP64 oracle may consume what it
produces.  The paper's data (AI City 2025 video and a trained Sparse4D
model) is not available, so these tensors stand in for the operator's inputs
with the shapes of the paper's outside-in workloads:

* feature maps ``feat[B, sum_hw, C]`` ~ N(0, 1) (times a scale), packed
  camera-major then scale-major, so ``start[k, s]`` is the running sum of the
  map areas;
* normalised sampling locations ``loc[B, A, P, Ncam, 2]`` ~ U[lo, hi]^2; for
  a fraction of (anchor, camera) pairs, chosen by a seeded permutation, 2.0
  is added to ``u`` of all keypoints so that the whole pair is out of view;
* weights ``w[B, A, P, Ncam, Nscale, G]`` = softmax over (P, Ncam, Nscale),
  for each (b, a, g), of N(0, 1) logits;
* an upstream gradient ``grad_out[B, A, C]`` ~ N(0, 1).

Reduced-precision tensors are drawn in FP32 and rounded to nearest-even once
(``Tensor.to``); both sides consume the rounded values.  Each workload is
seeded with its index, and the draws happen in a fixed order: feat,
locations, logits, out-of-view permutation, grad_out (the batched serving
workload first draws its per-scene sizes).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Sequence, Tuple

import torch

_DTYPES = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}

# Feature-map sizes.  The Sparse4D-shaped maps are a 256x704 image at strides
# 4..32; the outside-in maps are a 540x960 network input (1080p halved) at
# strides 8..64, each side rounded up; 720p gives 360x640 by the same rule.
SPARSE4D_MAPS = [(64, 176), (32, 88), (16, 44), (8, 22)]


def video_maps(height: int, width: int, strides: Sequence[int] = (8, 16, 32, 64)) -> List[Tuple[int, int]]:
    """Map sizes of a ``height x width`` video frame fed at half resolution."""
    return [(math.ceil(height / 2 / s), math.ceil(width / 2 / s)) for s in strides]


MAPS_1080P = video_maps(1080, 1920)   # 68x120, 34x60, 17x30, 9x15
MAPS_720P = video_maps(720, 1280)     # 45x80, 23x40, 12x20, 6x10


@dataclass
class Problem:
    """One MSDA problem (one launch of the single-scene entry points)."""
    feat: torch.Tensor                 # [B, sum_hw, C]
    spatial_shape: torch.Tensor        # [Ncam, Nscale, 2] int32 (H, W)
    scale_start_index: torch.Tensor    # [Ncam, Nscale] int32
    sampling_location: torch.Tensor    # [B, A, P, Ncam, 2] float32 (u, v)
    weights: torch.Tensor              # [B, A, P, Ncam, Nscale, G]
    grad_out: Optional[torch.Tensor]   # [B, A, C] float32
    name: str = ""
    meta: Dict = field(default_factory=dict)

    @property
    def dims(self) -> Dict[str, int]:
        B, sum_hw, C = self.feat.shape
        _, A, P, Ncam, _ = self.sampling_location.shape
        Nscale = self.spatial_shape.shape[1]
        G = self.weights.shape[-1]
        return dict(B=B, sum_hw=sum_hw, C=C, Ncam=Ncam, Nscale=Nscale, A=A, P=P, G=G)

    def tensors(self):
        return (self.feat, self.spatial_shape, self.scale_start_index,
                self.sampling_location, self.weights)

    def to(self, device) -> "Problem":
        mv = lambda t: None if t is None else t.to(device)
        return Problem(mv(self.feat), mv(self.spatial_shape), mv(self.scale_start_index),
                       mv(self.sampling_location), mv(self.weights), mv(self.grad_out),
                       self.name, dict(self.meta))

    def anchors(self, idx) -> "Problem":
        """The same problem restricted to the anchors ``idx`` (anchors are independent)."""
        idx = torch.as_tensor(idx, dtype=torch.long)
        go = None if self.grad_out is None else self.grad_out[:, idx]
        meta = dict(self.meta)
        if meta.get("out_mask") is not None:
            meta["out_mask"] = meta["out_mask"][:, idx]
        return Problem(self.feat, self.spatial_shape, self.scale_start_index,
                       self.sampling_location[:, idx].contiguous(), self.weights[:, idx].contiguous(),
                       None if go is None else go.contiguous(), self.name + "[anchors]", meta)


def make_visibility(pr: Problem, seed: int, zero_frac: float = 0.1) -> torch.Tensor:
    """Visibility scores [B, A, Ncam] for the occlusion-aware fusion: U(0, 1),
    0 for the (anchor, camera) pairs pushed out of view, and 0 for a further
    seeded `zero_frac` of pairs (occluded).  Drawn from its own generator so
    the problem's draws are unchanged."""
    gen = torch.Generator().manual_seed(10_000 + seed)
    B, A, _, K, _ = pr.sampling_location.shape
    v = torch.rand(B, A, K, generator=gen, dtype=torch.float32)
    v[torch.rand(B, A, K, generator=gen) < zero_frac] = 0.0
    mask = pr.meta.get("out_mask")
    if mask is not None:
        v[mask] = 0.0
    return v.contiguous()


def look_at_camera(eye, target, focal: float, width: int, height: int) -> torch.Tensor:
    """3x4 world -> homogeneous pixel matrix of a pinhole camera at `eye`
    looking at `target` (world z up), principal point at the image centre."""
    eye = torch.as_tensor(eye, dtype=torch.float64)
    fwd = torch.as_tensor(target, dtype=torch.float64) - eye
    fwd = fwd / fwd.norm()
    right = torch.linalg.cross(fwd, torch.tensor([0.0, 0.0, 1.0], dtype=torch.float64))
    right = right / right.norm()
    down = torch.linalg.cross(fwd, right)
    R = torch.stack([right, down, fwd])                  # world -> camera rows
    t = -R @ eye
    K = torch.tensor([[focal, 0.0, width / 2.0], [0.0, focal, height / 2.0], [0.0, 0.0, 1.0]], dtype=torch.float64)
    return K @ torch.cat([R, t[:, None]], dim=1)


def make_scene_geometry(seed: int, B: int, A: int, P: int, ncam: int, img=(1920, 1080)):
    """Synthetic outside-in rig and anchors for the keypoint prologue.

    Cameras sit on a 30 m circle at 6 m height looking at the centre of a
    40 m x 40 m floor; anchors are boxes on the floor (sizes 0.5..2 m, any
    yaw, velocity ~ N(0, 1) m/s, dt = 0.1 s); the first 7 keypoints are the
    box centre and its six face centres at 0.45 box units, the rest are
    learned-style offsets ~ U[-0.5, 0.5]^3.  Returns anchors [B, A, 11],
    offsets [B, A, P, 3], dt [B], proj [B, ncam, 3, 4], img_wh [ncam, 2]
    (float32)."""
    gen = torch.Generator().manual_seed(20_000 + seed)
    ctr = torch.rand(B, A, 3, generator=gen) * torch.tensor([40.0, 40.0, 1.0]) - torch.tensor([20.0, 20.0, 0.0])
    size = torch.rand(B, A, 3, generator=gen) * 1.5 + 0.5
    yaw = torch.rand(B, A, generator=gen) * 2 * math.pi - math.pi
    vel = torch.randn(B, A, 3, generator=gen)
    anchors = torch.cat([ctr, size, torch.sin(yaw)[..., None], torch.cos(yaw)[..., None], vel], dim=-1)
    fixed = torch.tensor([[0, 0, 0], [0.45, 0, 0], [-0.45, 0, 0], [0, 0.45, 0], [0, -0.45, 0], [0, 0, 0.45],
                          [0, 0, -0.45]], dtype=torch.float32)[:P]
    learned = torch.rand(B, A, max(0, P - fixed.shape[0]), 3, generator=gen) - 0.5
    offsets = torch.cat([fixed.expand(B, A, -1, -1), learned], dim=2)
    dt = torch.full((B,), 0.1)
    proj = []
    for k in range(ncam):
        ang = 2 * math.pi * k / max(ncam, 1)
        eye = [30 * math.cos(ang), 30 * math.sin(ang), 6.0]
        proj.append(look_at_camera(eye, [0.0, 0.0, 0.0], 1000.0, img[0], img[1]))
    proj = torch.stack(proj).float().expand(B, -1, -1, -1).contiguous()
    img_wh = torch.tensor([img] * ncam, dtype=torch.float32)
    return (anchors.float().contiguous(), offsets.float().contiguous(), dt, proj, img_wh)


def tables(cam_maps: Sequence[Sequence[Tuple[int, int]]]) -> Tuple[torch.Tensor, torch.Tensor, int]:
    """spatial_shape, scale_start_index and sum_hw for camera-major packing."""
    ncam = len(cam_maps)
    nscale = len(cam_maps[0])
    shape = torch.zeros(ncam, nscale, 2, dtype=torch.int32)
    start = torch.zeros(ncam, nscale, dtype=torch.int32)
    off = 0
    for k, maps in enumerate(cam_maps):
        if len(maps) != nscale:
            raise ValueError("every camera needs the same number of scales")
        for s, (h, w) in enumerate(maps):
            shape[k, s, 0], shape[k, s, 1] = h, w
            start[k, s] = off
            off += h * w
    return shape, start, off


def make_problem(gen: torch.Generator, *, B: int, cam_maps, C: int, G: int, A: int, P: int,
                 feat_scale: float = 1.0, loc_range: Tuple[float, float] = (0.0, 1.0),
                 out_frac: float = 0.0, feat_dtype: str = "f32", w_dtype: str = "f32",
                 with_grad: bool = True, name: str = "") -> Problem:
    """Draw one problem from ``gen`` in the fixed order described above."""
    shape, start, sum_hw = tables(cam_maps)
    ncam, nscale = shape.shape[0], shape.shape[1]
    feat = torch.randn(B, sum_hw, C, generator=gen, dtype=torch.float32)
    if feat_scale != 1.0:
        feat.mul_(feat_scale)
    feat = feat.to(_DTYPES[feat_dtype])
    lo, hi = loc_range
    loc = torch.rand(B, A, P, ncam, 2, generator=gen, dtype=torch.float32) * (hi - lo) + lo
    logits = torch.randn(B, A, P * ncam * nscale, G, generator=gen, dtype=torch.float64)
    w = torch.softmax(logits, dim=2).reshape(B, A, P, ncam, nscale, G)
    w = w.to(_DTYPES[w_dtype]).contiguous()
    n_out = int(round(out_frac * A * ncam))
    out_mask = torch.zeros(B, A, ncam, dtype=torch.bool)
    if n_out > 0:
        for b in range(B):
            perm = torch.randperm(A * ncam, generator=gen)[:n_out]
            out_mask[b].view(-1)[perm] = True
        loc[..., 0] += 2.0 * out_mask[:, :, None, :].to(loc.dtype)
    go = torch.randn(B, A, C, generator=gen, dtype=torch.float32) if with_grad else None
    meta = dict(out_frac=out_frac, feat_dtype=feat_dtype, w_dtype=w_dtype,
                n_out_pairs=int(out_mask.sum()), loc_range=loc_range, feat_scale=feat_scale,
                out_mask=out_mask)
    return Problem(feat.contiguous(), shape, start, loc.contiguous(), w, go, name, meta)


# ---------------------------------------------------------------------------
# The five workloads.  Index = seed.
# ---------------------------------------------------------------------------
WORKLOADS = {
    0: "tiny: B1 Ncam2 Nscale2 (16x16, 8x8) C32 G4 A16 P4, loc U[-0.1,1.1]^2, FP32",
    1: "sparse4d-6cam: B1 Ncam6 maps 64x176..8x22 C256 G8 A900 P13, loc U[-0.05,1.05]^2",
    2: "outside-in-64cam: B1 Ncam64 maps 68x120..9x15 C256 G8 A900 P13, feat N(0,1)*0.5, "
       "loc U[0,1]^2 with 40% of (anchor,camera) pairs out of view, BF16 feat+weights",
    3: "train-16cam: B4 Ncam16 maps 64x176..8x22 C256 G8 A900 P13, BF16 feat, FP32 weights, "
       "grad_out N(0,1)",
    4: "batched-serving: 16 scenes, Ncam U{4..96}, 720p/1080p maps, A U[600,1200], P13 C256 G8, BF16",
}


def make_workload(idx: int, *, feat_dtype: Optional[str] = None, w_dtype: Optional[str] = None,
                  with_grad: bool = True, ncam: Optional[int] = None, batch: Optional[int] = None):
    """Problem (or list of Problems for workload 4) of workload ``idx``.

    ``feat_dtype``/``w_dtype`` override the workload's dtypes; ``ncam`` and
    ``batch`` shrink workloads 2/3 for quick tests (the seed stays the index).
    """
    gen = torch.Generator().manual_seed(idx)
    if idx == 0:
        return make_problem(gen, B=1, cam_maps=[[(16, 16), (8, 8)]] * 2, C=32, G=4, A=16, P=4,
                            loc_range=(-0.1, 1.1), feat_dtype=feat_dtype or "f32",
                            w_dtype=w_dtype or "f32", with_grad=with_grad, name="tiny")
    if idx == 1:
        return make_problem(gen, B=1, cam_maps=[SPARSE4D_MAPS] * 6, C=256, G=8, A=900, P=13,
                            loc_range=(-0.05, 1.05), feat_dtype=feat_dtype or "f32",
                            w_dtype=w_dtype or "f32", with_grad=with_grad, name="sparse4d-6cam")
    if idx == 2:
        return make_problem(gen, B=1, cam_maps=[MAPS_1080P] * (ncam or 64), C=256, G=8, A=900,
                            P=13, feat_scale=0.5, loc_range=(0.0, 1.0), out_frac=0.4,
                            feat_dtype=feat_dtype or "bf16", w_dtype=w_dtype or "bf16",
                            with_grad=with_grad, name="outside-in-64cam")
    if idx == 3:
        return make_problem(gen, B=batch or 4, cam_maps=[SPARSE4D_MAPS] * (ncam or 16), C=256, G=8,
                            A=900, P=13, loc_range=(-0.05, 1.05), feat_dtype=feat_dtype or "bf16",
                            w_dtype=w_dtype or "f32", with_grad=with_grad, name="train-16cam")
    if idx == 4:
        return make_batched(gen, feat_dtype=feat_dtype or "bf16", w_dtype=w_dtype or "bf16",
                            with_grad=with_grad, n_scenes=batch or 16)
    raise ValueError(f"unknown workload {idx}")


def make_batched(gen: torch.Generator, *, n_scenes: int = 16, feat_dtype: str = "bf16",
                 w_dtype: str = "bf16", with_grad: bool = False, ncam_range=(4, 96),
                 a_range=(600, 1200)) -> List[Problem]:
    """Scenes of uneven camera count, resolution and anchor count."""
    ncams = torch.randint(ncam_range[0], ncam_range[1] + 1, (n_scenes,), generator=gen).tolist()
    res = torch.randint(0, 2, (n_scenes,), generator=gen).tolist()
    anchors = torch.randint(a_range[0], a_range[1] + 1, (n_scenes,), generator=gen).tolist()
    scenes = []
    for i in range(n_scenes):
        maps = MAPS_1080P if res[i] else MAPS_720P
        p = make_problem(gen, B=1, cam_maps=[maps] * ncams[i], C=256, G=8, A=anchors[i], P=13,
                         feat_scale=0.5, loc_range=(0.0, 1.0), out_frac=0.4,
                         feat_dtype=feat_dtype, w_dtype=w_dtype, with_grad=with_grad,
                         name=f"scene{i}")
        p.meta.update(resolution="1080p" if res[i] else "720p")
        scenes.append(p)
    return scenes
