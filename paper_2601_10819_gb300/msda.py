"""ctypes binding of libmsda_gb300 (include/msda.h) and a torch.autograd.Function.

Argument marshalling only: tensors are checked for device, dtype, layout and
shape, their device pointers and the current CUDA stream are passed to the
C-ABI, and every step of the computation runs in the library's kernels.
There is no fallback: if the library is missing or a call fails, a
``RuntimeError`` is raised.

The operator (arXiv 2601.10819, Sec. 3.2 and Sec. 5.3): for each anchor,
keypoint, camera and scale, sample the camera's map bilinearly at the
projected location (zero padding), weight by the group's attention weight
and sum into one C-channel feature per anchor.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass
from typing import List, Optional, Sequence

import torch

from . import build as _build

F32, BF16, F16 = 0, 1, 2
_DT = {torch.float32: F32, torch.bfloat16: BF16, torch.float16: F16}
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "UNSUPPORTED", 3: "CUDA", 4: "TIMEOUT", 5: "OUT_OF_RANGE",
          6: "WORKSPACE"}

_lock = threading.Lock()
_lib = None


class MSDAError(RuntimeError):
    def __init__(self, fn, code, msg):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)}: {msg}")
        self.code = code


class msda_tuning(ctypes.Structure):
    _fields_ = [("warps_per_block", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("variant", ctypes.c_int), ("vectors_per_lane", ctypes.c_int), ("flags", ctypes.c_int),
                ("reserved", ctypes.c_int * 3)]


FLAG_GRAD_FEAT_ZEROED = 1


class msda_scene(ctypes.Structure):
    _fields_ = [("feat", ctypes.c_void_p), ("spatial_shape", ctypes.c_void_p),
                ("scale_start_index", ctypes.c_void_p), ("sampling_location", ctypes.c_void_p),
                ("weights", ctypes.c_void_p), ("out", ctypes.c_void_p), ("sum_hw", ctypes.c_int32),
                ("Ncam", ctypes.c_int32), ("A", ctypes.c_int32), ("unit_begin", ctypes.c_int32)]


def library_path() -> str:
    return _build.LIB


def load(path: Optional[str] = None):
    """Load the shared library (no build).  Raises if it is missing."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or _build.LIB
        if not os.path.exists(p):
            raise RuntimeError(f"libmsda_gb300.so not found at {p}: run paper_2601_10819_gb300.build.build()")
        lib = ctypes.CDLL(p)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        tp = ctypes.POINTER(msda_tuning)
        lib.msda_forward_workspace_size.argtypes = [i] * 8
        lib.msda_forward_workspace_size.restype = sz
        lib.msda_forward.argtypes = [vp, i, vp, vp, vp, vp, i, vp, i] + [i] * 8 + [vp, sz, tp, vp]
        lib.msda_forward.restype = i
        lib.msda_forward_oae.argtypes = [vp, i, vp, vp, vp, vp, i, vp, vp, i] + [i] * 8 + [tp, vp]
        lib.msda_forward_oae.restype = i
        lib.msda_forward_train.argtypes = [vp, i, vp, vp, vp, vp, i, vp, i, vp] + [i] * 8 + [tp, vp]
        lib.msda_forward_train.restype = i
        lib.msda_keypoints.argtypes = [vp] * 6 + [i] * 4 + [vp]
        lib.msda_keypoints.restype = i
        lib.msda_backward_workspace_size.argtypes = [i] * 9
        lib.msda_backward_workspace_size.restype = sz
        lib.msda_backward.argtypes = [vp, i, vp, vp, vp, vp, i, vp, vp, vp, vp] + [i] * 8 + [i, vp, sz, tp, vp]
        lib.msda_backward.restype = i
        lib.msda_forward_batched_workspace_size.argtypes = [i]
        lib.msda_forward_batched_workspace_size.restype = sz
        lib.msda_forward_batched.argtypes = [vp, i, i, i, i, i, i, i, i, i, i, vp, sz, vp, tp, vp]
        lib.msda_forward_batched.restype = i
        lib.msda_get_device_status.argtypes = [vp]
        lib.msda_get_device_status.restype = i
        lib.msda_last_error.argtypes = []
        lib.msda_last_error.restype = ctypes.c_char_p
        lib.msda_version.argtypes = []
        lib.msda_version.restype = ctypes.c_char_p
        lib.msda_probe_read.argtypes = [vp, sz, i, i, i, vp, vp]
        lib.msda_probe_read.restype = i
        lib.msda_probe_reduce.argtypes = [vp, sz, i, i, i, vp]
        lib.msda_probe_reduce.restype = i
        lib.msda_debug_set_wait_limit.argtypes = [ctypes.c_longlong]
        lib.msda_debug_set_wait_limit.restype = i
        if path is None:
            _lib = lib
        return lib


def _check(fn: str, rc: int):
    if rc != 0:
        raise MSDAError(fn, rc, _lib.msda_last_error().decode())


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _tuning(warps: Optional[int], blocks_per_sm: Optional[int] = None, variant: int = 0, vec: int = 0,
            flags: int = 0):
    if not warps and not blocks_per_sm and not variant and not vec and not flags:
        return None
    t = msda_tuning()
    t.warps_per_block = int(warps or 0)
    t.blocks_per_sm = int(blocks_per_sm or 0)
    t.variant = int(variant)
    t.vectors_per_lane = int(vec or 0)
    t.flags = int(flags)
    return ctypes.byref(t)


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _dims(feat, spatial_shape, scale_start_index, sampling_location, weights):
    for name, t in (("feat", feat), ("spatial_shape", spatial_shape), ("scale_start_index", scale_start_index),
                    ("sampling_location", sampling_location), ("weights", weights)):
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    if spatial_shape.dtype != torch.int32 or scale_start_index.dtype != torch.int32:
        raise ValueError("spatial_shape and scale_start_index must be int32")
    if sampling_location.dtype != torch.float32:
        raise ValueError("sampling_location must be float32")
    if feat.dtype not in _DT or weights.dtype not in _DT:
        raise ValueError("feat/weights must be float32, bfloat16 or float16")
    B, sum_hw, C = feat.shape
    Ncam, Nscale, two = spatial_shape.shape
    if two != 2 or tuple(scale_start_index.shape) != (Ncam, Nscale):
        raise ValueError("spatial_shape must be [Ncam, Nscale, 2] and scale_start_index [Ncam, Nscale]")
    B2, A, P, Ncam2, two = sampling_location.shape
    if B2 != B or Ncam2 != Ncam or two != 2:
        raise ValueError("sampling_location must be [B, A, P, Ncam, 2]")
    if weights.dim() != 6 or tuple(weights.shape[:5]) != (B, A, P, Ncam, Nscale):
        raise ValueError("weights must be [B, A, P, Ncam, Nscale, G]")
    G = weights.shape[5]
    return B, sum_hw, C, Ncam, Nscale, A, P, G


def forward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G) -> int:
    return int(load().msda_forward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G))


AUTO = "auto"


def forward(feat, spatial_shape, scale_start_index, sampling_location, weights, *,
            out: Optional[torch.Tensor] = None, out_dtype: torch.dtype = torch.float32,
            workspace=None, warps: Optional[int] = None, variant: int = 0, vec: int = 0) -> torch.Tensor:
    """msda_forward: out[B, A, C] on the current stream of feat's device.

    workspace: None (default: the anchor-per-block kernel, no scratch, the
    faster form on the measured workloads), "auto" (a buffer from torch's
    allocator, which selects the staged camera-group kernels) or a uint8
    CUDA tensor (likewise).
    """
    lib = load()
    B, sum_hw, C, Ncam, Nscale, A, P, G = _dims(feat, spatial_shape, scale_start_index, sampling_location, weights)
    if out is None:
        out = torch.empty(B, A, C, dtype=out_dtype, device=feat.device)
    elif out.shape != (B, A, C) or not out.is_contiguous() or out.dtype not in _DT:
        raise ValueError("out must be a contiguous [B, A, C] tensor")
    if isinstance(workspace, str):
        need = forward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G)
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=feat.device)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = lib.msda_forward(_ptr(feat), _DT[feat.dtype], _ptr(spatial_shape), _ptr(scale_start_index),
                          _ptr(sampling_location), _ptr(weights), _DT[weights.dtype], _ptr(out), _DT[out.dtype],
                          B, sum_hw, C, Ncam, Nscale, A, P, G, _ptr(workspace), ws_bytes, _tuning(warps, None, variant, vec),
                          ctypes.c_void_p(_stream(feat.device)))
    _check("msda_forward", rc)
    return out


def forward_train(feat, spatial_shape, scale_start_index, sampling_location, weights, grad_feat, *,
                  out: Optional[torch.Tensor] = None, out_dtype: torch.dtype = torch.float32,
                  warps: Optional[int] = None, variant: int = 0, vec: int = 0) -> torch.Tensor:
    """msda_forward_train: the forward, also clearing grad_feat (float32 [B, sum_hw, C]) for a following
    backward(..., grads=(grad_feat, ...), grad_feat_zeroed=True)."""
    lib = load()
    B, sum_hw, C, Ncam, Nscale, A, P, G = _dims(feat, spatial_shape, scale_start_index, sampling_location, weights)
    if grad_feat.dtype != torch.float32 or not grad_feat.is_cuda or not grad_feat.is_contiguous() or \
            tuple(grad_feat.shape) != (B, sum_hw, C):
        raise ValueError("grad_feat must be a contiguous float32 CUDA tensor [B, sum_hw, C]")
    if out is None:
        out = torch.empty(B, A, C, dtype=out_dtype, device=feat.device)
    elif out.shape != (B, A, C) or not out.is_contiguous() or out.dtype not in _DT:
        raise ValueError("out must be a contiguous [B, A, C] tensor")
    rc = lib.msda_forward_train(_ptr(feat), _DT[feat.dtype], _ptr(spatial_shape), _ptr(scale_start_index),
                                _ptr(sampling_location), _ptr(weights), _DT[weights.dtype], _ptr(out), _DT[out.dtype],
                                _ptr(grad_feat), B, sum_hw, C, Ncam, Nscale, A, P, G,
                                _tuning(warps, None, variant, vec), ctypes.c_void_p(_stream(feat.device)))
    _check("msda_forward_train", rc)
    return out


def forward_oae(feat, spatial_shape, scale_start_index, sampling_location, weights, visibility, *,
                out: Optional[torch.Tensor] = None, out_dtype: torch.dtype = torch.float32,
                warps: Optional[int] = None, vec: int = 0, variant: int = 0) -> torch.Tensor:
    """msda_forward_oae: the operator fused with the visibility-weighted mean over cameras."""
    lib = load()
    B, sum_hw, C, Ncam, Nscale, A, P, G = _dims(feat, spatial_shape, scale_start_index, sampling_location, weights)
    if visibility.dtype != torch.float32 or not visibility.is_cuda or not visibility.is_contiguous() or \
            tuple(visibility.shape) != (B, A, Ncam):
        raise ValueError("visibility must be a contiguous float32 CUDA tensor [B, A, Ncam]")
    if out is None:
        out = torch.empty(B, A, C, dtype=out_dtype, device=feat.device)
    rc = lib.msda_forward_oae(_ptr(feat), _DT[feat.dtype], _ptr(spatial_shape), _ptr(scale_start_index),
                              _ptr(sampling_location), _ptr(weights), _DT[weights.dtype], _ptr(visibility),
                              _ptr(out), _DT[out.dtype], B, sum_hw, C, Ncam, Nscale, A, P, G,
                              _tuning(warps, None, variant, vec), ctypes.c_void_p(_stream(feat.device)))
    _check("msda_forward_oae", rc)
    return out


def keypoints(anchors, offsets, dt, proj, img_wh, *, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """msda_keypoints: sampling_location [B, A, P, Ncam, 2] from anchors and cameras."""
    lib = load()
    for name, t in (("anchors", anchors), ("offsets", offsets), ("dt", dt), ("proj", proj), ("img_wh", img_wh)):
        if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    B, A, _ = anchors.shape
    P = offsets.shape[2]
    Ncam = proj.shape[1]
    if anchors.shape[2] != 11 or tuple(offsets.shape) != (B, A, P, 3) or tuple(dt.shape) != (B,) or \
            tuple(proj.shape) != (B, Ncam, 3, 4) or tuple(img_wh.shape) != (Ncam, 2):
        raise ValueError("bad keypoint prologue shapes")
    if out is None:
        out = torch.empty(B, A, P, Ncam, 2, dtype=torch.float32, device=anchors.device)
    rc = lib.msda_keypoints(_ptr(anchors), _ptr(offsets), _ptr(dt), _ptr(proj), _ptr(img_wh), _ptr(out),
                            B, A, P, Ncam, ctypes.c_void_p(_stream(anchors.device)))
    _check("msda_keypoints", rc)
    return out


def backward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G, deterministic: bool) -> int:
    return int(load().msda_backward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G, int(bool(deterministic))))


def backward(feat, spatial_shape, scale_start_index, sampling_location, weights, grad_out, *,
             deterministic: bool = False, workspace: Optional[torch.Tensor] = None,
             grads=None, warps: Optional[int] = None, variant: int = 0, vec: int = 0,
             grad_feat_zeroed: bool = False, flags: int = 0):
    """msda_backward: (grad_feat, grad_loc, grad_weights), all float32.

    grad_feat_zeroed: the caller already cleared grads[0] (atomic mode only).
    workspace: allocated when None (or, in deterministic mode, too small).  In
    atomic mode a caller's workspace is passed through as is: one of fewer
    than 8 bytes selects the static-stride item order.
    flags: extra MSDA_FLAG_* bits.
    """
    lib = load()
    B, sum_hw, C, Ncam, Nscale, A, P, G = _dims(feat, spatial_shape, scale_start_index, sampling_location, weights)
    if grad_out.dtype != torch.float32 or not grad_out.is_contiguous() or tuple(grad_out.shape) != (B, A, C):
        raise ValueError("grad_out must be a contiguous float32 [B, A, C] tensor")
    dev = feat.device
    if grads is None:
        gf = torch.empty(B, sum_hw, C, dtype=torch.float32, device=dev)
        gl = torch.empty(B, A, P, Ncam, 2, dtype=torch.float32, device=dev)
        gw = torch.empty(B, A, P, Ncam, Nscale, G, dtype=torch.float32, device=dev)
    else:
        gf, gl, gw = grads
    need = backward_workspace_size(B, sum_hw, C, Ncam, Nscale, A, P, G, deterministic)
    small = workspace is not None and workspace.numel() * workspace.element_size() < need
    if need and (workspace is None or (small and deterministic)):
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    rc = lib.msda_backward(_ptr(feat), _DT[feat.dtype], _ptr(spatial_shape), _ptr(scale_start_index),
                           _ptr(sampling_location), _ptr(weights), _DT[weights.dtype], _ptr(grad_out),
                           _ptr(gf), _ptr(gl), _ptr(gw), B, sum_hw, C, Ncam, Nscale, A, P, G,
                           int(bool(deterministic)), _ptr(workspace), ws_bytes,
                           _tuning(warps, None, variant, vec,
                                   (FLAG_GRAD_FEAT_ZEROED if grad_feat_zeroed else 0) | int(flags)),
                           ctypes.c_void_p(_stream(dev)))
    _check("msda_backward", rc)
    return gf, gl, gw


def debug_set_wait_limit(polls: int):
    """msda_debug_set_wait_limit: poll limit of the staged kernels' first wait (0: give up at once; < 0:
    the default).  A testing aid."""
    _check("msda_debug_set_wait_limit", load().msda_debug_set_wait_limit(int(polls)))


def device_status(stream=None) -> int:
    """Synchronise and read-and-clear the library's device status word."""
    lib = load()
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    return int(lib.msda_get_device_status(ctypes.c_void_p(s)))


def version() -> str:
    return load().msda_version().decode()


def probe_read(buf: torch.Tensor, reps: int, blocks: int, rows: int = 0, sink: Optional[torch.Tensor] = None):
    lib = load()
    if sink is None:
        sink = torch.zeros(blocks, dtype=torch.int32, device=buf.device)
    rc = lib.msda_probe_read(_ptr(buf), buf.numel() * buf.element_size(), reps, blocks, rows, _ptr(sink),
                             ctypes.c_void_p(_stream(buf.device)))
    _check("msda_probe_read", rc)
    return sink


def probe_reduce(buf: torch.Tensor, reps: int, blocks: int, rows: int):
    """msda_probe_reduce on a float32 CUDA buffer (its contents change)."""
    lib = load()
    if buf.dtype != torch.float32 or not buf.is_contiguous():
        raise ValueError("probe_reduce needs a contiguous float32 buffer")
    rc = lib.msda_probe_reduce(_ptr(buf), buf.numel() * 4, reps, blocks, rows, ctypes.c_void_p(_stream(buf.device)))
    _check("msda_probe_reduce", rc)


# ---------------------------------------------------------------------------
# Batched serving
# ---------------------------------------------------------------------------
@dataclass
class BatchedPlan:
    """Device-side descriptors and scratch for msda_forward_batched.

    Build once per set of scene tensors; ``run()`` enqueues the single
    persistent launch and can be captured in a CUDA graph.
    """
    scenes_dev: torch.Tensor
    workspace: torch.Tensor
    done_ns: torch.Tensor
    outs: List[torch.Tensor]
    num_scenes: int
    total: int
    max_ncam: int
    Nscale: int
    C: int
    P: int
    G: int
    ft: int
    wt: int
    ot: int
    warps: Optional[int] = None
    blocks_per_sm: Optional[int] = None
    vec: int = 0
    _keep: tuple = ()

    def run(self):
        lib = load()
        dev = self.scenes_dev.device
        rc = lib.msda_forward_batched(_ptr(self.scenes_dev), self.num_scenes, self.total, self.max_ncam,
                                      self.Nscale, self.C, self.P, self.G, self.ft, self.wt, self.ot,
                                      _ptr(self.workspace), self.workspace.numel(), _ptr(self.done_ns),
                                      _tuning(self.warps, self.blocks_per_sm, 0, self.vec),
                                      ctypes.c_void_p(_stream(dev)))
        _check("msda_forward_batched", rc)
        return self.outs


def plan_batched(scenes: Sequence, out_dtype: torch.dtype = torch.float32, warps: Optional[int] = None,
                 blocks_per_sm: Optional[int] = None, vec: int = 0) -> BatchedPlan:
    """scenes: objects with feat [1,sum_hw,C], spatial_shape, scale_start_index,
    sampling_location [1,A,P,Ncam,2], weights [1,A,P,Ncam,Nscale,G] CUDA tensors."""
    load()
    if not scenes:
        raise ValueError("no scenes")
    arr = (msda_scene * len(scenes))()
    outs, unit = [], 0
    dims0 = None
    max_ncam = 0
    for i, s in enumerate(scenes):
        B, sum_hw, C, Ncam, Nscale, A, P, G = _dims(s.feat, s.spatial_shape, s.scale_start_index,
                                                    s.sampling_location, s.weights)
        if B != 1:
            raise ValueError("batched scenes must have B == 1")
        d = (C, Nscale, P, G, s.feat.dtype, s.weights.dtype)
        if dims0 is None:
            dims0 = d
        elif d != dims0:
            raise ValueError("all scenes must share C, Nscale, P, G and dtypes")
        out = torch.empty(A, C, dtype=out_dtype, device=s.feat.device)
        outs.append(out)
        arr[i] = msda_scene(s.feat.data_ptr(), s.spatial_shape.data_ptr(), s.scale_start_index.data_ptr(),
                            s.sampling_location.data_ptr(), s.weights.data_ptr(), out.data_ptr(),
                            sum_hw, Ncam, A, unit)
        unit += A
        max_ncam = max(max_ncam, Ncam)
    dev = scenes[0].feat.device
    raw = torch.frombuffer(bytearray(bytes(arr)), dtype=torch.uint8)
    scenes_dev = raw.to(dev)
    ws = torch.zeros(int(load().msda_forward_batched_workspace_size(len(scenes))), dtype=torch.uint8, device=dev)
    done = torch.zeros(len(scenes) + 1, dtype=torch.int64, device=dev)
    C, Nscale, P, G, fdt, wdt = dims0
    keep = tuple(t for s in scenes for t in (s.feat, s.spatial_shape, s.scale_start_index,
                                             s.sampling_location, s.weights))
    return BatchedPlan(scenes_dev, ws, done, outs, len(scenes), unit, max_ncam, Nscale, C, P, G,
                       _DT[fdt], _DT[wdt], _DT[out_dtype], warps, blocks_per_sm, vec, keep)


# ---------------------------------------------------------------------------
# Autograd
# ---------------------------------------------------------------------------
class MSDAFunction(torch.autograd.Function):
    """Differentiable MSDA: gradients for feat, sampling_location and weights.

    The forward output is float32; the gradients are float32 and are cast to
    the input dtypes when those are reduced precision.  The backward is the
    deterministic mode unless deterministic=False (the atomic mode).
    """

    @staticmethod
    def forward(ctx, feat, spatial_shape, scale_start_index, sampling_location, weights,
                deterministic: bool = True):
        ctx.save_for_backward(feat, spatial_shape, scale_start_index, sampling_location, weights)
        ctx.deterministic = bool(deterministic)
        return forward(feat, spatial_shape, scale_start_index, sampling_location, weights)

    @staticmethod
    def backward(ctx, grad_out):
        feat, shape, start, loc, w = ctx.saved_tensors
        gf, gl, gw = backward(feat, shape, start, loc, w, grad_out.contiguous().float(),
                              deterministic=ctx.deterministic)
        return (gf.to(feat.dtype) if ctx.needs_input_grad[0] else None, None, None,
                gl if ctx.needs_input_grad[3] else None,
                gw.to(w.dtype) if ctx.needs_input_grad[4] else None, None)


def msda(feat, spatial_shape, scale_start_index, sampling_location, weights, deterministic: bool = True):
    """Differentiable entry point (see MSDAFunction)."""
    return MSDAFunction.apply(feat, spatial_shape, scale_start_index, sampling_location, weights, deterministic)
