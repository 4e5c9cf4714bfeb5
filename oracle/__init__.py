"""FP64 CPU oracle for Multi-Scale Deformable Aggregation (MSDA).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py`` may import this package.  The product
path (``paper_2601_10819_gb300``) never imports it and shares no code with
it; the CUDA library refuses to fall back to it.

The arithmetic lives in ``msda_oracle.c`` (plain C loops in double
precision, following Sec. 3.1, Sec. 3.2 and Sec. 5.3 of the paper; the
readings of the paper taken there are listed in that file's header).  This
module compiles it with gcc and wraps it with ctypes.  All array arguments
are numpy arrays; floating-point inputs are widened to float64 (a BF16 or
FP16 input is widened exactly, so the oracle sees the rounded values the GPU
sees).

Pins: ``tests/test_oracle_pins.py`` checks this oracle against closed forms
(constant map, pixel centres, linear map, out-of-range points), a
tent-kernel brute force, torch's float64 ``grid_sample``, central finite
differences, the adjoint identity and a hand-computed golden fixture, and
``tests/test_oracle_mutants.py`` shows that planted mistakes fail them.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msda_oracle.c")
_BUILD_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD_DIR, "libmsda_oracle.so")
_lock = threading.Lock()
_lib = None


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH, openmp: bool = True) -> str:
    """Compile ``src`` into a shared library at ``out`` with gcc; returns ``out``."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    cmd = ["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", out, src, "-lm"]
    if openmp:
        cmd.insert(1, "-fopenmp")
    try:
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    except subprocess.CalledProcessError:
        if not openmp:
            raise
        cmd.remove("-fopenmp")
        subprocess.run(cmd, check=True, capture_output=True, text=True)
    return out


def build() -> str:
    """Compile the oracle if the library is missing or older than its source."""
    if not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        compile_oracle()
    return _LIB_PATH


def load_library(path: str):
    """Load an oracle shared library and declare its signatures."""
    lib = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int32)
    i = ctypes.c_int
    lib.msda_oracle_forward.argtypes = [dp, ip, ip, dp, dp, dp] + [i] * 9
    lib.msda_oracle_forward.restype = i
    lib.msda_oracle_backward.argtypes = [dp, ip, ip, dp, dp, dp, dp, dp, dp] + [i] * 8
    lib.msda_oracle_backward.restype = i
    lib.msda_oracle_forward_oae.argtypes = [dp, ip, ip, dp, dp, dp, dp] + [i] * 8
    lib.msda_oracle_forward_oae.restype = i
    lib.msda_oracle_keypoints.argtypes = [dp, dp, dp, dp, dp, dp] + [i] * 4
    lib.msda_oracle_keypoints.restype = i
    lib.msda_oracle_max_threads.argtypes = []
    lib.msda_oracle_max_threads.restype = i
    return lib


def _get_lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
    return _lib


def _f64(x) -> np.ndarray:
    if hasattr(x, "detach"):  # torch tensor: widen exactly through float64
        x = x.detach().to("cpu").double().numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.float64))


def _i32(x) -> np.ndarray:
    if hasattr(x, "detach"):
        x = x.detach().to("cpu").numpy()
    return np.ascontiguousarray(np.asarray(x, dtype=np.int32))


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _dims(feat, shape, loc, w, G):
    B, sum_hw, C = feat.shape
    Ncam, Nscale, _ = shape.shape
    B2, A, P, Ncam2, two = loc.shape
    if B2 != B or Ncam2 != Ncam or two != 2:
        raise ValueError("sampling_location must be [B, A, P, Ncam, 2]")
    if w.shape != (B, A, P, Ncam, Nscale, G):
        raise ValueError("weights must be [B, A, P, Ncam, Nscale, G]")
    return B, sum_hw, C, Ncam, Nscale, A, P


def forward(feat, spatial_shape, scale_start_index, sampling_location, weights,
            nthreads: int = 1, lib=None) -> np.ndarray:
    """out[B, A, C] (float64) of the operator; see ``msda_oracle.c``."""
    lib = lib or _get_lib()
    feat, loc, w = _f64(feat), _f64(sampling_location), _f64(weights)
    shape, start = _i32(spatial_shape), _i32(scale_start_index)
    G = w.shape[-1]
    B, sum_hw, C, Ncam, Nscale, A, P = _dims(feat, shape, loc, w, G)
    out = np.zeros((B, A, C), dtype=np.float64)
    rc = lib.msda_oracle_forward(
        _ptr(feat, ctypes.c_double), _ptr(shape, ctypes.c_int32), _ptr(start, ctypes.c_int32),
        _ptr(loc, ctypes.c_double), _ptr(w, ctypes.c_double), _ptr(out, ctypes.c_double),
        B, sum_hw, C, Ncam, Nscale, A, P, G, int(nthreads))
    if rc != 0:
        raise ValueError("oracle forward rejected its arguments")
    return out


def backward(feat, spatial_shape, scale_start_index, sampling_location, weights, grad_out,
             lib=None):
    """(grad_feat, grad_loc, grad_w) in float64; see ``msda_oracle.c``."""
    lib = lib or _get_lib()
    feat, loc, w = _f64(feat), _f64(sampling_location), _f64(weights)
    go = _f64(grad_out)
    shape, start = _i32(spatial_shape), _i32(scale_start_index)
    G = w.shape[-1]
    B, sum_hw, C, Ncam, Nscale, A, P = _dims(feat, shape, loc, w, G)
    if go.shape != (B, A, C):
        raise ValueError("grad_out must be [B, A, C]")
    gf = np.empty_like(feat)
    gl = np.empty_like(loc)
    gw = np.empty_like(w)
    rc = lib.msda_oracle_backward(
        _ptr(feat, ctypes.c_double), _ptr(shape, ctypes.c_int32), _ptr(start, ctypes.c_int32),
        _ptr(loc, ctypes.c_double), _ptr(w, ctypes.c_double), _ptr(go, ctypes.c_double),
        _ptr(gf, ctypes.c_double), _ptr(gl, ctypes.c_double), _ptr(gw, ctypes.c_double),
        B, sum_hw, C, Ncam, Nscale, A, P, G)
    if rc != 0:
        raise ValueError("oracle backward rejected its arguments")
    return gf, gl, gw


def forward_oae(feat, spatial_shape, scale_start_index, sampling_location, weights, visibility,
                lib=None) -> np.ndarray:
    """Visibility-weighted fusion over cameras (Sec. 3.2, Eq. 2); see msda_oracle.c."""
    lib = lib or _get_lib()
    feat, loc, w = _f64(feat), _f64(sampling_location), _f64(weights)
    vis = _f64(visibility)
    shape, start = _i32(spatial_shape), _i32(scale_start_index)
    G = w.shape[-1]
    B, sum_hw, C, Ncam, Nscale, A, P = _dims(feat, shape, loc, w, G)
    if vis.shape != (B, A, Ncam):
        raise ValueError("visibility must be [B, A, Ncam]")
    out = np.zeros((B, A, C), dtype=np.float64)
    rc = lib.msda_oracle_forward_oae(
        _ptr(feat, ctypes.c_double), _ptr(shape, ctypes.c_int32), _ptr(start, ctypes.c_int32),
        _ptr(loc, ctypes.c_double), _ptr(w, ctypes.c_double), _ptr(vis, ctypes.c_double),
        _ptr(out, ctypes.c_double), B, sum_hw, C, Ncam, Nscale, A, P, G)
    if rc != 0:
        raise ValueError("oracle forward_oae rejected its arguments")
    return out


def keypoints(anchors, offsets, dt, proj, img_wh, lib=None) -> np.ndarray:
    """Sampling locations [B, A, P, Ncam, 2] of the keypoint prologue; see msda_oracle.c."""
    lib = lib or _get_lib()
    an, of, dtt, pr, wh = _f64(anchors), _f64(offsets), _f64(dt), _f64(proj), _f64(img_wh)
    B, A, _ = an.shape
    P = of.shape[2]
    Ncam = pr.shape[1]
    if an.shape[2] != 11 or of.shape != (B, A, P, 3) or dtt.shape != (B,) or pr.shape != (B, Ncam, 3, 4) \
            or wh.shape != (Ncam, 2):
        raise ValueError("bad keypoint prologue shapes")
    loc = np.zeros((B, A, P, Ncam, 2), dtype=np.float64)
    rc = lib.msda_oracle_keypoints(_ptr(an, ctypes.c_double), _ptr(of, ctypes.c_double), _ptr(dtt, ctypes.c_double),
                                   _ptr(pr, ctypes.c_double), _ptr(wh, ctypes.c_double), _ptr(loc, ctypes.c_double),
                                   B, A, P, Ncam)
    if rc != 0:
        raise ValueError("oracle keypoints rejected its arguments")
    return loc


def max_threads(lib=None) -> int:
    """OpenMP threads the forward can use on this host (1 if built without OpenMP)."""
    return int((lib or _get_lib()).msda_oracle_max_threads())
