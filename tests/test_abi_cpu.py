"""The C-ABI library builds, loads and exports what include/msda.h declares.

Runs without a GPU: only host-side argument validation is exercised (it
returns before any CUDA call), plus the workspace-size queries.
"""
import ctypes
import os
import re

import pytest
import torch

from paper_2601_10819_gb300 import build as msda_build
from paper_2601_10819_gb300 import msda

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "msda.h")


@pytest.fixture(scope="module")
def lib():
    msda_build.build()
    return msda.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(msda_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["msda_forward", "msda_backward", "msda_backward_workspace_size", "msda_forward_batched",
              "msda_forward_batched_workspace_size", "msda_get_device_status", "msda_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert "sm_103a" in msda.version()


def test_abi_struct_layouts_match_header():
    # msda_tuning: 8 ints; msda_scene: 6 pointers + 4 int32
    assert ctypes.sizeof(msda.msda_tuning) == 32
    assert ctypes.sizeof(msda.msda_scene) == 6 * 8 + 4 * 4


def _fwd(lib, **kw):
    args = dict(feat=16, ft=msda.F32, shape=16, start=16, loc=16, w=16, wt=msda.F32, out=16, ot=msda.F32,
                B=1, sum_hw=64, C=32, Ncam=1, Nscale=1, A=2, P=1, G=4)
    args.update(kw)
    vp = ctypes.c_void_p
    return lib.msda_forward(vp(args["feat"]), args["ft"], vp(args["shape"]), vp(args["start"]), vp(args["loc"]),
                            vp(args["w"]), args["wt"], vp(args["out"]), args["ot"], args["B"], args["sum_hw"],
                            args["C"], args["Ncam"], args["Nscale"], args["A"], args["P"], args["G"], None, 0,
                            None, None)


@pytest.mark.parametrize("kw,code", [
    (dict(C=30, G=4), 1),              # C % G != 0
    (dict(G=0), 1),
    (dict(A=-1), 1),
    (dict(feat=0), 1),                 # NULL feat
    (dict(out=0), 1),                  # NULL out
    (dict(loc=0), 1),
    (dict(ft=7), 1),                   # unknown dtype
    (dict(C=8, G=4), 2),               # (C/G)*4 = 8 bytes: not a multiple of 16
    (dict(feat=24), 2),                # misaligned pointer
    (dict(Nscale=17), 2),
    (dict(C=4096, G=1), 2),            # no lane split (row wider than one warp of 64-byte lanes)
])
def test_forward_validation(lib, kw, code):
    rc = _fwd(lib, **kw)
    assert rc == code, lib.msda_last_error()
    assert lib.msda_last_error().decode()


def test_backward_validation(lib):
    vp = ctypes.c_void_p
    rc = lib.msda_backward(vp(16), msda.F32, vp(16), vp(16), vp(16), vp(16), msda.F32, vp(0), vp(16), vp(16),
                           vp(16), 1, 64, 32, 1, 1, 2, 1, 4, 0, None, 0, None, None)
    assert rc == 1  # NULL grad_out
    rc = lib.msda_backward(vp(16), msda.F32, vp(16), vp(16), vp(16), vp(16), msda.F32, vp(16), vp(16), vp(16),
                           vp(20), 1, 64, 32, 1, 1, 2, 1, 4, 0, None, 0, None, None)
    assert rc == 2  # misaligned grad_weights


def test_batched_validation(lib):
    vp = ctypes.c_void_p
    rc = lib.msda_forward_batched(vp(0), 2, 10, 4, 4, 256, 13, 8, 1, 1, 0, vp(16), 64, None, None, None)
    assert rc == 1  # NULL scenes
    rc = lib.msda_forward_batched(vp(16), 1, 10, 4, 4, 250, 13, 8, 1, 1, 0, vp(16), 64, None, None, None)
    assert rc == 1  # C % G


def test_workspace_sizes(lib):
    assert lib.msda_forward_workspace_size(2, 100, 32, 3, 2, 5, 4, 4) >= 2 * 3 * 5 * 32 * 4
    assert lib.msda_backward_workspace_size(1, 100, 32, 2, 2, 4, 3, 4, 0) == 256  # atomic mode: work counter
    n = 1 * 4 * 3 * 2 * 2
    ws = lib.msda_backward_workspace_size(1, 100, 32, 2, 2, 4, 3, 4, 1)
    assert ws >= 4 * 4 * n * 4 + 4 * 101  # slot ids, three flat arrays per contribution, row offsets
    assert lib.msda_forward_batched_workspace_size(16) >= 17 * 4


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_valid_call_without_gpu_fails_loudly(lib):
    rc = _fwd(lib)
    assert rc == 3  # MSDA_ERR_CUDA, never a silent CPU fallback
    assert lib.msda_last_error().decode()
