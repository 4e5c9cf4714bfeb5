"""The allocation-free batched forward, msda_forward_batched_noalloc.

Callers that cannot allocate device memory at the point where they launch
work (an inference engine plugin's enqueue, a real-time loop with a fixed
memory budget, a C host program with no device allocator) call this entry
point: its scratch counters live in a device array built into the library.
This file is collected last, so a failure here leaves every other test run.
"""
import ctypes

import pytest
import torch

from gpu_util import TOL_LOWP_OUT, ensure_lib, relerr
from paper_2601_10819_gb300 import inputs, msda


def _declare(lib):
    vp, i = ctypes.c_void_p, ctypes.c_int
    lib.msda_forward_batched_noalloc.argtypes = [vp, i, i, i, i, i, i, i, i, i, i, vp,
                                                 ctypes.POINTER(msda.msda_tuning), vp]
    lib.msda_forward_batched_noalloc.restype = i
    lib.msda_forward_batched_noalloc_max_scenes.argtypes = []
    lib.msda_forward_batched_noalloc_max_scenes.restype = i
    return lib


def _call_noalloc(lib, plan, stream):
    return lib.msda_forward_batched_noalloc(
        ctypes.c_void_p(plan.scenes_dev.data_ptr()), plan.num_scenes, plan.total, plan.max_ncam, plan.Nscale,
        plan.C, plan.P, plan.G, plan.ft, plan.wt, plan.ot, ctypes.c_void_p(plan.done_ns.data_ptr()), None,
        ctypes.c_void_p(stream))


def test_noalloc_rejects_more_scenes_than_its_scratch_holds():
    lib = _declare(ensure_lib())
    limit = lib.msda_forward_batched_noalloc_max_scenes()
    assert limit >= 16
    rc = lib.msda_forward_batched_noalloc(ctypes.c_void_p(16), limit + 1, 10, 4, 4, 256, 13, 8, 1, 1, 0,
                                          None, None, None)
    assert rc == 1  # MSDA_ERR_INVALID_ARG
    assert "limit" in lib.msda_last_error().decode()


@pytest.mark.gpu
def test_noalloc_matches_workspace_entry_point_on_two_calls():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lib = _declare(ensure_lib())
    gen = torch.Generator().manual_seed(21)
    scenes = [s.to("cuda") for s in inputs.make_batched(gen, n_scenes=6, ncam_range=(1, 12), a_range=(1, 90))]
    plan = msda.plan_batched(scenes)
    ref = [o.clone() for o in plan.run()]          # existing entry point, caller workspace
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):                              # two calls in a row reuse the built-in scratch
        for o in plan.outs:
            o.fill_(float("nan"))
        plan.done_ns.zero_()
        assert _call_noalloc(lib, plan, stream) == 0, lib.msda_last_error().decode()
        torch.cuda.synchronize()
        for o, r in zip(plan.outs, ref):
            assert relerr(o.cpu().double().numpy(), r.cpu().double().numpy()) <= TOL_LOWP_OUT
        t = plan.done_ns.cpu()
        assert t[0] > 0 and torch.all(t[1:] >= t[0])
    assert msda.device_status() == 0


@pytest.mark.gpu
def test_noalloc_at_its_scene_limit_matches_workspace_entry_point():
    """Exactly the advertised number of scenes (tiny ones: 1 camera, 1 anchor each) must run."""
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    lib = _declare(ensure_lib())
    limit = lib.msda_forward_batched_noalloc_max_scenes()
    gen = torch.Generator().manual_seed(22)
    scenes = [inputs.make_problem(gen, B=1, cam_maps=[[(4, 6), (2, 3)]], C=32, G=4, A=1, P=2,
                                  loc_range=(-0.1, 1.1), with_grad=False).to("cuda") for _ in range(limit)]
    plan = msda.plan_batched(scenes)
    ref = [o.clone() for o in plan.run()]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream().cuda_stream
    for o in plan.outs:
        o.fill_(float("nan"))
    plan.done_ns.zero_()
    assert _call_noalloc(lib, plan, stream) == 0, lib.msda_last_error().decode()
    torch.cuda.synchronize()
    got = torch.stack(plan.outs).cpu().double()
    want = torch.stack(ref).cpu().double()
    assert torch.equal(got, want)  # same kernel, same launch: bitwise equal
    assert msda.device_status() == 0
