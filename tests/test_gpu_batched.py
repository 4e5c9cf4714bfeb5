"""Batched serving: one persistent launch over uneven scenes, CUDA-graph replay."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_LOWP_OUT, ensure_lib, oracle_forward, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


def small_scenes(n=5, seed=11):
    gen = torch.Generator().manual_seed(seed)
    return inputs.make_batched(gen, n_scenes=n, ncam_range=(1, 9), a_range=(1, 70), with_grad=False)


@pytest.mark.parametrize("warps,bps", [(8, None), (4, 2), (16, 1), (2, 8)])
def test_batched_equals_single_scene_calls(warps, bps):
    scenes = [s.to("cuda") for s in small_scenes()]
    plan = msda.plan_batched(scenes, warps=warps, blocks_per_sm=bps)
    outs = plan.run()
    torch.cuda.synchronize()
    for s, o in zip(scenes, outs):
        single = msda.forward(s.feat, s.spatial_shape, s.scale_start_index, s.sampling_location, s.weights,
                              warps=warps, workspace=None)
        assert torch.equal(o, single[0])  # same kernel body, same reduction order
    assert msda.device_status() == 0


def test_batched_against_oracle_and_timestamps():
    scenes_cpu = small_scenes(6, seed=12)
    scenes = [s.to("cuda") for s in scenes_cpu]
    plan = msda.plan_batched(scenes)
    outs = plan.run()
    torch.cuda.synchronize()
    for sc, o in zip(scenes_cpu, outs):
        assert relerr(o.cpu().double().numpy(), oracle_forward(sc)[0]) <= TOL_LOWP_OUT
    t = plan.done_ns.cpu()
    assert t[0] > 0 and torch.all(t[1:] >= t[0])


def test_cuda_graph_capture_and_replay():
    scenes = [s.to("cuda") for s in small_scenes(4, seed=13)]
    plan = msda.plan_batched(scenes)
    plan.run()  # first call outside capture (device set-up)
    torch.cuda.synchronize()
    ref = [o.clone() for o in plan.outs]
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        for o in plan.outs:
            o.zero_()
        with torch.cuda.graph(g, stream=s):
            plan.run()
    for _ in range(3):
        for o in plan.outs:
            o.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for o, r in zip(plan.outs, ref):
            assert torch.equal(o, r)


def test_full_serving_workload_matches_single_scene_calls():
    """The 16-scene, 4..96-camera, 720p/1080p workload."""
    scenes_cpu = inputs.make_workload(4, with_grad=False)
    scenes = [s.to("cuda") for s in scenes_cpu]
    plan = msda.plan_batched(scenes)
    outs = plan.run()
    torch.cuda.synchronize()
    for i, (s, o) in enumerate(zip(scenes, outs)):
        single = msda.forward(s.feat, s.spatial_shape, s.scale_start_index, s.sampling_location, s.weights,
                              workspace=None, warps=8)  # the batched default
        assert torch.equal(o, single[0]), i
    # oracle on sampled anchors of two scenes
    for i in (0, 7):
        idx = torch.arange(0, scenes_cpu[i].sampling_location.shape[1], 97)
        sub = scenes_cpu[i].anchors(idx)
        assert relerr(outs[i].cpu()[idx].double().numpy(), oracle_forward(sub)[0]) <= TOL_LOWP_OUT
    assert msda.device_status() == 0


def test_bad_descriptor_is_reported_not_faulted():
    scenes = [s.to("cuda") for s in small_scenes(3, seed=14)]
    plan = msda.plan_batched(scenes)
    plan.max_ncam = 0  # every scene has more cameras than the staged tables allow
    plan.run()
    torch.cuda.synchronize()
    assert msda.device_status() == 5


def test_full_serving_batch_in_its_launch_configuration_sampled():
    """The 16-scene serving batch of bench.py (762 cameras, 14 161 anchors) with the shipped GB300 mapping,
    checked against the oracle on 12 anchors per scene (first, last and spread between)."""
    import json
    from paper_2601_10819_gb300 import tune
    scenes_cpu = inputs.make_workload(4, with_grad=False)
    scenes = [s.to("cuda") for s in scenes_cpu]
    table = json.load(open(tune.SHIPPED))
    cfg = next((v["best"] for k, v in table.items() if "|batched|" in k), {})
    plan = msda.plan_batched(scenes, warps=cfg.get("warps") or None, blocks_per_sm=cfg.get("bps") or None,
                             vec=cfg.get("vec", 0))
    outs = plan.run()
    torch.cuda.synchronize()
    worst = 0.0
    for s, o in zip(scenes_cpu, outs):
        A = s.sampling_location.shape[1]
        idx = sorted(set(np.linspace(0, A - 1, 12).round().astype(int).tolist()))
        ref = oracle_forward(s.anchors(idx))
        got = o.cpu()[idx].double().numpy()[None]
        worst = max(worst, relerr(got, ref))
    print(f"full serving batch, sampled anchors: rel err {worst:.2e}")
    assert worst <= TOL_LOWP_OUT
    assert msda.device_status() == 0
