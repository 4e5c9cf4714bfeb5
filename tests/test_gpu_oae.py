"""Fused occlusion-aware fusion (Sec. 3.2, Eq. 2) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_FP32, TOL_LOWP_OUT, ensure_lib, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


def gpu_oae(pr, vis, **kw):
    d = pr.to("cuda")
    out = msda.forward_oae(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights,
                           vis.cuda(), **kw)
    torch.cuda.synchronize()
    return out.cpu().double().numpy()


@pytest.mark.parametrize("wl,tol", [(0, TOL_FP32), (1, TOL_FP32), (2, TOL_LOWP_OUT)])
def test_fused_fusion_matches_oracle(wl, tol):
    pr = inputs.make_workload(wl, with_grad=False)
    if wl == 1:
        pr = pr.anchors(range(300))
    vis = inputs.make_visibility(pr, wl)
    got = gpu_oae(pr, vis)
    ref = oracle.forward_oae(*pr.tensors(), vis)
    err = relerr(got, ref)
    print(f"fused fusion workload {wl}: rel err {err:.2e}")
    assert err <= tol


@pytest.mark.parametrize("vec", [1, 2, 4])
def test_uniform_visibility_is_forward_over_ncam(vec):
    pr = inputs.make_workload(1, feat_dtype="bf16", with_grad=False).anchors(range(100))
    vis = torch.full(pr.sampling_location.shape[:2] + (pr.sampling_location.shape[3],), 0.25)
    got = gpu_oae(pr, vis, vec=vec)
    d = pr.to("cuda")
    plain = msda.forward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights,
                         workspace=None, vec=vec).cpu().double().numpy()
    assert relerr(got, plain / 6.0) <= 1e-6


def test_zero_visibility_anchor_is_zero_and_one_hot_selects_camera():
    pr = inputs.make_workload(0)
    vis = torch.rand(1, 16, 2)
    vis[0, 3] = 0.0
    vis[0, 5] = torch.tensor([0.0, 2.0])
    got = gpu_oae(pr, vis)
    assert np.all(got[0, 3] == 0.0)
    ref = oracle.forward_oae(*pr.tensors(), vis)
    assert relerr(got, ref) <= TOL_FP32


def test_single_stage_fused_fusion_matches_the_default_form():
    pr = inputs.make_workload(2, with_grad=False).anchors(range(100))
    vis = inputs.make_visibility(pr, 3).to("cuda")
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    a = msda.forward_oae(*T, vis)
    b = msda.forward_oae(*T, vis, variant=4)
    assert relerr(b.cpu().double().numpy(), a.cpu().double().numpy()) <= TOL_FP32  # another FP32 sum order
