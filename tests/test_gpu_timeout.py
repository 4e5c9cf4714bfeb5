"""Failure detection of the staged kernels' bounded waits, without a GPU fault.

The staged kernels wait on an mbarrier for their bulk copies and give up after a bounded number of polls,
reporting MSDA_ERR_TIMEOUT through the device status word instead of hanging.  msda_debug_set_wait_limit(0)
makes the first wait of every staging step give up at once (the copies still land: a second, full-length
wait drains them), so each call below must report TIMEOUT, and the next call at the default limit must
report OK and match the oracle.
"""
import pytest
import torch

import oracle
from gpu_util import TOL_FP32, TOL_LOWP_GRAD, ensure_lib, oracle_backward, oracle_forward, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu

TIMEOUT = 4


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


def tensors(pr):
    d = pr.to("cuda")
    return d, (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)


def gives_up_then_recovers(call):
    """call() runs the staged path once; returns its result on the second, normal run."""
    msda.device_status()  # clear
    msda.debug_set_wait_limit(0)
    try:
        call()
        assert msda.device_status() == TIMEOUT
    finally:
        msda.debug_set_wait_limit(-1)
    res = call()
    torch.cuda.synchronize()
    assert msda.device_status() == 0
    return res


def test_staged_forward():
    pr = inputs.make_workload(0)
    d, T = tensors(pr)
    B, sum_hw, C = d.feat.shape
    _, A, P, K, _ = d.sampling_location.shape
    S, G = d.weights.shape[4], d.weights.shape[5]
    ws = torch.empty(msda.forward_workspace_size(B, sum_hw, C, K, S, A, P, G), dtype=torch.uint8, device="cuda")
    out = gives_up_then_recovers(lambda: msda.forward(*T, workspace=ws))
    assert relerr(out.cpu().double().numpy(), oracle_forward(pr)) <= TOL_FP32


@pytest.mark.parametrize("variant", [0, 2])  # cell-binned band staging; staged camera-group form
def test_staged_deterministic_backward(variant):
    pr = inputs.make_workload(0)
    d, T = tensors(pr)
    g = gives_up_then_recovers(lambda: msda.backward(*T, d.grad_out, deterministic=True, variant=variant))
    for x, r in zip(g, oracle_backward(pr)):
        assert relerr(x.cpu().double().numpy(), r) <= TOL_FP32


def test_bands_read_in_place_give_up_then_recover():
    """A dense coarse map whose bands exceed a buffer and are swept in place: their barrier phase completes with a
    plain arrival, and the give-up path and the recovery behave as for staged bands."""
    gen = torch.Generator().manual_seed(1604)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(2, 3), (1, 2)]], C=256, G=8, A=900, P=4, loc_range=(0.0, 1.0),
                             feat_dtype="bf16", w_dtype="bf16")
    d, T = tensors(pr)
    g = gives_up_then_recovers(lambda: msda.backward(*T, d.grad_out, deterministic=True))
    for x, r in zip(g, oracle_backward(pr)):
        assert relerr(x.cpu().double().numpy(), r) <= TOL_LOWP_GRAD
