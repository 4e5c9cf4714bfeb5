"""The half2-accumulating forward (the paper's FP16 plugin arithmetic, Sec. 5.3).

Its error against the FP64 oracle (same rounded FP16 inputs) is measured and
bounded; the FP32-accumulating kernel on the same inputs is far more exact.
"""
import pytest
import torch

import oracle
from gpu_util import ensure_lib, gpu_forward, oracle_forward, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu

TOL_HALF_ACC = 3e-2  # fp16 sums of ~3000 terms of ~1e-4 each carry ~1e-3..1e-2 relative error


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


@pytest.mark.parametrize("wl", [1, 2])
@pytest.mark.parametrize("vec", [1, 2])
def test_half2_accumulation_error_is_bounded(wl, vec):
    pr = inputs.make_workload(wl, feat_dtype="f16", w_dtype="f16", with_grad=False)
    if wl == 1:
        pr = pr.anchors(range(300))
    ref = oracle_forward(pr)
    e_h = relerr(gpu_forward(pr, workspace=None, variant=3, vec=vec).cpu().double().numpy(), ref)
    e_f = relerr(gpu_forward(pr, workspace=None, vec=vec).cpu().double().numpy(), ref)
    print(f"workload {wl} vec {vec}: half2 accumulation rel err {e_h:.2e}, fp32 accumulation {e_f:.2e}")
    assert e_h <= TOL_HALF_ACC
    assert e_f <= 1e-5 and e_f < e_h


def test_half2_requires_fp16():
    pr = inputs.make_workload(0)
    with pytest.raises(msda.MSDAError):
        gpu_forward(pr, workspace=None, variant=3)
