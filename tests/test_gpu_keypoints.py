"""Keypoint prologue on the GPU against the FP64 oracle, and the chained path
prologue -> operator against the oracle chain."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_LOWP_OUT, ensure_lib, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


@pytest.mark.parametrize("B,A,P,K", [(1, 900, 13, 64), (2, 37, 9, 5), (1, 1, 1, 1), (1, 0, 13, 4)])
def test_keypoints_match_oracle(B, A, P, K):
    geo = inputs.make_scene_geometry(B + A + K, B=B, A=A, P=P, ncam=K)
    got = msda.keypoints(*[t.cuda() for t in geo]).cpu().double().numpy()
    ref = oracle.keypoints(*geo)
    if ref.size:
        # normalised image coordinates: absolute error; behind-camera markers must agree exactly
        assert np.abs(got - ref).max() <= 1e-5
        assert np.array_equal(got == -2.0, ref == -2.0)


def test_prologue_then_operator():
    pr = inputs.make_workload(2, ncam=16, with_grad=False)
    geo = inputs.make_scene_geometry(5, B=1, A=900, P=13, ncam=16)
    loc = msda.keypoints(*[t.cuda() for t in geo])
    d = pr.to("cuda")
    out = msda.forward(d.feat, d.spatial_shape, d.scale_start_index, loc, d.weights)
    ref = oracle.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, loc.cpu(), pr.weights, nthreads=8)
    assert relerr(out.cpu().double().numpy(), ref) <= TOL_LOWP_OUT
