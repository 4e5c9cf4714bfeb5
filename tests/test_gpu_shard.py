"""The camera split of the operator run through the CUDA kernels on one GPU.

The operator is a sum over cameras, so a frame splits exactly by camera: each shard (a camera subset with its
maps re-packed densely, paper_2601_10819_gb300.shard) gives a partial output, and the partial outputs summed
give the frame's output; each camera's feature, location and weight gradients come from its own shard.  Here
every shard runs through msda.forward / msda.backward on the same GPU, the stand-in for one rank per shard.
"""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_LOWP_OUT, ensure_lib, oracle_forward, relerr
from paper_2601_10819_gb300 import inputs, msda, shard

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


@pytest.fixture(scope="module")
def frame():
    """The 64-camera benchmark frame, its unsharded output and gradients (both backward modes)."""
    pr = inputs.make_workload(2)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    out = msda.forward(*T)
    grads = {det: [g.clone() for g in msda.backward(*T, d.grad_out, deterministic=det)] for det in (False, True)}
    torch.cuda.synchronize()
    return pr, d, T, out, grads


def shard_rows(spatial_shape, scale_start_index, cams):
    """Rows of the unsharded feature tensor that the shard of `cams` re-packs, in the shard's order."""
    rows = []
    for k in cams:
        for s in range(spatial_shape.shape[1]):
            h, w = int(spatial_shape[k, s, 0]), int(spatial_shape[k, s, 1])
            st = int(scale_start_index[k, s])
            rows.extend(range(st, st + h * w))
    return torch.tensor(rows, dtype=torch.long)


@pytest.mark.parametrize("nshards", [2, 3, 8])
def test_partial_outputs_sum_to_the_frame(frame, nshards):
    pr, d, T, out, _ = frame
    total = torch.zeros_like(out)
    for cams in shard.split_cameras(pr.spatial_shape.shape[0], nshards):
        sub = shard.shard_problem(*T, cams)
        total += msda.forward(*sub)  # partial sums added in shard order, as one sum all-reduce would
    torch.cuda.synchronize()
    e_full = relerr(total.cpu().double().numpy(), out.cpu().double().numpy())
    e_oracle = relerr(total.cpu().double().numpy(), oracle_forward(pr))
    print(f"{nshards} shards: rel err vs unsharded {e_full:.2e}, vs oracle {e_oracle:.2e}")
    assert e_full <= 1e-5  # the same FP32 products summed in another order
    assert e_oracle <= TOL_LOWP_OUT
    assert msda.device_status() == 0


@pytest.mark.parametrize("nshards", [2, 3, 8])
@pytest.mark.parametrize("det", [False, True])
def test_shard_gradients_are_the_frames_slices(frame, nshards, det):
    """Each shard's gradients equal the unsharded gradients of its cameras: bitwise in the deterministic mode
    (every row and every point-scale is summed in the same order), to rounding in the atomic one."""
    pr, d, T, _, grads = frame
    gf, gl, gw = grads[det]
    for cams in shard.split_cameras(pr.spatial_shape.shape[0], nshards):
        sub = shard.shard_problem(*T, cams)
        sgf, sgl, sgw = msda.backward(*sub, d.grad_out, deterministic=det)
        torch.cuda.synchronize()
        rows = shard_rows(pr.spatial_shape, pr.scale_start_index, cams).to("cuda")
        c = torch.tensor(cams, dtype=torch.long, device="cuda")
        want = (gf.index_select(1, rows), gl.index_select(3, c), gw.index_select(3, c))
        for name, x, y in zip(("dfeat", "dloc", "dw"), (sgf, sgl, sgw), want):
            if det:
                assert torch.equal(x, y), f"{nshards} shards, {name} of cameras {cams[0]}..{cams[-1]}"
            else:
                e = relerr(x.cpu().double().numpy(), y.cpu().double().numpy())
                assert e <= 1e-5, (name, e)
    assert msda.device_status() == 0
