"""Forward parity: the CUDA kernels against the FP64 oracle, through the C-ABI."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (TOL_FP32, TOL_LOWP_OUT, ensure_lib, gpu_forward, is_lowp, oracle_forward, relerr)
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


# the two forward kernels: staged camera-group (workspace) and anchor-per-block (none)
PATHS = ["auto", None]


@pytest.mark.parametrize("warps", [1, 2, 4, 8])
def test_tiny_fp32_all_tunings(warps):
    pr = inputs.make_workload(0)
    out = gpu_forward(pr, warps=warps, workspace=None).cpu().double().numpy()
    ref = oracle_forward(pr)
    assert relerr(out, ref) <= TOL_FP32


def test_tiny_fp32_staged():
    pr = inputs.make_workload(0)
    assert relerr(gpu_forward(pr).cpu().double().numpy(), oracle_forward(pr)) <= TOL_FP32


@pytest.mark.parametrize("ws", PATHS)
def test_sparse4d_6cam_fp32_full(ws):
    pr = inputs.make_workload(1, with_grad=False)
    err = relerr(gpu_forward(pr, workspace=ws).cpu().double().numpy(), oracle_forward(pr))
    print(f"sparse4d-6cam FP32 ws={ws} rel err {err:.3e}")
    assert err <= TOL_FP32


@pytest.mark.parametrize("ws", PATHS)
@pytest.mark.parametrize("fdt,wdt", [("bf16", "f32"), ("bf16", "bf16"), ("f16", "f16"), ("f16", "f32")])
def test_sparse4d_6cam_lowp(fdt, wdt, ws):
    pr = inputs.make_workload(1, feat_dtype=fdt, w_dtype=wdt, with_grad=False)
    err = relerr(gpu_forward(pr, workspace=ws).cpu().double().numpy(), oracle_forward(pr))
    print(f"sparse4d-6cam {fdt}/{wdt} rel err {err:.3e}")
    assert err <= TOL_LOWP_OUT
    assert err <= 1e-5  # same rounded inputs on both sides: only FP32 arithmetic differs


@pytest.mark.parametrize("ws", PATHS)
def test_outside_in_64cam_bf16_full(ws):
    pr = inputs.make_workload(2, with_grad=False)
    out = gpu_forward(pr, workspace=ws)
    err = relerr(out.cpu().double().numpy(), oracle_forward(pr))
    print(f"outside-in-64cam BF16 ws={ws} rel err {err:.3e}")
    assert err <= TOL_LOWP_OUT
    # same launch configuration: bitwise reproducible
    out2 = gpu_forward(pr, workspace=ws)
    assert torch.equal(out, out2)


@pytest.mark.parametrize("ws", PATHS)
def test_train_16cam_forward_full(ws):
    pr = inputs.make_workload(3, with_grad=False)
    err = relerr(gpu_forward(pr, workspace=ws).cpu().double().numpy(), oracle_forward(pr))
    print(f"train-16cam BF16/FP32 rel err {err:.3e}")
    assert err <= TOL_LOWP_OUT


@pytest.mark.parametrize("ws", PATHS)
@pytest.mark.parametrize("odt", [torch.bfloat16, torch.float16])
def test_reduced_precision_output_is_rounded_fp32(odt, ws):
    pr = inputs.make_workload(1, feat_dtype="bf16", with_grad=False).anchors(range(200))
    o32 = gpu_forward(pr, workspace=ws)
    olp = gpu_forward(pr, out_dtype=odt, workspace=ws)
    assert torch.equal(olp, o32.to(odt))


HETERO = [[(5, 7), (3, 4), (2, 2)], [(9, 4), (4, 2), (1, 1)], [(6, 13), (3, 7), (2, 3)]]


def split_supported(C, G, fdt):
    """The channel-split rule stated in include/msda.h."""
    vec = 16 // (4 if fdt == "f32" else 2)
    for n in (1, 2, 4):
        cpl = vec * n
        if C % cpl == 0 and (C // G) % cpl == 0:
            r = C // cpl
            if r <= 32 and r & (r - 1) == 0:
                return True
    return False


@pytest.mark.parametrize("ws", PATHS)
@pytest.mark.parametrize("C,G,fdt", [(32, 4, "f32"), (64, 4, "f32"), (64, 8, "bf16"), (128, 2, "bf16"),
                                     (512, 8, "bf16"), (1024, 8, "bf16"), (96, 2, "f32"), (48, 3, "bf16"),
                                     (256, 32, "bf16"), (256, 2, "f32")])
def test_channel_splits_and_ragged_maps(C, G, fdt, ws):
    gen = torch.Generator().manual_seed(C * 7 + G)
    pr = inputs.make_problem(gen, B=2, cam_maps=HETERO, C=C, G=G, A=37, P=5, loc_range=(-0.3, 1.3),
                             feat_dtype=fdt, w_dtype=fdt, with_grad=False)
    if not split_supported(C, G, fdt):
        # the header's channel-split rule rejects this split: the call must say so, not compute
        with pytest.raises(msda.MSDAError) as e:
            gpu_forward(pr, workspace=ws)
        assert e.value.code == 2
        return
    out = gpu_forward(pr, workspace=ws)
    tol = TOL_FP32 if fdt == "f32" else TOL_LOWP_OUT
    assert relerr(out.cpu().double().numpy(), oracle_forward(pr)) <= tol


def test_unsupported_split_is_an_error():
    gen = torch.Generator().manual_seed(1)
    pr = inputs.make_problem(gen, B=1, cam_maps=HETERO, C=48, G=6, A=3, P=2, with_grad=False)  # Cg*4 = 32 B, rt=12
    with pytest.raises(msda.MSDAError):
        gpu_forward(pr)


def test_many_cameras_and_scales():
    gen = torch.Generator().manual_seed(5)
    maps = [[(12 + k % 5, 9 + k % 3), (6, 5), (3, 3), (2, 1), (1, 2), (1, 1)] for k in range(96)]
    pr = inputs.make_problem(gen, B=1, cam_maps=maps, C=64, G=8, A=20, P=13, loc_range=(-0.1, 1.1),
                             feat_dtype="bf16", w_dtype="bf16", with_grad=False)
    assert relerr(gpu_forward(pr).cpu().double().numpy(), oracle_forward(pr)) <= TOL_LOWP_OUT


@pytest.mark.parametrize("ws", PATHS)
@pytest.mark.parametrize("dims", [dict(A=0), dict(B=0), dict(P=0), dict(Ncam=0)])
def test_empty_problems(dims, ws):
    B, A, P = dims.get("B", 2), dims.get("A", 5), dims.get("P", 3)
    maps = [] if dims.get("Ncam", 1) == 0 else [[(4, 4), (2, 2)]]
    if not maps:
        feat = torch.randn(B, 0, 32)
        shape = torch.zeros(0, 2, 2, dtype=torch.int32)
        start = torch.zeros(0, 2, dtype=torch.int32)
        loc = torch.rand(B, A, P, 0, 2)
        w = torch.rand(B, A, P, 0, 2, 4)
        pr = inputs.Problem(feat, shape, start, loc, w, None)
    else:
        gen = torch.Generator().manual_seed(0)
        pr = inputs.make_problem(gen, B=B, cam_maps=maps, C=32, G=4, A=A, P=P, with_grad=False)
    out = gpu_forward(pr, workspace=ws)
    assert out.shape == (B, A, 32)
    assert torch.all(out == 0)


@pytest.mark.parametrize("ws", PATHS)
def test_nan_inf_and_far_points_contribute_nothing(ws):
    pr = inputs.make_workload(0)
    loc = pr.sampling_location.clone()
    loc[0, 0, 0, 0, 0] = float("nan")
    loc[0, 1, 1, 1, 1] = float("inf")
    loc[0, 2, 2, 0, 0] = -float("inf")
    loc[0, 3, :, :, 0] = 5.0
    loc[0, 4, :, :, 1] = -1e30
    pr.sampling_location = loc
    out = gpu_forward(pr, workspace=ws).cpu().double().numpy()
    ref = oracle_forward(pr)
    assert np.all(out[0, 3] == 0) and np.all(out[0, 4] == 0)
    assert relerr(out, ref) <= TOL_FP32


@pytest.mark.parametrize("ws", PATHS)
def test_boundary_points_exact_grid(ws):
    """Points exactly on pixel centres, cell borders and the drop border (-0.5/W, 1+0.5/W)."""
    gen = torch.Generator().manual_seed(9)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(16, 16), (8, 8)], [(4, 32), (2, 16)]], C=32, G=4, A=8, P=16,
                             with_grad=False)
    vals = torch.tensor([-1 / 32, -1 / 64, 0.0, 1 / 64, 1 / 32, 0.5, 1 - 1 / 64, 1.0, 1 + 1 / 64, 1 + 1 / 32,
                         0.25, 0.75, 3 / 32, 29 / 32, -0.0, 0.125])
    loc = pr.sampling_location
    for a in range(8):
        for p in range(16):
            loc[0, a, p, :, 0] = vals[p]
            loc[0, a, p, :, 1] = vals[(p + a) % 16]
    out = gpu_forward(pr, workspace=ws).cpu().double().numpy()
    assert relerr(out, oracle_forward(pr)) <= TOL_FP32


@pytest.mark.parametrize("ws", PATHS)
def test_bad_map_table_is_reported_and_skipped(ws):
    pr = inputs.make_workload(0)
    start = pr.scale_start_index.clone()
    start[1, 0] = pr.feat.shape[1] - 10  # map would run past sum_hw
    bad = inputs.Problem(pr.feat, pr.spatial_shape, start, pr.sampling_location, pr.weights, None)
    msda.device_status()  # clear
    out = gpu_forward(bad, workspace=ws).cpu().double().numpy()
    assert msda.device_status() == 5  # MSDA_ERR_OUT_OF_RANGE
    w = pr.weights.clone()
    w[:, :, :, 1, 0, :] = 0  # the skipped map contributes nothing
    ref = oracle_forward(inputs.Problem(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, w, None))
    assert relerr(out, ref) <= TOL_FP32
    assert msda.device_status() == 0


@pytest.mark.parametrize("ws", PATHS)
def test_anchor_and_camera_permutation_invariance(ws):
    pr = inputs.make_workload(1, feat_dtype="bf16", with_grad=False).anchors(range(64))
    out = gpu_forward(pr, workspace=ws).cpu()
    perm = torch.randperm(64, generator=torch.Generator().manual_seed(3))
    out_p = gpu_forward(pr.anchors(perm), workspace=ws).cpu()
    assert torch.equal(out_p, out[:, perm])
    # relabel cameras: permute the tables and the camera axis of loc/weights
    cp = torch.tensor([3, 0, 5, 1, 4, 2])
    pr2 = inputs.Problem(pr.feat, pr.spatial_shape[cp].contiguous(), pr.scale_start_index[cp].contiguous(),
                         pr.sampling_location[:, :, :, cp].contiguous(), pr.weights[:, :, :, cp].contiguous(), None)
    out_c = gpu_forward(pr2, workspace=ws).cpu().double().numpy()
    assert relerr(out_c, out.double().numpy()) <= 1e-6  # same terms, different summation order


def test_staged_and_anchor_kernels_agree():
    pr = inputs.make_workload(2, ncam=12, with_grad=False)
    a = gpu_forward(pr).cpu().double().numpy()
    b = gpu_forward(pr, workspace=None).cpu().double().numpy()
    assert relerr(a, b) <= 1e-6


@pytest.mark.parametrize("wl,fdt,wdt", [(0, None, None), (1, "f32", "f32"), (1, "bf16", "bf16"), (1, "f16", "f32"),
                                        (2, None, None), (3, None, None)])
@pytest.mark.parametrize("vec", [1, 2, 4])
def test_two_stage_and_single_stage_forwards(wl, fdt, wdt, vec):
    """The default two-stage forward (each chunk of point-scales culled and located once into a shared-memory
    list that the teams share out) and the single-stage one (variant 4, every lane locates its own
    point-scales): both equal to the oracle, equal to each other within FP32 rounding, bitwise stable."""
    kw = dict(feat_dtype=fdt, w_dtype=wdt) if fdt else {}
    pr = inputs.make_workload(wl, with_grad=False, **kw)
    if wl >= 2:
        pr = pr.anchors(range(120))
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    ref = oracle_forward(pr)
    for warps in (1, 2, 8):
        got = msda.forward(*T, warps=warps, vec=vec, variant=4)
        again = msda.forward(*T, warps=warps, vec=vec, variant=4)
        plain = msda.forward(*T, warps=warps, vec=vec)
        torch.cuda.synchronize()
        assert torch.equal(got, again)
        assert relerr(got.cpu().double().numpy(), plain.cpu().double().numpy()) <= TOL_FP32  # another sum order
        err = relerr(got.cpu().double().numpy(), ref)
        assert err <= (TOL_LOWP_OUT if is_lowp(pr) else TOL_FP32), (warps, err)
    assert msda.device_status() == 0


def test_single_stage_forward_edge_cases():
    """NaN and far points, boundary cells, maps of one pixel, no anchors, no points (variant 4; the default form
    meets the same cases in the tests above)."""
    gen = torch.Generator().manual_seed(21)
    pr = inputs.make_problem(gen, B=2, cam_maps=[[(5, 7), (3, 2), (1, 1)]] * 3, C=64, G=4, A=9, P=5,
                             loc_range=(-0.3, 1.3))
    loc = pr.sampling_location.clone()
    loc[0, 0, 0, 0] = float("nan")
    loc[1, 2, 1, 1] = torch.tensor([1e9, -1e9])
    loc[0, 3, 2, 2] = torch.tensor([0.0, 1.0])
    pr = inputs.Problem(pr.feat, pr.spatial_shape, pr.scale_start_index, loc.contiguous(), pr.weights, None)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    for warps in (1, 4):
        got = msda.forward(*T, variant=4, warps=warps)
        assert relerr(got.cpu().double().numpy(), oracle_forward(pr)) <= TOL_FP32
    for A, P in ((0, 2), (3, 0)):
        e = inputs.make_problem(gen, B=1, cam_maps=[[(4, 4)]], C=32, G=4, A=A, P=P).to("cuda")
        out = msda.forward(e.feat, e.spatial_shape, e.scale_start_index, e.sampling_location, e.weights, variant=4)
        assert out.shape == (1, A, 32) and (out.numel() == 0 or torch.all(out == 0))
    assert msda.device_status() == 0
