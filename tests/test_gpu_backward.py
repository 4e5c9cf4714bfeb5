"""Backward parity: atomic and deterministic modes against the FP64 oracle."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (TOL_FP32, TOL_LOWP_GRAD, TOL_LOWP_OUT, ensure_lib, is_lowp, oracle_backward, oracle_forward,
                      relerr)
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


def gpu_backward(pr, deterministic, warps=None, variant=0):
    d = pr.to("cuda")
    g = msda.backward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights, d.grad_out,
                      deterministic=deterministic, warps=warps, variant=variant)
    torch.cuda.synchronize()
    return [t.cpu() for t in g]


def check_against_oracle(pr, grads, tol, label=""):
    ref = oracle_backward(pr)
    errs = [relerr(g.double().numpy(), r) for g, r in zip(grads, ref)]
    print(f"{label} rel err dfeat {errs[0]:.2e} dloc {errs[1]:.2e} dw {errs[2]:.2e}")
    assert max(errs) <= tol, errs
    return errs


# (deterministic, variant): atomic scatter, deterministic (cell-binned where it applies), staged deterministic,
# deterministic corner-slot form
MODES = [(False, 0), (True, 0), (True, 2), (True, 5)]


@pytest.mark.parametrize("det,variant", MODES)
@pytest.mark.parametrize("warps", [1, 4, 8])
def test_tiny_fp32(det, variant, warps):
    pr = inputs.make_workload(0)
    check_against_oracle(pr, gpu_backward(pr, det, warps, variant), TOL_FP32, f"tiny det={det}/{variant} warps={warps}")


@pytest.mark.parametrize("det,variant", MODES)
def test_sparse4d_fp32_subset(det, variant):
    pr = inputs.make_workload(1).anchors(range(150))
    check_against_oracle(pr, gpu_backward(pr, det, None, variant), TOL_FP32, f"sparse4d fp32 det={det}/{variant}")


@pytest.mark.parametrize("det,variant", MODES)
def test_train_16cam_bf16_subset(det, variant):
    pr = inputs.make_workload(3, batch=2).anchors(range(120))
    check_against_oracle(pr, gpu_backward(pr, det, None, variant), TOL_LOWP_GRAD, f"train bf16 det={det}/{variant}")


HETERO = [[(5, 7), (3, 4), (2, 2)], [(9, 4), (4, 2), (1, 1)], [(6, 13), (3, 7), (2, 3)]]


@pytest.mark.parametrize("C,G,fdt", [(32, 4, "f32"), (64, 8, "bf16"), (128, 2, "f16"), (512, 8, "bf16"),
                                     (256, 32, "bf16"), (256, 2, "f32")])
@pytest.mark.parametrize("det,variant", MODES)
def test_ragged_maps_and_splits(C, G, fdt, det, variant):
    gen = torch.Generator().manual_seed(C + G)
    pr = inputs.make_problem(gen, B=2, cam_maps=HETERO, C=C, G=G, A=23, P=5, loc_range=(-0.3, 1.3),
                             feat_dtype=fdt, w_dtype=fdt)
    tol = TOL_FP32 if not is_lowp(pr) else TOL_LOWP_GRAD
    check_against_oracle(pr, gpu_backward(pr, det, None, variant), tol, f"ragged C={C} G={G} {fdt} det={det}/{variant}")


@pytest.mark.parametrize("variant", [0, 2, 5])
def test_deterministic_mode_is_bitwise_reproducible(variant):
    pr = inputs.make_workload(2, ncam=8)
    a = gpu_backward(pr, True, 8, variant)
    b = gpu_backward(pr, True, 8, variant)
    c = gpu_backward(pr, True, 4, variant)
    for x, y, z in zip(a, b, c):
        assert torch.equal(x, y)
        assert torch.equal(x, z)  # every gradient is computed in a fixed order independent of the warps


def test_all_modes_agree():
    pr = inputs.make_workload(2, ncam=8)
    a = gpu_backward(pr, False)
    d = gpu_backward(pr, True)           # rows grouped by a counting sort
    st = gpu_backward(pr, True, None, 2)  # staged camera-group form
    # dw: the same per-scale expression and group sum in the atomic kernel and the anchor-block kernel of the
    # row-grouped form, no atomics (dloc sums in another fixed order: per-scale team sums, in scale order)
    assert torch.equal(a[2], d[2])
    for x, y, z in zip(a, d, st):
        assert relerr(x.double().numpy(), y.double().numpy()) <= 1e-6
        assert relerr(x.double().numpy(), z.double().numpy()) <= 1e-6


def test_outside_in_64cam_full_backward():
    """The benchmark's workload: every gradient against the oracle at full size."""
    pr = inputs.make_workload(2)
    ga = gpu_backward(pr, False)
    ref = oracle_backward(pr)
    for g, r, name in zip(ga, ref, ["dfeat", "dloc", "dw"]):
        e = relerr(g.double().numpy(), r)
        print(f"outside-in-64cam {name} rel err {e:.2e}")
        assert e <= TOL_LOWP_GRAD
    for variant in (0, 2, 5):
        gd = gpu_backward(pr, True, None, variant)
        for g, r, name in zip(gd, ref, ["dfeat", "dloc", "dw"]):
            e = relerr(g.double().numpy(), r)
            print(f"outside-in-64cam deterministic/{variant} {name} rel err {e:.2e}")
            assert e <= TOL_LOWP_GRAD


def test_train_16cam_full_elementwise():
    """The 16-camera training batch at full size (B=4, BF16 features, FP32 weights): every element of the three
    gradients against the oracle, frame by frame, in the atomic and the deterministic mode; plus the adjoint
    identities <grad_out, out> = <grad_feat, feat> = <grad_w, w> on the whole batch."""
    pr = inputs.make_workload(3)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    out = msda.forward(*T)
    modes = {det: [g.cpu() for g in msda.backward(*T, d.grad_out, deterministic=det)] for det in (False, True)}
    gf = modes[False][0]
    lhs = float((d.grad_out.double() * out.double()).sum())
    assert abs(lhs - float((gf.double() * pr.feat.double()).sum())) <= 1e-4 * abs(lhs)
    assert abs(lhs - float((modes[False][2].double() * pr.weights.double()).sum())) <= 1e-4 * abs(lhs)
    for b in range(pr.feat.shape[0]):
        frame = inputs.Problem(pr.feat[b:b + 1].contiguous(), pr.spatial_shape, pr.scale_start_index,
                               pr.sampling_location[b:b + 1].contiguous(), pr.weights[b:b + 1].contiguous(),
                               pr.grad_out[b:b + 1].contiguous())
        ref = oracle_backward(frame)
        for det, grads in modes.items():
            for name, g, r in zip(("dfeat", "dloc", "dw"), grads, ref):
                e = relerr(g[b:b + 1].double().numpy(), r)
                print(f"train-16cam frame {b} det={det} {name} rel err {e:.2e}")
                assert e <= TOL_LOWP_GRAD, (b, det, name, e)


def test_autograd_function_matches_direct_calls_and_gradcheck():
    pr = inputs.make_workload(0)
    d = pr.to("cuda")
    feat = d.feat.clone().requires_grad_()
    loc = d.sampling_location.clone().requires_grad_()
    w = d.weights.clone().requires_grad_()
    out = msda.msda(feat, d.spatial_shape, d.scale_start_index, loc, w)
    out.backward(d.grad_out)
    gf, gl, gw = msda.backward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights,
                               d.grad_out, deterministic=True)
    # the autograd function's default backward is the deterministic mode: bitwise the direct call
    assert torch.equal(w.grad, gw) and torch.equal(loc.grad, gl) and torch.equal(feat.grad, gf)
    feat.grad = loc.grad = w.grad = None
    msda.msda(feat, d.spatial_shape, d.scale_start_index, loc, w, False).backward(d.grad_out)
    ga = msda.backward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights, d.grad_out)
    assert torch.equal(w.grad, ga[2]) and torch.equal(loc.grad, ga[1])  # no atomics in dloc, dw
    assert relerr(feat.grad.cpu().double().numpy(), ga[0].cpu().double().numpy()) <= 1e-6  # atomic order varies
    # the operator is linear in feat and weights: finite differences are exact up to rounding
    f0 = d.feat.clone().requires_grad_()
    w0 = d.weights.clone().requires_grad_()
    fn = lambda f, ww: msda.msda(f, d.spatial_shape, d.scale_start_index, d.sampling_location, ww, True)
    assert torch.autograd.gradcheck(fn, (f0, w0), eps=1e-2, atol=2e-3, rtol=1e-2, fast_mode=True)


@pytest.mark.parametrize("det,variant", MODES)
def test_out_of_view_points_have_zero_gradients(det, variant):
    pr = inputs.make_workload(0)
    pr.sampling_location[0, :5, :, :, 0] = 3.0
    gf, gl, gw = gpu_backward(pr, det, None, variant)
    assert torch.all(gl[0, :5] == 0) and torch.all(gw[0, :5] == 0)
    check_against_oracle(pr, (gf, gl, gw), TOL_FP32, "out of view")


def test_empty_backward():
    gen = torch.Generator().manual_seed(0)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(4, 4)]], C=32, G=4, A=0, P=2)
    for det, variant in MODES:
        gf, gl, gw = gpu_backward(pr, det, None, variant)
        assert torch.all(gf == 0) and gl.numel() == 0 and gw.numel() == 0


def test_uncovered_rows_are_zero_and_overlaps_reported():
    """Rows outside every map get zero gradient; overlapping maps raise the status word (staged mode)."""
    gen = torch.Generator().manual_seed(3)
    pr = inputs.make_problem(gen, B=2, cam_maps=[[(6, 5), (3, 2)], [(4, 4), (2, 2)]], C=32, G=4, A=7, P=3)
    pad = 9
    feat = torch.cat([pr.feat, torch.randn(2, pad, 32)], dim=1)  # rows no map covers
    gap = inputs.Problem(feat.contiguous(), pr.spatial_shape, pr.scale_start_index, pr.sampling_location,
                         pr.weights, pr.grad_out)
    msda.device_status()
    for det, variant in MODES:
        g = gpu_backward(gap, det, None, variant)
        assert torch.all(g[0][:, -pad:] == 0)
        check_against_oracle(gap, g, TOL_FP32, f"padded rows det={det}/{variant}")
    assert msda.device_status() == 0
    start = pr.scale_start_index.clone()
    start[1, 0] = 0  # camera 1 scale 0 overlaps camera 0
    ov = inputs.Problem(pr.feat, pr.spatial_shape, start, pr.sampling_location, pr.weights, pr.grad_out)
    gpu_backward(ov, True, None, 2)  # the staged form needs disjoint maps and reports the overlap
    assert msda.device_status() == 5
    g = gpu_backward(ov, True)  # the row-grouped form handles overlapping maps
    check_against_oracle(ov, g, TOL_FP32, "overlapping maps, row-grouped form")
    assert msda.device_status() == 0


def test_caller_zeroed_flag_accumulates_into_grad_feat():
    pr = inputs.make_workload(0)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    ref = msda.backward(*T, d.grad_out)
    gf = torch.zeros_like(ref[0])
    got = msda.backward(*T, d.grad_out, grads=(gf, torch.empty_like(ref[1]), torch.empty_like(ref[2])),
                        grad_feat_zeroed=True)
    assert relerr(got[0].cpu().double().numpy(), ref[0].cpu().double().numpy()) <= 1e-6
    assert torch.equal(got[1], ref[1]) and torch.equal(got[2], ref[2])
    ones = torch.ones_like(ref[0])
    got = msda.backward(*T, d.grad_out, grads=(ones, torch.empty_like(ref[1]), torch.empty_like(ref[2])),
                        grad_feat_zeroed=True)
    assert relerr(got[0].cpu().double().numpy() - 1.0, ref[0].cpu().double().numpy()) <= 1e-6


def _relayout(pr, layout, gen):
    """The same maps with another row layout: scale-major, padded with uncovered rows, or overlapping."""
    shape, start = pr.spatial_shape, pr.scale_start_index.clone()
    ncam, nscale = start.shape
    sizes = (shape[..., 0] * shape[..., 1]).long()
    feat = pr.feat
    if layout == "scale-major":
        pos = 0
        for s in range(nscale):
            for k in range(ncam):
                start[k, s] = pos
                pos += int(sizes[k, s])
    elif layout == "padded":
        pos = 5  # uncovered rows before, between and after the maps
        for k in range(ncam):
            for s in range(nscale):
                start[k, s] = pos
                pos += int(sizes[k, s]) + 3
        B, _, C = feat.shape
        feat = torch.randn(B, pos + 7, C, generator=gen).to(feat.dtype)
    elif layout == "overlapping":
        start[ncam - 1, 0] = 0  # the last camera's finest map reuses the first camera's rows
    elif layout != "camera-major":
        raise ValueError(layout)
    return inputs.Problem(feat.contiguous(), shape, start, pr.sampling_location, pr.weights, pr.grad_out)


@pytest.mark.parametrize("layout", ["camera-major", "scale-major", "padded", "overlapping"])
def test_atomic_item_orders_over_row_layouts(layout):
    """The atomic backward's ordered hand-out (a work counter in the workspace) and static stride (no
    workspace) over row layouts that do not follow the camera order, against the oracle; the output
    buffers start out as NaN, so every element must be written (uncovered rows as zero)."""
    gen = torch.Generator().manual_seed(11)
    maps = [[(9, 13), (5, 7), (3, 4)], [(8, 8), (4, 4), (2, 2)], [(12, 5), (6, 3), (3, 2)]]
    pr = _relayout(inputs.make_problem(gen, B=3, cam_maps=maps, C=64, G=4, A=37, P=5, loc_range=(-0.1, 1.1)),
                   layout, gen)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    B, sum_hw, C = d.feat.shape
    msda.device_status()
    res = {}
    for name, ws_bytes in (("ordered", 256), ("static", 0)):
        grads = tuple(torch.full(s, float("nan"), device="cuda")
                      for s in ((B, sum_hw, C), d.sampling_location.shape, d.weights.shape))
        ws = torch.full((ws_bytes,), 0xAB, dtype=torch.uint8, device="cuda")
        for _ in range(2):  # the second call starts from the first one's counter and gradients
            g = msda.backward(*T, d.grad_out, workspace=ws, grads=grads, warps=2)
        torch.cuda.synchronize()
        res[name] = [t.cpu() for t in g]
        assert not any(torch.isnan(t).any() for t in res[name])
        check_against_oracle(pr, res[name], TOL_FP32, f"{name} order, layout {layout}")
    assert msda.device_status() == 0
    assert torch.equal(res["ordered"][1], res["static"][1]) and torch.equal(res["ordered"][2], res["static"][2])
    if layout == "padded":
        covered = torch.zeros(sum_hw, dtype=torch.bool)
        for k in range(3):
            for s in range(3):
                st = int(pr.scale_start_index[k, s])
                covered[st:st + int(pr.spatial_shape[k, s, 0] * pr.spatial_shape[k, s, 1])] = True
        assert torch.all(res["ordered"][0][:, ~covered] == 0)


def test_atomic_orders_and_splits_agree_on_training_shape():
    """Every warp count and vector split of the ordered hand-out on the 16-camera training shape (4 batch
    elements), against the static stride."""
    pr = inputs.make_workload(3, ncam=16, batch=4, feat_dtype="bf16", w_dtype="f32")
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    ref = msda.backward(*T, d.grad_out, workspace=torch.empty(0, dtype=torch.uint8, device="cuda"))
    for warps in (1, 2, 4, 8):
        for vec in (1, 2, 4):
            g = msda.backward(*T, d.grad_out, warps=warps, vec=vec)
            e = relerr(g[0].cpu().double().numpy(), ref[0].cpu().double().numpy())
            assert e <= 1e-5, (warps, vec, e)
    assert msda.device_status() == 0


def test_side_stream_clear_then_zeroed_backward():
    """The training-step pattern: grad_feat cleared on a side stream while the forward runs, then the atomic
    backward with MSDA_FLAG_GRAD_FEAT_ZEROED; equal to a backward that clears by itself."""
    pr = inputs.make_workload(1, feat_dtype="bf16", w_dtype="bf16").anchors(range(200))
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    ref = [t.cpu() for t in msda.backward(*T, d.grad_out)]
    B, sum_hw, C = d.feat.shape
    gf = torch.full((B, sum_hw, C), float("nan"), device="cuda")
    gl, gw = torch.empty(d.sampling_location.shape, device="cuda"), torch.empty(d.weights.shape, device="cuda")
    main, side = torch.cuda.current_stream(), torch.cuda.Stream()
    side.wait_stream(main)
    with torch.cuda.stream(side):
        gf.zero_()
    msda.forward(*T)
    main.wait_stream(side)
    g = [t.cpu() for t in msda.backward(*T, d.grad_out, grads=(gf, gl, gw), grad_feat_zeroed=True)]
    assert relerr(g[0].double().numpy(), ref[0].double().numpy()) <= 1e-6
    assert torch.equal(g[1], ref[1]) and torch.equal(g[2], ref[2])
    assert msda.device_status() == 0


@pytest.mark.parametrize("case", ["tiny", "sparse4d-200", "no-anchors", "no-points", "half2"])
def test_forward_train_clears_grad_feat_and_matches_forward(case):
    """msda_forward_train: the same output as msda_forward (bitwise: same kernel and mapping) and a grad_feat of
    zeros (it starts as NaN), so that the zeroed-flag backward equals a backward that clears by itself."""
    if case == "tiny":
        pr = inputs.make_workload(0)
    elif case == "sparse4d-200":
        pr = inputs.make_workload(1, feat_dtype="bf16", w_dtype="bf16").anchors(range(200))
    elif case == "half2":
        pr = inputs.make_workload(1, feat_dtype="f16", w_dtype="f16").anchors(range(50))
    else:
        gen = torch.Generator().manual_seed(5)
        A, P = (0, 3) if case == "no-anchors" else (7, 0)
        pr = inputs.make_problem(gen, B=2, cam_maps=[[(6, 5), (3, 2)]] * 2, C=32, G=4, A=A, P=P)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    B, sum_hw, C = d.feat.shape
    variant = 3 if case == "half2" else 0
    gf = torch.full((B, sum_hw, C), float("nan"), device="cuda")
    for warps, v in ((2, variant), (8, variant), (8, 4 if variant == 0 else variant)):
        gf.fill_(float("nan"))
        got = msda.forward_train(*T, gf, warps=warps, variant=v)
        ref = msda.forward(*T, warps=warps, variant=v)
        torch.cuda.synchronize()
        assert torch.equal(got, ref), case
        assert torch.all(gf == 0), case
    if d.grad_out is not None and case in ("tiny", "sparse4d-200"):
        refg = [t.cpu() for t in msda.backward(*T, d.grad_out)]
        gl, gw = torch.empty(d.sampling_location.shape, device="cuda"), torch.empty(d.weights.shape, device="cuda")
        g = [t.cpu() for t in msda.backward(*T, d.grad_out, grads=(gf, gl, gw), grad_feat_zeroed=True)]
        assert relerr(g[0].double().numpy(), refg[0].double().numpy()) <= 1e-6
        assert torch.equal(g[1], refg[1]) and torch.equal(g[2], refg[2])
    assert msda.device_status() == 0


def test_bench_step_in_its_launch_configuration_full_size():
    """The timed step of bench.py exactly as it runs (the shipped GB300 mappings, msda_forward_train clearing
    grad_feat, then the atomic backward with the zeroed flag) on the full 64-camera frame, against the oracle."""
    import json
    import os
    from paper_2601_10819_gb300 import tune
    pr = inputs.make_workload(2)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    table = json.load(open(tune.SHIPPED))
    pick = lambda kind: next((v["best"] for k, v in table.items() if f"|{kind}|" in k and "hw694080" in k), {})
    ft, bt = pick("fwd"), pick("bwd")
    B, sum_hw, C = d.feat.shape
    gf = torch.full((B, sum_hw, C), float("nan"), device="cuda")
    gl, gw = torch.empty(d.sampling_location.shape, device="cuda"), torch.empty(d.weights.shape, device="cuda")
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    for _ in range(2):  # a second step over the first one's gradients
        out = msda.forward_train(*T, gf, warps=ft.get("warps") or None, vec=ft.get("vec", 0))
        msda.backward(*T, d.grad_out, workspace=ws, grads=(gf, gl, gw), warps=bt.get("warps") or None,
                      vec=bt.get("vec", 0), grad_feat_zeroed=True)
    torch.cuda.synchronize()
    assert relerr(out.cpu().double().numpy(), oracle_forward(pr)) <= TOL_LOWP_OUT
    ref = oracle_backward(pr)
    for g, r, name in zip((gf, gl, gw), ref, ["dfeat", "dloc", "dw"]):
        e = relerr(g.cpu().double().numpy(), r)
        print(f"bench step {name} rel err {e:.2e}")
        assert e <= TOL_LOWP_GRAD
    assert msda.device_status() == 0


@pytest.mark.parametrize("G", [4, 2])
def test_deterministic_large_anchor_takes_the_per_point_kernel(G):
    """An anchor whose point-scales do not fit the anchor-block kernel's shared memory (100 keypoints x 64 cameras
    x 4 scales) takes the per-point kernel for dloc and dw; the result still matches the oracle and is bitwise
    reproducible.  G = 2 exercises the scalar zero stores of dropped point-scales in the anchor-block kernel's
    small case below, G = 4 the 16-byte ones."""
    gen = torch.Generator().manual_seed(64 + G)
    maps = [[(6, 5), (3, 3), (2, 2), (1, 1)]] * 64
    pr = inputs.make_problem(gen, B=1, cam_maps=maps, C=32, G=G, A=3, P=100, loc_range=(-0.5, 1.5))
    a = gpu_backward(pr, True, 8)
    b = gpu_backward(pr, True, 4)
    for x, y in zip(a, b):
        assert torch.equal(x, y)
    check_against_oracle(pr, a, TOL_FP32, f"large anchor G={G}")
    small = inputs.make_problem(gen, B=1, cam_maps=maps, C=32, G=G, A=3, P=3, loc_range=(-0.5, 1.5))
    check_against_oracle(small, gpu_backward(small, True, 4), TOL_FP32, f"64 cameras, small anchor G={G}")


def test_deterministic_rows_with_thousands_of_contributions():
    """Every point falls on the same few feature rows (2x2 and 1x1 maps), so each row gathers about 1600 (or
    about 480) contributions: the per-row sort takes its rank path (more than 1024 slots) or its shared-memory
    path (257 to 1024); a medium case (tens per row) takes the register paths.  All match the oracle and are
    bitwise reproducible over launches."""
    gen = torch.Generator().manual_seed(1600)
    for maps, A in (([[(2, 2), (1, 1)]] * 2, 200), ([[(2, 2), (1, 1)]] * 2, 60), ([[(4, 4), (2, 3)]] * 3, 12)):
        pr = inputs.make_problem(gen, B=1, cam_maps=maps, C=32, G=4, A=A, P=8, loc_range=(0.0, 1.0))
        for variant in (0, 5):  # the cell-binned form and the corner-slot form with its per-row sorts
            a = gpu_backward(pr, True, 8, variant)
            b = gpu_backward(pr, True, 2, variant)
            for x, y in zip(a, b):
                assert torch.equal(x, y)
            check_against_oracle(pr, a, TOL_FP32, f"many contributions per row A={A} variant={variant}")
