"""The cell-binned deterministic feature gradient against the FP64 oracle and the corner-slot form.

The deterministic backward takes the cell-binned path (each map's points binned by bilinear cell, every
feature row summed over its four cells' bins with grad_out staged per channel group) whenever the maps are
disjoint and the sizes fit; the first int of its workspace is the plan's flag, 1 when that path ran.
tuning variant 5 forces the corner-slot path on the same inputs.
"""
import random

import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_FP32, TOL_LOWP_GRAD, ensure_lib, is_lowp, oracle_backward, relerr
from paper_2601_10819_gb300 import inputs, msda

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    oracle.build()
    return ensure_lib()


def run(pr, variant=0, warps=None):
    """Deterministic backward with an explicit workspace; returns the gradients and the plan flag."""
    d = pr.to("cuda")
    B, sum_hw, C = d.feat.shape
    _, A, P, K, _ = d.sampling_location.shape
    S, G = d.weights.shape[4], d.weights.shape[5]
    need = msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, True)
    ws = torch.full((max(need, 16),), 0x7f, dtype=torch.uint8, device="cuda")
    g = msda.backward(d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights, d.grad_out,
                      deterministic=True, workspace=ws, warps=warps, variant=variant)
    torch.cuda.synchronize()
    flag = int(ws[:4].view(torch.int32).item())
    return [t.cpu() for t in g], flag


def check(pr, label, expect_cells=True):
    tol = TOL_LOWP_GRAD if is_lowp(pr) else TOL_FP32
    ref = oracle_backward(pr)
    a, fa = run(pr)
    b, _ = run(pr)
    c, _ = run(pr, variant=5)
    if expect_cells:
        assert fa == 1, f"{label}: the cell-binned path did not run"
    for x, y in zip(a, b):
        assert torch.equal(x, y), f"{label}: not bitwise reproducible"
    errs = [relerr(x.double().numpy(), r) for x, r in zip(a, ref)]
    print(f"{label}: cells={fa} rel err dfeat {errs[0]:.2e} dloc {errs[1]:.2e} dw {errs[2]:.2e}")
    assert max(errs) <= tol, errs
    # the corner-slot form computes the same sums in another order
    assert relerr(a[0].double().numpy(), c[0].double().numpy()) <= tol
    return a, fa


HETERO = [[(5, 7), (3, 4), (2, 2)], [(9, 4), (4, 2), (1, 1)], [(6, 13), (3, 7), (2, 3)]]


@pytest.mark.parametrize("C,G,fdt", [(32, 4, "f32"), (64, 4, "f32"), (64, 8, "bf16"), (128, 2, "bf16"),
                                     (256, 2, "f32"), (256, 32, "bf16"), (512, 8, "bf16"), (128, 32, "f32")])
def test_channel_groups_and_ragged_maps(C, G, fdt):
    """Every lane-group width (C/G / 4 = 1 .. 32 lanes), points around and across map borders, B = 2."""
    gen = torch.Generator().manual_seed(C * 5 + G)
    pr = inputs.make_problem(gen, B=2, cam_maps=HETERO, C=C, G=G, A=37, P=5, loc_range=(-0.3, 1.3),
                             feat_dtype=fdt, w_dtype=fdt)
    check(pr, f"ragged C={C} G={G} {fdt}")


def test_tiny_and_fp16_weights():
    check(inputs.make_workload(0), "tiny")
    gen = torch.Generator().manual_seed(11)
    pr = inputs.make_problem(gen, B=1, cam_maps=HETERO, C=64, G=4, A=20, P=4, loc_range=(-0.2, 1.2),
                             feat_dtype="f16", w_dtype="f16")
    check(pr, "fp16")


def test_heavy_rows_take_whole_warps():
    """Tiny maps under many points: every row gathers hundreds of contributions (a warp sweeps a column), and
    cells of 17 to 256 points take the warp sorts."""
    gen = torch.Generator().manual_seed(1601)
    for maps, A in (([[(2, 2), (1, 1)]] * 2, 60), ([[(4, 4), (2, 3)]] * 3, 40), ([[(9, 15), (5, 8)]] * 2, 300)):
        pr = inputs.make_problem(gen, B=1, cam_maps=maps, C=32, G=4, A=A, P=8, loc_range=(0.0, 1.0))
        check(pr, f"heavy maps {maps[0]} A={A}")


def test_few_cells_under_hundreds_of_points():
    """About 400 points in each cell of a 1x1 map: maps of few cells place their points stably (per-warp
    cursors, no per-cell sort), so any number of points per cell stays on the cell-binned path."""
    gen = torch.Generator().manual_seed(1602)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(2, 2), (1, 1)]] * 2, C=32, G=4, A=200, P=8, loc_range=(0.0, 1.0))
    check(pr, "hundreds of points per cell")


def test_dense_coarse_map_reads_its_bands_in_place():
    """3600 points in a 2x3 map with 900 anchors' grad_out staged: the records of one image row (two cell rows,
    about 2400) exceed a band buffer, so that band is swept from the workspace in place, not staged."""
    gen = torch.Generator().manual_seed(1604)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(2, 3), (1, 2)]], C=256, G=8, A=900, P=4, loc_range=(0.0, 1.0),
                             feat_dtype="bf16", w_dtype="bf16")
    check(pr, "dense coarse map, bands in place")


def test_overfull_cell_of_a_large_map_takes_the_corner_slot_form():
    """A map of many cells (sorted per cell after an atomic placement) with 320 points in one cell: more than a
    binning block sorts, so the plan's flag is cleared and the corner-slot form computes the gradient."""
    gen = torch.Generator().manual_seed(1603)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(100, 100)]], C=32, G=4, A=40, P=8, loc_range=(0.0, 1.0))
    loc = pr.sampling_location.clone()
    loc.fill_(0.5051)  # one bilinear cell
    loc += (torch.rand(loc.shape, generator=gen) - 0.5) * 2e-5
    one = inputs.Problem(pr.feat, pr.spatial_shape, pr.scale_start_index, loc.contiguous(), pr.weights,
                         pr.grad_out)
    _, flag = check(one, "overfull cell", expect_cells=False)
    assert flag == 0


def test_sparse4d_subset_and_batches():
    check(inputs.make_workload(1).anchors(range(150)), "sparse4d fp32 subset")
    check(inputs.make_workload(3, batch=3, ncam=4).anchors(range(90)), "train-16cam B=3, 4 cameras, bf16")


def test_uncovered_rows_are_zero():
    gen = torch.Generator().manual_seed(3)
    pr = inputs.make_problem(gen, B=2, cam_maps=[[(6, 5), (3, 2)], [(4, 4), (2, 2)]], C=32, G=4, A=7, P=3)
    pad = 9
    feat = torch.cat([torch.randn(2, 5, 32), pr.feat, torch.randn(2, pad, 32)], dim=1)  # rows before and after
    start = pr.scale_start_index + 5
    gap = inputs.Problem(feat.contiguous(), pr.spatial_shape, start.contiguous(), pr.sampling_location,
                         pr.weights, pr.grad_out)
    (gf, _, _), _ = check(gap, "rows outside every map")
    assert torch.all(gf[:, :5] == 0) and torch.all(gf[:, -pad:] == 0)
    assert msda.device_status() == 0


def test_overlapping_maps_take_the_corner_slot_form():
    gen = torch.Generator().manual_seed(4)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(6, 5), (3, 2)], [(4, 4), (2, 2)]], C=32, G=4, A=9, P=3)
    start = pr.scale_start_index.clone()
    start[1, 0] = 2  # camera 1 scale 0 overlaps camera 0
    ov = inputs.Problem(pr.feat, pr.spatial_shape, start, pr.sampling_location, pr.weights, pr.grad_out)
    _, flag = check(ov, "overlapping maps", expect_cells=False)
    assert flag == 0
    assert msda.device_status() == 0


def test_invalid_map_is_skipped_like_the_corner_slot_form():
    gen = torch.Generator().manual_seed(5)
    pr = inputs.make_problem(gen, B=1, cam_maps=HETERO, C=32, G=4, A=11, P=3, loc_range=(-0.2, 1.2))
    shape = pr.spatial_shape.clone()
    shape[1, 0, 0] = 1000  # map (1, 0) runs past the end of feat
    bad = inputs.Problem(pr.feat, shape, pr.scale_start_index, pr.sampling_location, pr.weights, pr.grad_out)
    msda.device_status()
    a, fa = run(bad)
    assert msda.device_status() == 5
    c, _ = run(bad, variant=5)
    assert msda.device_status() == 5
    assert fa == 1
    for x, y in zip(a, c):
        assert relerr(x.double().numpy(), y.double().numpy()) <= TOL_FP32


def test_too_many_points_per_camera_take_the_corner_slot_form():
    """A * P above 65535 (16-bit point indices of the binning block): the corner-slot form, no plan."""
    gen = torch.Generator().manual_seed(6)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(4, 4), (2, 2)]], C=32, G=4, A=4100, P=16)
    g, _ = run(pr)
    ref = oracle_backward(pr)
    errs = [relerr(x.double().numpy(), r) for x, r in zip(g, ref)]
    assert max(errs) <= TOL_FP32, errs


def test_train_16cam_full_size_takes_the_cells():
    """The 16-camera B = 4 batch at full size: its 8x22 maps hold about 11 000 points per camera (bands in place),
    the cell-binned path runs for the whole call and agrees with the corner-slot form (the per-frame oracle
    comparison of both is in test_gpu_backward)."""
    pr = inputs.make_workload(3)
    (gf, gl, gw), flag = run(pr)
    assert flag == 1
    (cf, cl, cw), _ = run(pr, variant=5)
    for name, x, y in (("dfeat", gf, cf), ("dloc", gl, cl), ("dw", gw, cw)):
        e = relerr(x.double().numpy(), y.double().numpy())
        print(f"train-16cam cells vs corner-slot {name} rel diff {e:.2e}")
        assert e <= TOL_FP32


def test_outside_in_64cam_full_size_cells_against_oracle():
    """The benchmark frame at full size: the cell-binned path runs and matches the oracle element-wise."""
    pr = inputs.make_workload(2)
    (gf, gl, gw), flag = run(pr)
    assert flag == 1
    rf, rl, rw = oracle_backward(pr)
    for name, x, r in (("dfeat", gf, rf), ("dloc", gl, rl), ("dw", gw, rw)):
        e = relerr(x.double().numpy(), r)
        print(f"outside-in-64cam cells {name} rel err {e:.2e}")
        assert e <= TOL_LOWP_GRAD


@pytest.mark.parametrize("seed", range(24))
def test_random_problems(seed):
    """Seeded random problems: 1-5 cameras of 1-4 maps of 1..40 x 1..40 pixels each, several channel groupings and
    dtype pairs, 1-200 anchors of 1-8 keypoints, B = 1..3, location ranges from narrow (dense cells, heavy maps)
    to wide (points across and beyond the borders), some pairs out of view. Whichever deterministic form runs (the
    cell-binned one, unless a check sends the call to the corner-slot one), it must match the oracle, the other
    form and itself, bitwise."""
    rng = random.Random(seed)
    gen = torch.Generator().manual_seed(10_000 + seed)
    ncam, nscale = rng.randint(1, 5), rng.randint(1, 4)
    maps = [[(rng.randint(1, 40), rng.randint(1, 40)) for _ in range(nscale)] for _ in range(ncam)]
    C, G, fdt = rng.choice([(32, 4, "f32"), (64, 8, "bf16"), (128, 4, "bf16"), (256, 8, "bf16"), (64, 2, "f32"),
                            (256, 8, "f16")])
    wdt = fdt if rng.random() < 0.7 else "f32"
    lo = rng.uniform(-0.3, 0.6)
    hi = max(lo + rng.choice([rng.uniform(0.02, 0.2), rng.uniform(0.5, 1.6)]), 0.05)
    pr = inputs.make_problem(gen, B=rng.randint(1, 3), cam_maps=maps, C=C, G=G, A=rng.randint(1, 200),
                             P=rng.randint(1, 8), loc_range=(lo, hi), out_frac=rng.choice([0.0, 0.0, 0.3]),
                             feat_dtype=fdt, w_dtype=wdt)
    check(pr, f"random {seed}: {ncam}x{nscale} maps, C={C} G={G} {fdt}/{wdt}, loc ({lo:.2f}, {hi:.2f})",
          expect_cells=False)


def _overlapping(pr):
    start = pr.scale_start_index.clone()
    start[1, 0] = 2  # camera 1 scale 0 overlaps camera 0: the plan clears its flag
    return inputs.Problem(pr.feat, pr.spatial_shape, start, pr.sampling_location, pr.weights, pr.grad_out)


@pytest.mark.parametrize("overlap", [False, True])
def test_deterministic_backward_replayed_from_a_cuda_graph(overlap):
    """The deterministic backward captured in a CUDA graph and replayed gives the eager gradients bitwise: on the
    cell-binned path, and, with overlapping maps, on the corner-slot form that the path's launcher issues from the
    device after reading the plan's flag."""
    gen = torch.Generator().manual_seed(7)
    pr = inputs.make_problem(gen, B=1, cam_maps=[[(6, 5), (3, 2)], [(4, 4), (2, 2)]], C=32, G=4, A=9, P=3)
    if overlap:
        pr = _overlapping(pr)
    d = pr.to("cuda")
    T = (d.feat, d.spatial_shape, d.scale_start_index, d.sampling_location, d.weights)
    B, sum_hw, C = d.feat.shape
    _, A, P, K, _ = d.sampling_location.shape
    S, G = d.weights.shape[4], d.weights.shape[5]
    ws = torch.empty(msda.backward_workspace_size(B, sum_hw, C, K, S, A, P, G, True), dtype=torch.uint8,
                     device="cuda")
    grads = (torch.empty(B, sum_hw, C, device="cuda"), torch.empty(B, A, P, K, 2, device="cuda"),
             torch.empty(B, A, P, K, S, G, device="cuda"))
    msda.backward(*T, d.grad_out, deterministic=True, workspace=ws, grads=grads)  # eager, outside capture
    torch.cuda.synchronize()
    ref = [x.clone() for x in grads]
    assert int(ws[:4].view(torch.int32).item()) == (0 if overlap else 1)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            msda.backward(*T, d.grad_out, deterministic=True, workspace=ws, grads=grads)
    for _ in range(3):
        for x in grads:
            x.fill_(float("nan"))
        g.replay()
        torch.cuda.synchronize()
        for x, r in zip(grads, ref):
            assert torch.equal(x, r)
    assert msda.device_status() == 0
    rf = oracle_backward(pr)
    for x, r in zip(grads, rf):
        assert relerr(x.cpu().double().numpy(), r) <= TOL_FP32
