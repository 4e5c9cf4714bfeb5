"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to a value the mathematics determines: a worked
example computed by hand (tests/golden), closed forms (constant map, pixel
centres, linear map, out-of-range points), an independent tent-kernel brute
force, torch's float64 ``grid_sample`` with autograd, central finite
differences and the adjoint identities.  tests/test_oracle_mutants.py shows
that plausible mistakes planted in the oracle fail these pins.
"""
import json
import os

import numpy as np
import pytest
import torch

from paper_2601_10819_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


def small_problem(seed, cam_maps, C=8, G=2, A=3, P=4, loc_range=(-0.3, 1.3), out_frac=0.0):
    gen = torch.Generator().manual_seed(seed)
    return inputs.make_problem(gen, B=2, cam_maps=cam_maps, C=C, G=G, A=A, P=P,
                               loc_range=loc_range, out_frac=out_frac)


HETERO = [[(5, 7), (3, 4)], [(4, 4), (2, 2)], [(6, 3), (1, 5)]]   # uneven cameras, ragged sizes


def np_(t):
    return t.detach().double().numpy()


# --------------------------------------------------------------------------------------
# 1. Worked example computed by hand
# --------------------------------------------------------------------------------------
def test_hand_worked_example(oracle_lib):
    d = json.load(open(os.path.join(HERE, "golden", "hand_worked_example.json")))
    args = (np.array(d["feat"], float), np.array(d["spatial_shape"]), np.array(d["scale_start_index"]),
            np.array(d["sampling_location"], float), np.array(d["weights"], float))
    out = oracle_lib.forward(*args)
    np.testing.assert_array_equal(out, np.array(d["out"]))
    gf, gl, gw = oracle_lib.backward(*args, np.array(d["grad_out"], float))
    np.testing.assert_array_equal(gw, np.array(d["grad_weights"]))
    np.testing.assert_array_equal(gf, np.array(d["grad_feat"]))
    np.testing.assert_array_equal(gl, np.array(d["grad_sampling_location"]))


# --------------------------------------------------------------------------------------
# 2. Closed forms
# --------------------------------------------------------------------------------------
def test_constant_map_interior(oracle_lib):
    """f == gamma_c everywhere and every point inside all maps: out_c = gamma_c * sum(w_g)."""
    pr = small_problem(1, [[(16, 16), (8, 8)]] * 2, C=8, G=4, loc_range=(0.07, 0.93))
    gamma = torch.linspace(-2.0, 3.0, 8, dtype=torch.float64)
    feat = gamma.expand(pr.feat.shape).clone()
    out = oracle_lib.forward(feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, pr.weights)
    wsum = np_(pr.weights).sum(axis=(2, 3, 4))                # [B, A, G]
    expect = np.repeat(wsum, 2, axis=-1) * gamma.numpy()    # Cg = 2
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-13)


def tent_mass(x, n):
    """Mass of the unit tent centred at x that falls on pixels 0..n-1 (closed form)."""
    if x <= -1 or x >= n:
        return 0.0
    if x < 0:
        return 1.0 + x
    if x > n - 1:
        return float(n) - x
    return 1.0


def test_constant_map_boundary(oracle_lib):
    """Near and beyond the borders a constant map returns gamma times the in-map tent mass."""
    pr = small_problem(2, HETERO, C=4, G=1, loc_range=(-0.4, 1.4))
    feat = torch.full(pr.feat.shape, 1.5, dtype=torch.float64)
    out = oracle_lib.forward(feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, pr.weights)
    loc, w, shp = np_(pr.sampling_location), np_(pr.weights), pr.spatial_shape.numpy()
    B, A, P, K, S, G = w.shape
    expect = np.zeros((B, A))
    for b in range(B):
        for a in range(A):
            for p in range(P):
                for k in range(K):
                    for s in range(S):
                        H, W = shp[k, s]
                        u, v = loc[b, a, p, k]
                        expect[b, a] += w[b, a, p, k, s, 0] * tent_mass(u * W - 0.5, W) * tent_mass(v * H - 0.5, H)
    np.testing.assert_allclose(out[..., 0], 1.5 * expect, rtol=1e-12, atol=1e-14)


def test_pixel_centres_return_pixels(oracle_lib):
    """u = (j+0.5)/W, v = (i+0.5)/H samples exactly feature row (i, j)."""
    gen = torch.Generator().manual_seed(3)
    maps = [[(5, 7)], [(4, 4)], [(3, 11)]]
    pr = inputs.make_problem(gen, B=1, cam_maps=maps, C=6, G=3, A=4, P=5)
    shp, start = pr.spatial_shape.numpy(), pr.scale_start_index.numpy()
    loc = np.zeros(pr.sampling_location.shape)
    feat = np_(pr.feat)
    w = np_(pr.weights)
    expect = np.zeros((1, 4, 6))
    rng = np.random.default_rng(3)
    for a in range(4):
        for p in range(5):
            for k in range(3):
                H, W = shp[k, 0]
                i, j = rng.integers(0, H), rng.integers(0, W)
                loc[0, a, p, k] = [(j + 0.5) / W, (i + 0.5) / H]
                row = start[k, 0] + i * W + j
                expect[0, a] += np.repeat(w[0, a, p, k, 0], 2) * feat[0, row]
    out = oracle_lib.forward(feat, pr.spatial_shape, pr.scale_start_index, loc, w)
    np.testing.assert_allclose(out, expect, rtol=1e-13, atol=1e-14)


def test_linear_map_reproduced(oracle_lib):
    """f(i, j) = alpha*j + beta*i + gamma is reproduced exactly at interior points,
    with x = u*W - 0.5 and y = v*H - 0.5 (pixel centres at (j+0.5)/W)."""
    pr = small_problem(4, [[(9, 13), (5, 6)], [(7, 7), (4, 3)]], C=4, G=2, loc_range=(0.0, 1.0))
    shp, start = pr.spatial_shape.numpy(), pr.scale_start_index.numpy()
    rng = np.random.default_rng(4)
    K, S = shp.shape[:2]
    coef = rng.normal(size=(K, S, 3, 4))  # alpha, beta, gamma per channel
    feat = np.zeros(pr.feat.shape)
    for k in range(K):
        for s in range(S):
            H, W = shp[k, s]
            i, j = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
            rows = start[k, s] + (i * W + j).ravel()
            for b in range(feat.shape[0]):
                feat[b, rows] = (coef[k, s, 0] * j.ravel()[:, None] + coef[k, s, 1] * i.ravel()[:, None]
                                 + coef[k, s, 2])
    # keep every point inside [0, W-1] x [0, H-1] at every scale
    lo = np.max(0.5 / shp, axis=(0, 1))
    loc = np_(pr.sampling_location)
    loc = lo[::-1] + (1 - 2 * lo[::-1]) * np.clip(loc, 0, 1)
    w = np_(pr.weights)
    out = oracle_lib.forward(feat, pr.spatial_shape, pr.scale_start_index, loc, w)
    B, A, P = loc.shape[:3]
    expect = np.zeros_like(out)
    for b in range(B):
        for a in range(A):
            for p in range(P):
                for k in range(K):
                    for s in range(S):
                        H, W = shp[k, s]
                        x = loc[b, a, p, k, 0] * W - 0.5
                        y = loc[b, a, p, k, 1] * H - 0.5
                        val = coef[k, s, 0] * x + coef[k, s, 1] * y + coef[k, s, 2]
                        expect[b, a] += np.repeat(w[b, a, p, k, s], 2) * val
    np.testing.assert_allclose(out, expect, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("u,v", [(2.0, 0.5), (2.9, 0.1), (-0.2, 0.5), (0.5, -0.3), (0.5, 1.2),
                                 (float("nan"), 0.5), (0.5, float("inf")), (-1.0 / 32, 0.5)])
def test_out_of_range_points_are_zero(oracle_lib, u, v):
    """A point whose tent misses every pixel contributes 0, and has zero gradients.
    (-1/32 on a 16-wide map gives x = -1 exactly, the first dropped position.)"""
    pr = small_problem(5, [[(16, 16), (16, 16)]], C=4, G=2, A=1, P=1)
    loc = torch.tensor([[[[[u, v]]]]], dtype=torch.float64).expand(2, 1, 1, 1, 2).clone()
    out = oracle_lib.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, loc, pr.weights)
    assert np.all(out == 0.0)
    gf, gl, gw = oracle_lib.backward(pr.feat, pr.spatial_shape, pr.scale_start_index, loc, pr.weights,
                                     pr.grad_out)
    assert np.all(gf == 0.0) and np.all(gl == 0.0) and np.all(gw == 0.0)


# --------------------------------------------------------------------------------------
# 3. Independent formulations
# --------------------------------------------------------------------------------------
def brute_force_tent(feat, shape, start, loc, w):
    """S(x, y) = sum_ij max(0, 1-|x-j|) max(0, 1-|y-i|) F(i, j) over all pixels."""
    B, _, C = feat.shape
    _, A, P, K, _ = loc.shape
    S_, G = w.shape[4], w.shape[5]
    Cg = C // G
    out = np.zeros((B, A, C))
    for k in range(K):
        for s in range(S_):
            H, W = shape[k, s]
            fm = feat[:, start[k, s]:start[k, s] + H * W].reshape(B, H, W, C)
            x = loc[..., k, 0] * W - 0.5        # [B, A, P]
            y = loc[..., k, 1] * H - 0.5
            tx = np.maximum(0, 1 - np.abs(x[..., None] - np.arange(W)))  # [B,A,P,W]
            ty = np.maximum(0, 1 - np.abs(y[..., None] - np.arange(H)))  # [B,A,P,H]
            samp = np.einsum("bapi,bapj,bijc->bapc", ty, tx, fm)
            wc = np.repeat(w[:, :, :, k, s, :], Cg, axis=-1)          # [B,A,P,C]
            out += (wc * samp).sum(axis=2)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_brute_force_tent_kernel(oracle_lib, seed):
    pr = small_problem(10 + seed, HETERO, C=8, G=4, A=5, P=3, loc_range=(-0.3, 1.3))
    args = [np_(pr.feat), pr.spatial_shape.numpy(), pr.scale_start_index.numpy(),
            np_(pr.sampling_location), np_(pr.weights)]
    out = oracle_lib.forward(*args)
    np.testing.assert_allclose(out, brute_force_tent(*args), rtol=1e-12, atol=1e-13)


def grid_sample_composite(feat, shape, start, loc, w):
    """The operator as a weighted sum of torch grid_sample calls (float64 CPU)."""
    B, _, C = feat.shape
    _, A, P, K, _ = loc.shape
    S_, G = w.shape[4], w.shape[5]
    Cg = C // G
    out = torch.zeros(B, A, C, dtype=torch.float64)
    for k in range(K):
        for s in range(S_):
            H, W = int(shape[k, s, 0]), int(shape[k, s, 1])
            st = int(start[k, s])
            fm = feat[:, st:st + H * W].reshape(B, H, W, C).permute(0, 3, 1, 2)  # [B,C,H,W]
            grid = (2 * loc[:, :, :, k, :] - 1).reshape(B, A * P, 1, 2)
            samp = torch.nn.functional.grid_sample(fm, grid, mode="bilinear", padding_mode="zeros",
                                                   align_corners=False)           # [B,C,A*P,1]
            samp = samp[..., 0].permute(0, 2, 1).reshape(B, A, P, C)
            wc = w[:, :, :, k, s, :].repeat_interleave(Cg, dim=-1)
            out = out + (wc * samp).sum(dim=2)
    return out


@pytest.mark.parametrize("seed", [0, 1])
def test_grid_sample_forward_and_autograd(oracle_lib, seed):
    pr = small_problem(20 + seed, HETERO, C=8, G=2, A=4, P=3, loc_range=(-0.2, 1.2))
    feat = pr.feat.double().requires_grad_()
    loc = pr.sampling_location.double().requires_grad_()
    w = pr.weights.double().requires_grad_()
    ref = grid_sample_composite(feat, pr.spatial_shape, pr.scale_start_index, loc, w)
    go = pr.grad_out.double()
    ref.backward(go)
    out = oracle_lib.forward(feat, pr.spatial_shape, pr.scale_start_index, loc, w)
    np.testing.assert_allclose(out, ref.detach().numpy(), rtol=1e-12, atol=1e-13)
    gf, gl, gw = oracle_lib.backward(feat, pr.spatial_shape, pr.scale_start_index, loc, w, go)
    np.testing.assert_allclose(gf, feat.grad.numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(gw, w.grad.numpy(), rtol=1e-12, atol=1e-13)
    np.testing.assert_allclose(gl, loc.grad.numpy(), rtol=1e-10, atol=1e-11)


def test_grid_sample_camera_packing_any_order(oracle_lib):
    """Cameras packed in reverse order (start offsets permuted) give the same result."""
    pr = small_problem(30, HETERO, C=4, G=2, A=3, P=2)
    out = oracle_lib.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, pr.weights)
    shp = pr.spatial_shape.numpy()
    K, S = shp.shape[:2]
    new_start = np.zeros((K, S), np.int32)
    off = 0
    order = [(k, s) for k in reversed(range(K)) for s in reversed(range(S))]
    feat_new = torch.zeros_like(pr.feat)
    for k, s in order:
        n = int(shp[k, s, 0] * shp[k, s, 1])
        new_start[k, s] = off
        st = int(pr.scale_start_index[k, s])
        feat_new[:, off:off + n] = pr.feat[:, st:st + n]
        off += n
    out2 = oracle_lib.forward(feat_new, pr.spatial_shape, new_start, pr.sampling_location, pr.weights)
    np.testing.assert_array_equal(out, out2)


# --------------------------------------------------------------------------------------
# 4. Finite differences and adjoints
# --------------------------------------------------------------------------------------
def test_finite_differences_location(oracle_lib):
    pr = small_problem(40, HETERO, C=8, G=4, A=3, P=3, loc_range=(-0.1, 1.1))
    feat, loc, w = np_(pr.feat), np_(pr.sampling_location), np_(pr.weights)
    shp, start = pr.spatial_shape.numpy(), pr.scale_start_index.numpy()
    go = np_(pr.grad_out)
    _, gl, _ = oracle_lib.backward(feat, shp, start, loc, w, go)
    h = 1e-6
    B, A, P, K, _ = loc.shape
    checked = 0
    for b in range(B):
        for a in range(A):
            for p in range(P):
                for k in range(K):
                    # reject points within 1e-3 px of a grid line or the drop border at any scale
                    near = False
                    for s in range(shp.shape[1]):
                        H, W = shp[k, s]
                        for coord in (loc[b, a, p, k, 0] * W - 0.5, loc[b, a, p, k, 1] * H - 0.5):
                            if abs(coord - np.round(coord)) < 1e-3:
                                near = True
                    if near:
                        continue
                    for d in range(2):
                        lp, lm = loc.copy(), loc.copy()
                        lp[b, a, p, k, d] += h
                        lm[b, a, p, k, d] -= h
                        fd = ((oracle_lib.forward(feat, shp, start, lp, w) -
                               oracle_lib.forward(feat, shp, start, lm, w)) * go).sum() / (2 * h)
                        assert abs(fd - gl[b, a, p, k, d]) <= 1e-6 * max(1.0, abs(fd)), (b, a, p, k, d)
                        checked += 1
    assert checked > 40


def test_finite_differences_feat_and_weights(oracle_lib):
    pr = small_problem(41, HETERO, C=4, G=2, A=2, P=3)
    feat, loc, w = np_(pr.feat), np_(pr.sampling_location), np_(pr.weights)
    shp, start = pr.spatial_shape.numpy(), pr.scale_start_index.numpy()
    go = np_(pr.grad_out)
    gf, _, gw = oracle_lib.backward(feat, shp, start, loc, w, go)
    rng = np.random.default_rng(41)
    h = 1e-5
    for _ in range(25):
        idx = tuple(rng.integers(0, n) for n in feat.shape)
        fp, fm = feat.copy(), feat.copy()
        fp[idx] += h
        fm[idx] -= h
        fd = ((oracle_lib.forward(fp, shp, start, loc, w) - oracle_lib.forward(fm, shp, start, loc, w)) * go).sum() / (2 * h)
        assert abs(fd - gf[idx]) < 1e-8
    for _ in range(25):
        idx = tuple(rng.integers(0, n) for n in w.shape)
        wp, wm = w.copy(), w.copy()
        wp[idx] += h
        wm[idx] -= h
        fd = ((oracle_lib.forward(feat, shp, start, loc, wp) - oracle_lib.forward(feat, shp, start, loc, wm)) * go).sum() / (2 * h)
        assert abs(fd - gw[idx]) < 1e-8


def test_adjoint_identities(oracle_lib):
    """out is linear in feat and in w: <go, out> = <dfeat, feat> = <dw, w>."""
    pr = small_problem(42, HETERO, C=8, G=4, A=6, P=5, loc_range=(-0.2, 1.2))
    args = (np_(pr.feat), pr.spatial_shape.numpy(), pr.scale_start_index.numpy(),
            np_(pr.sampling_location), np_(pr.weights))
    out = oracle_lib.forward(*args)
    go = np_(pr.grad_out)
    gf, _, gw = oracle_lib.backward(*args, go)
    lhs = (go * out).sum()
    assert abs(lhs - (gf * args[0]).sum()) < 1e-12 * max(1, abs(lhs))
    assert abs(lhs - (gw * args[4]).sum()) < 1e-12 * max(1, abs(lhs))


def test_thread_count_does_not_change_forward(oracle_lib):
    pr = inputs.make_workload(1, ncam=None).anchors(range(40))
    o1 = oracle_lib.forward(*pr.tensors(), nthreads=1)
    o4 = oracle_lib.forward(*pr.tensors(), nthreads=4)
    np.testing.assert_array_equal(o1, o4)


def test_bad_arguments_rejected(oracle_lib):
    pr = small_problem(43, HETERO, C=8, G=4)
    start = pr.scale_start_index.clone()
    start[0, 0] = pr.feat.shape[1]  # map runs past sum_hw
    with pytest.raises(ValueError):
        oracle_lib.forward(pr.feat, pr.spatial_shape, start, pr.sampling_location, pr.weights)
