"""Pins of the oracle's visibility-weighted fusion (Sec. 3.2, Eq. 2).

f = sum_i v_i g_i / sum_i v_i, with g_i the operator restricted to camera i.
Pinned against the already-pinned plain operator: uniform visibility gives
the plain output divided by Ncam, a one-hot visibility gives camera i alone,
scaling all visibilities changes nothing, and the fusion is the weighted mean
of per-camera runs.
"""
import numpy as np
import pytest
import torch

from paper_2601_10819_gb300 import inputs

MAPS = [[(7, 9), (4, 5)], [(6, 6), (3, 3)], [(8, 5), (4, 3)]]


def problem(seed=0):
    gen = torch.Generator().manual_seed(seed)
    return inputs.make_problem(gen, B=2, cam_maps=MAPS, C=8, G=2, A=5, P=3, loc_range=(-0.2, 1.2))


def cam_only(pr, k):
    w = pr.weights.clone()
    keep = torch.zeros(w.shape[3], dtype=torch.bool)
    keep[k] = True
    w[:, :, :, ~keep] = 0
    return w


def test_uniform_visibility_is_mean_over_cameras(oracle_lib):
    pr = problem(1)
    vis = torch.full((2, 5, 3), 0.7, dtype=torch.float64)
    f = oracle_lib.forward_oae(*pr.tensors(), vis)
    plain = oracle_lib.forward(*pr.tensors())
    np.testing.assert_allclose(f, plain / 3.0, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("k", [0, 1, 2])
def test_one_hot_visibility_selects_a_camera(oracle_lib, k):
    pr = problem(2)
    vis = torch.zeros(2, 5, 3, dtype=torch.float64)
    vis[:, :, k] = 0.3
    f = oracle_lib.forward_oae(*pr.tensors(), vis)
    ref = oracle_lib.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, cam_only(pr, k))
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-14)


def test_weighted_mean_of_camera_runs_and_scale_invariance(oracle_lib):
    pr = problem(3)
    vis = torch.rand(2, 5, 3, generator=torch.Generator().manual_seed(3), dtype=torch.float64)
    f = oracle_lib.forward_oae(*pr.tensors(), vis)
    g = [oracle_lib.forward(pr.feat, pr.spatial_shape, pr.scale_start_index, pr.sampling_location, cam_only(pr, k))
         for k in range(3)]
    v = vis.numpy()
    ref = sum(v[:, :, k:k + 1] * g[k] for k in range(3)) / v.sum(axis=2, keepdims=True)
    np.testing.assert_allclose(f, ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(oracle_lib.forward_oae(*pr.tensors(), vis * 5.0), f, rtol=1e-12, atol=1e-14)


def test_zero_visibility_gives_zero(oracle_lib):
    pr = problem(4)
    vis = torch.rand(2, 5, 3, dtype=torch.float64)
    vis[1, 2] = 0.0
    f = oracle_lib.forward_oae(*pr.tensors(), vis)
    assert np.all(f[1, 2] == 0.0) and np.any(f[0, 0] != 0.0)
