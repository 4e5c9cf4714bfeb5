"""Pins of the oracle's keypoint prologue (Sec. 3.1, 3.2).

Checked against geometry that does not restate the formula: a camera whose
matrix is written by hand from its pose (golden values worked out below),
rotation and translation invariants, motion compensation equal to moving the
centre, and points behind a camera.
"""
import math

import numpy as np
import torch

from paper_2601_10819_gb300 import inputs


def one(anchor, offsets, proj, wh=(100.0, 50.0), dt=0.0, lib=None):
    an = torch.tensor([[anchor]], dtype=torch.float64)
    of = torch.tensor([[offsets]], dtype=torch.float64)
    pr = torch.tensor([proj], dtype=torch.float64)
    return lib.keypoints(an, of, torch.tensor([dt], dtype=torch.float64), pr,
                         torch.tensor([list(wh)] * pr.shape[1], dtype=torch.float64))[0, 0]


# camera at the origin looking along world +x, image x = world -y, image y = world -z,
# f = 100 px, principal point (50, 25):  pixel = (50 - 100*y/x, 25 - 100*z/x)
CAM_X = [[[50.0, -100.0, 0.0, 0.0], [25.0, 0.0, -100.0, 0.0], [1.0, 0.0, 0.0, 0.0]]]


def test_hand_worked_projection(oracle_lib):
    # box centre (10, 1, -0.5), size (2, 4, 1), yaw 0, keypoints: centre and +0.5 along box y
    anchor = [10.0, 1.0, -0.5, 2.0, 4.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    loc = one(anchor, [[0, 0, 0], [0, 0.5, 0]], CAM_X, lib=oracle_lib)
    # centre: pixel (50 - 100*1/10, 25 - 100*(-0.5)/10) = (40, 30) -> (0.4, 0.6)
    np.testing.assert_allclose(loc[0, 0], [0.4, 0.6], rtol=0, atol=1e-15)
    # +0.5 box-y at l=4: point (10, 3, -0.5): pixel (50 - 30, 25 + 5) = (20, 30) -> (0.2, 0.6)
    np.testing.assert_allclose(loc[1, 0], [0.2, 0.6], rtol=0, atol=1e-15)


def test_yaw_rotates_box_offsets(oracle_lib):
    # yaw = 90 deg maps box +x onto world +y: offset (0.5, 0, 0) with w = 2 -> world (cx, cy + 1, cz)
    a90 = [10.0, 0.0, 0.0, 2.0, 3.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0]
    moved = [10.0, 1.0, 0.0, 2.0, 3.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    got = one(a90, [[0.5, 0, 0]], CAM_X, lib=oracle_lib)
    ref = one(moved, [[0, 0, 0]], CAM_X, lib=oracle_lib)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_yaw_rotates_box_y_offsets(oracle_lib):
    # yaw = 90 deg maps box +y onto world -x: offset (0, 0.5, 0) with l = 4 -> world (cx - 2, cy, cz)
    a90 = [12.0, 0.5, 0.0, 2.0, 4.0, 1.0, 1.0, 0.0, 0.0, 0.0, 0.0]
    moved = [10.0, 0.5, 0.0, 2.0, 4.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0]
    got = one(a90, [[0, 0.5, 0]], CAM_X, lib=oracle_lib)
    ref = one(moved, [[0, 0, 0]], CAM_X, lib=oracle_lib)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-14)


def test_motion_compensation_moves_the_centre(oracle_lib):
    a = [12.0, -2.0, 1.0, 1.0, 1.0, 1.0, 0.6, 0.8, 3.0, -1.0, 0.5]
    b = [12.0 + 0.3, -2.0 - 0.1, 1.0 + 0.05, 1.0, 1.0, 1.0, 0.6, 0.8, 0.0, 0.0, 0.0]
    offs = [[0.2, -0.3, 0.1], [0, 0, 0]]
    np.testing.assert_allclose(one(a, offs, CAM_X, dt=0.1, lib=oracle_lib), one(b, offs, CAM_X, lib=oracle_lib),
                               rtol=0, atol=1e-14)


def test_points_behind_the_camera_are_marked_out(oracle_lib):
    loc = one([-5.0, 0.0, 0.0, 1.0, 1.0, 1.0, 0.0, 1.0, 0.0, 0.0, 0.0], [[0, 0, 0]], CAM_X, lib=oracle_lib)
    assert np.all(loc == -2.0)


def test_synthetic_rig_sees_the_floor(oracle_lib):
    an, of, dt, pr, wh = inputs.make_scene_geometry(0, B=1, A=50, P=13, ncam=8)
    loc = oracle_lib.keypoints(an, of, dt, pr, wh)
    inside = ((loc > 0) & (loc < 1)).all(axis=-1)
    assert inside.mean() > 0.5  # cameras on the ring look at the floor
    # scaling the whole matrix of a camera does not move its projections
    pr2 = pr.double().clone()
    pr2[:, 3] *= 7.0
    np.testing.assert_allclose(oracle_lib.keypoints(an, of, dt, pr2, wh), loc, rtol=1e-12, atol=1e-12)
