"""The algorithmic byte counts behind the roofline fractions: a case counted by hand and a brute force over every
point-scale and corner of a random ragged problem."""
import torch

from paper_2601_10819_gb300 import inputs, roofline


def _problem(shapes, loc, C, G, feat_dtype=torch.bfloat16, w_dtype=torch.float32):
    shape, start, sum_hw = inputs.tables(shapes)
    B, A, P, K, _ = loc.shape
    S = shape.shape[1]
    feat = torch.zeros(B, sum_hw, C, dtype=feat_dtype)
    w = torch.zeros(B, A, P, K, S, G, dtype=w_dtype)
    return inputs.Problem(feat, shape, start, loc, w, None)


def test_hand_counted_case():
    # one 4x4 map; C = 8 BF16 channels, G = 2 FP32 weights
    loc = torch.tensor([[[[[0.375, 0.375]], [[0.0, 0.0]], [[2.0, 0.5]]]]], dtype=torch.float32)  # [1, 1, 3, 1, 2]
    pr = _problem([[(4, 4)]], loc, C=8, G=2)
    c = roofline.count(pr)
    # point 0: x = y = 1.0, corners (1,1) (1,2) (2,1) (2,2): rows 5, 6, 9, 10
    # point 1: x = y = -0.5, only corner (0,0) is on the map: row 0
    # point 2: x = 7.5 >= W: out of view
    assert (c.nominal_samples, c.inview_samples, c.inbound_corners, c.touched_rows, c.total_rows) == (3, 2, 5, 5, 16)
    loc_b, out_b = 3 * 2 * 4, 8 * 4
    assert c.fwd_hbm_bytes == 5 * 8 * 2 + loc_b + 2 * 2 * 4 + out_b
    assert c.fwd_l2_gather_bytes == 5 * 8 * 2
    assert c.bwd_hbm_bytes == c.fwd_hbm_bytes + 16 * 8 * 4 + loc_b + 3 * 2 * 4
    assert c.bwd_l2_bytes == 5 * 8 * 2 + 5 * 8 * 4


def test_brute_force_over_a_ragged_problem():
    gen = torch.Generator().manual_seed(7)
    shapes = [[(5, 7), (3, 4), (2, 2)], [(9, 4), (4, 2), (1, 1)]]
    B, A, P, K = 2, 5, 3, 2
    loc = torch.rand(B, A, P, K, 2, generator=gen) * 1.6 - 0.3
    pr = _problem(shapes, loc, C=16, G=4)
    c = roofline.count(pr)
    shape, start = pr.spatial_shape.tolist(), pr.scale_start_index.tolist()
    sum_hw = pr.feat.shape[1]
    inview = corners = 0
    touched = set()
    for b in range(B):
        for a in range(A):
            for p in range(P):
                for k in range(K):
                    u, v = (float(t) for t in loc[b, a, p, k].double())
                    for s in range(3):
                        H, W = shape[k][s]
                        x, y = u * W - 0.5, v * H - 0.5
                        if not (-1 < x < W and -1 < y < H):
                            continue
                        inview += 1
                        x0, y0 = int(torch.floor(torch.tensor(x, dtype=torch.float64))), \
                            int(torch.floor(torch.tensor(y, dtype=torch.float64)))
                        for i in (y0, y0 + 1):
                            for j in (x0, x0 + 1):
                                if 0 <= i < H and 0 <= j < W:
                                    corners += 1
                                    touched.add((b, start[k][s] + i * W + j))
    assert c.nominal_samples == B * A * P * K * 3
    assert (c.inview_samples, c.inbound_corners, c.touched_rows, c.total_rows) == \
        (inview, corners, len(touched), B * sum_hw)
    assert c.fwd_l2_gather_bytes == corners * 16 * 2
    assert c.bwd_l2_bytes == corners * 16 * (2 + 4)
