"""The synthetic input recipe: the workload shapes, the readings of the paper's video-map sizes and of its
out-of-view fraction, seeding, and the batched-serving ranges."""
import torch

from paper_2601_10819_gb300 import inputs


def test_video_map_sizes():
    assert inputs.video_maps(1080, 1920) == [(68, 120), (34, 60), (17, 30), (9, 15)]
    assert inputs.video_maps(720, 1280) == [(45, 80), (23, 40), (12, 20), (6, 10)]


def test_tables_pack_maps_camera_major():
    shape, start, sum_hw = inputs.tables([[(2, 3), (1, 2)], [(4, 1), (1, 1)]])
    assert shape.tolist() == [[[2, 3], [1, 2]], [[4, 1], [1, 1]]]
    assert start.tolist() == [[0, 6], [8, 12]] and sum_hw == 13
    assert shape.dtype == torch.int32 and start.dtype == torch.int32


def test_outside_in_workload_shapes_and_out_of_view_pairs():
    pr = inputs.make_workload(2, ncam=8, with_grad=False)
    d = pr.dims
    assert (d["B"], d["Ncam"], d["Nscale"], d["C"], d["G"], d["A"], d["P"]) == (1, 8, 4, 256, 8, 900, 13)
    assert pr.feat.dtype == torch.bfloat16 and pr.weights.dtype == torch.bfloat16
    assert pr.spatial_shape[0].tolist() == [[68, 120], [34, 60], [17, 30], [9, 15]]
    # exactly round(0.4 * A * Ncam) (anchor, camera) pairs moved out of view, every keypoint of the pair
    mask = pr.meta["out_mask"]
    assert int(mask.sum()) == round(0.4 * 900 * 8) == pr.meta["n_out_pairs"]
    u = pr.sampling_location[..., 0]
    out_pairs = (u > 1.5).all(dim=2)
    assert torch.equal(out_pairs, mask)
    # the weights of every (anchor, group) sum to one over keypoints, cameras and scales (softmax), before
    # rounding to BF16
    s = pr.weights.double().sum(dim=(2, 3, 4))
    assert torch.allclose(s, torch.ones_like(s), atol=0.05)


def test_seeded_and_reproducible():
    a = inputs.make_workload(0)
    b = inputs.make_workload(0)
    for x, y in zip(a.tensors() + (a.grad_out,), b.tensors() + (b.grad_out,)):
        assert torch.equal(x, y)


def test_batched_serving_ranges():
    scenes = inputs.make_workload(4, batch=6, with_grad=False)
    assert len(scenes) == 6
    for pr in scenes:
        d = pr.dims
        assert 4 <= d["Ncam"] <= 96 and 600 <= d["A"] <= 1200 and (d["P"], d["C"], d["G"]) == (13, 256, 8)
        hw = pr.spatial_shape[0, 0].tolist()
        assert hw in ([68, 120], [45, 80])
