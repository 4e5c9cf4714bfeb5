"""Planted mistakes in the oracle must fail its pins.

Each mutant is a copy of oracle/msda_oracle.c with one plausible mistake
(a dropped term, a wrong sign, index or operand, an off-by-one), compiled on
the CPU into a temporary library.  The pins of tests/test_oracle_pins.py are
then run against it; at least one must fail.  Nothing here touches a GPU.
"""
import importlib.util
import multiprocessing
import os
import types
from functools import partial

import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(os.path.dirname(HERE), "oracle", "msda_oracle.c")

_spec = importlib.util.spec_from_file_location("_oracle_pins", os.path.join(HERE, "test_oracle_pins.py"))
pins = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(pins)
_spec2 = importlib.util.spec_from_file_location("_oracle_oae_pins", os.path.join(HERE, "test_oracle_oae_pins.py"))
oae_pins = importlib.util.module_from_spec(_spec2)
_spec2.loader.exec_module(oae_pins)
_spec3 = importlib.util.spec_from_file_location("_oracle_kp_pins", os.path.join(HERE, "test_oracle_keypoint_pins.py"))
kp_pins = importlib.util.module_from_spec(_spec3)
_spec3.loader.exec_module(kp_pins)

MUTANTS = {
    "no_half_pixel_shift": ("double x = u * (double)W - 0.5;", "double x = u * (double)W;"),
    "x_uses_height": ("double x = u * (double)W - 0.5;   /* R1 */\n    double y = v * (double)H - 0.5;",
                      "double x = u * (double)H - 0.5;   /* R1 */\n    double y = v * (double)W - 0.5;"),
    "truncate_not_floor": ("double xf = floor(x), yf = floor(y);",
                           "double xf = (double)(long)x, yf = (double)(long)y;"),
    "corner_weights_swapped": ("double wx = dx ? c.fx : 1.0 - c.fx;", "double wx = dx ? 1.0 - c.fx : c.fx;"),
    "row_index_transposed": ("row0 + i * (long)W + j", "row0 + j * (long)H + i"),
    "group_interleaved": ("o[c] += wg[c / Cg] * cr.omega[q] * f[c];", "o[c] += wg[c % G] * cr.omega[q] * f[c];"),
    "corner_dropped": ("for (int q = 0; q < 4; ++q) {\n                        if (!cr.valid[q]) continue;\n"
                       "                        const double* f = feat + cr.row[q] * (long)C;\n"
                       "                        for (int c = 0; c < C; ++c)\n",
                       "for (int q = 0; q < 3; ++q) {\n                        if (!cr.valid[q]) continue;\n"
                       "                        const double* f = feat + cr.row[q] * (long)C;\n"
                       "                        for (int c = 0; c < C; ++c)\n"),
    "keypoint_yaw_sign": ("q[0] = cy * bx - sy * by + an[0] + an[8] * dt[b];", "q[0] = cy * bx + sy * by + an[0] + an[8] * dt[b];"),
    "keypoint_no_motion": ("q[2] = bz + an[2] + an[10] * dt[b];", "q[2] = bz + an[2];"),
    "fusion_not_normalised": ("        for (int c = 0; c < C; ++c) o[c] /= vsum;", "        for (int c = 0; c < C; ++c) o[c] /= 1.0;"),
    "fusion_wrong_camera_visibility": ("const double vk = vis[ba * Ncam + k];", "const double vk = vis[ba * Ncam + (k + 1) % Ncam];"),
    "fusion_corner_dropped": ("for (int c = 0; c < C; ++c) g[c] += wg[c / Cg] * cr.omega[q] * f[c];",
                              "for (int c = 0; c < C; ++c) g[c] += (q == 3 ? 0.0 : 1.0) * wg[c / Cg] * cr.omega[q] * f[c];"),
    "bounds_off_by_one": ("j >= 0 && j < W", "j >= 0 && j <= W"),
    "drop_border_too_tight": ("x > -1.0 && x < (double)W", "x > -0.5 && x < (double)W"),
    "du_sign": ("((1.0 - fy) * (F[1] - F[0]) + fy * (F[3] - F[2]))", "((1.0 - fy) * (F[0] - F[1]) + fy * (F[3] - F[2]))"),
    "dv_missing_scale": ("dv += (double)H * wg[g]", "dv += wg[g]"),
    "du_wrong_fraction": ("((1.0 - fy) * (F[1] - F[0]) + fy * (F[3] - F[2]))", "((1.0 - fx) * (F[1] - F[0]) + fx * (F[3] - F[2]))"),
    "dfeat_missing_omega": ("grad_feat[cr.row[q] * (long)C + c] += wg[g] * cr.omega[q] * go[c];",
                            "grad_feat[cr.row[q] * (long)C + c] += wg[g] * go[c];"),
    "dw_missing_grad": ("dwg[g] += go[c] * S;", "dwg[g] += S;"),
    "dfeat_wrong_group_weight": ("+= wg[g] * cr.omega[q] * go[c];", "+= wg[0] * cr.omega[q] * go[c];"),
}

PIN_TESTS = [
    ("hand", lambda lib: pins.test_hand_worked_example(lib)),
    ("const_boundary", lambda lib: pins.test_constant_map_boundary(lib)),
    ("linear", lambda lib: pins.test_linear_map_reproduced(lib)),
    ("tent", lambda lib: pins.test_brute_force_tent_kernel(lib, 0)),
    ("grid_sample", lambda lib: pins.test_grid_sample_forward_and_autograd(lib, 0)),
    ("fd_loc", lambda lib: pins.test_finite_differences_location(lib)),
    ("adjoint", lambda lib: pins.test_adjoint_identities(lib)),
    ("oae_uniform", lambda lib: oae_pins.test_uniform_visibility_is_mean_over_cameras(lib)),
    ("oae_weighted", lambda lib: oae_pins.test_weighted_mean_of_camera_runs_and_scale_invariance(lib)),
    ("kp_hand", lambda lib: kp_pins.test_hand_worked_projection(lib)),
    ("kp_yaw", lambda lib: kp_pins.test_yaw_rotates_box_offsets(lib)),
    ("kp_yaw_y", lambda lib: kp_pins.test_yaw_rotates_box_y_offsets(lib)),
    ("kp_motion", lambda lib: kp_pins.test_motion_compensation_moves_the_centre(lib)),
]


def _mutant_oracle(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not unique/found"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = oracle.compile_oracle(str(path), str(tmp_path / f"lib{name}.so"), openmp=False)
    lib = oracle.load_library(so)
    return types.SimpleNamespace(forward=partial(oracle.forward, lib=lib),
                                 backward=partial(oracle.backward, lib=lib),
                                 forward_oae=partial(oracle.forward_oae, lib=lib),
                                 keypoints=partial(oracle.keypoints, lib=lib))


def test_unmutated_copy_passes_every_pin(tmp_path):
    src = open(SRC).read()
    path = tmp_path / "same.c"
    path.write_text(src)
    lib = oracle.load_library(oracle.compile_oracle(str(path), str(tmp_path / "libsame.so"), openmp=False))
    ns = types.SimpleNamespace(forward=partial(oracle.forward, lib=lib), backward=partial(oracle.backward, lib=lib),
                               forward_oae=partial(oracle.forward_oae, lib=lib),
                               keypoints=partial(oracle.keypoints, lib=lib))
    for _, t in PIN_TESTS:
        t(ns)


def _run_pins_in_child(tmp, name, q):
    old, new = MUTANTS[name]
    import pathlib
    lib = _mutant_oracle(pathlib.Path(tmp), name, old, new)
    q.put("started")
    caught = []
    for pin, t in PIN_TESTS:
        try:
            t(lib)
        except (AssertionError, ValueError):
            caught.append(pin)
    q.put(caught)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    """A mutant may also crash (an off-by-one bound reads past the map); that counts as caught."""
    ctx = multiprocessing.get_context("spawn")
    q = ctx.Queue()
    proc = ctx.Process(target=_run_pins_in_child, args=(str(tmp_path), name, q))
    proc.start()
    proc.join(300)
    if proc.is_alive():
        proc.kill()
        pytest.fail(f"mutant {name} did not finish")
    first = q.get(timeout=10) if not q.empty() else None
    assert first == "started", f"mutant {name} failed before its pins ran (exit {proc.exitcode})"
    if proc.exitcode != 0:
        print(f"{name}: crashed inside the pins (caught)")
        return
    caught = q.get(timeout=10)
    print(f"{name}: caught by {caught}")
    assert caught, f"mutant {name} passed every pin"
