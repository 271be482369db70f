"""Pins for the oracle's multi-resolution PST alternation (Sec. 4, "Multi-resolution
PST"): one level reduces exactly to the pinned single-resolution Algorithm 1;
two identical levels with the centre-particle threshold reduce to it as well;
the level schedule cycles as stated; and on a tiny fully observed room the
alternating run still beats a brute-force 7^6 pose grid on the full-resolution
objective."""
import math

import numpy as np
import pytest

from paper_2105_05600_gb300 import synth
from test_oracle_pfo import _params, _scene_volume


def _frame(oracle, W=40, H=30):
    scene, v = _scene_volume(oracle)
    K = synth.intrinsics(W, H)
    eye = np.array([0.72, 0.70, 0.68])
    T = np.concatenate([synth.look_at_quat(eye, [1.5, 1.45, 1.5]), eye])
    depth = synth.render_depth(scene, T, K)
    c0 = oracle.compose_offset(T, [0.010, -0.015, 0.012, 0.02, -0.01, 0.015])
    return v, K, T, depth, c0


def test_single_level_is_algorithm_1(oracle):
    v, K, T, depth, c0 = _frame(oracle)
    pts = oracle.unproject(depth, K, 2)
    omega = oracle.pst_uniform(512, 1)
    p = _params(oracle, flags=oracle.DEFAULT_FLAGS, k_max=8)
    a = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, p)
    b = v.pfo_frame_sched([pts], [512], depth, K, c0, c0, np.full(6, 0.05), omega, p)
    assert a["iters"] == b["iters"] and a["status"] == b["status"]
    np.testing.assert_array_equal(a["pose"], b["pose"])
    np.testing.assert_array_equal(a["r1"], b["r1"])
    np.testing.assert_array_equal(a["trace"][:, :30], b["trace"][:, :30])


def test_two_identical_levels_with_centre_threshold(oracle):
    v, K, T, depth, c0 = _frame(oracle)
    pts = oracle.unproject(depth, K, 2)
    omega = oracle.pst_uniform(512, 1)
    p = _params(oracle, flags=oracle.DEFAULT_FLAGS | oracle.RHO_REF_CENTER, k_max=8)
    a = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, p)
    b = v.pfo_frame_sched([pts, pts], [512, 512], depth, K, c0, c0, np.full(6, 0.05), omega, p)
    np.testing.assert_array_equal(a["pose"], b["pose"])
    np.testing.assert_array_equal(a["trace"][:, :30], b["trace"][:, :30])


def test_level_schedule_cycles(oracle):
    v, K, T, depth, c0 = _frame(oracle)
    sets = [oracle.unproject(depth, K, s) for s in (3, 2, 1)]
    omega = oracle.pst_uniform(1024, 1)
    p = _params(oracle, flags=oracle.NORMALIZE | oracle.COMPENSATED, k_max=7)  # no overlap: |O| = valid points
    res = v.pfo_frame_sched(sets, [256, 512, 1024], depth, K, c0, c0, np.full(6, 0.2), omega, p)
    for row in res["trace"]:
        k = int(row[0])
        lvl = (k - 1) % 3
        assert row[30] == lvl and row[31] == [256, 512, 1024][lvl]
        assert row[1] == int((sets[lvl][:, 3] > 0).sum())
        assert 0 <= row[6] < [256, 512, 1024][lvl]  # argmax within the level's particles


def test_multires_beats_brute_force_grid(oracle):
    v, K, T, depth, c0 = _frame(oracle)
    full = oracle.unproject(depth, K, 1)
    sets = [oracle.unproject(depth, K, s) for s in (3, 2, 1)]
    omega = oracle.pst_uniform(2048, 1)
    p = _params(oracle, flags=oracle.NORMALIZE | oracle.COMPENSATED, k_max=21)
    res = v.pfo_frame_sched(sets, [512, 1024, 2048], depth, K, c0, c0, np.full(6, 0.05), omega, p)
    assert res["status"] == 0
    valid = (full[:, 3] > 0).astype(np.int32)
    rho_pfo = v.fitness(full, valid, res["pose"], flags=oracle.NORMALIZE)[3]
    half = [math.sin(math.radians(2.5))] * 3 + [0.05] * 3
    rho_grid, _ = v.grid_search(full, valid, c0, half, 7, flags=oracle.NORMALIZE)
    assert rho_pfo >= rho_grid - 1e-4
    assert np.linalg.norm(res["pose"][4:] - T[4:]) < 0.02
