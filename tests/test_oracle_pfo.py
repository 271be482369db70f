"""Pins for the oracle's Algorithm 1 (PFO with PST) on tiny inputs:

* brute force: on a fully observed analytic room TSDF, the pose PFO returns
  scores at least as well as the best pose of a 7^6 grid of offsets spanning
  +-5 cm / +-5 degrees around the start (117,649 candidates), and lands within
  2 cm / 1.5 degrees of the true pose;
* the empty-APS corner case and the stop rule "APS empty twice" (Sec. 4) on a
  constant volume, where no particle can beat the centre;
* an empty overlap set leaves the pose unchanged and reports EMPTY."""
import math

import numpy as np
import pytest

from paper_2105_05600_gb300 import synth


def _scene_volume(oracle):
    dims, voxel, trunc = (32, 32, 32), 0.05, 0.15
    scene = synth.make_scene(dims[0] * voxel, 0.1, seed=3)
    F = synth.analytic_tsdf(scene.sdf, dims, voxel, (0, 0, 0), trunc)
    v = oracle.Volume(dims, voxel, (0, 0, 0), trunc)
    v.F[:] = F.reshape(-1)
    return scene, v


def _params(oracle, **kw):
    p = dict(tau=1.0, beta=0.1, eps=1e-3, stop_eps=1e-6, k_max=20, flags=oracle.NORMALIZE | oracle.COMPENSATED)
    p.update(kw)
    return p


def _rot_err_deg(a, b):
    return math.degrees(2 * math.acos(min(1.0, abs(float(np.dot(a[:4], b[:4]))))))


def test_pfo_beats_brute_force_grid(oracle):
    scene, v = _scene_volume(oracle)
    K = synth.intrinsics(20, 15)
    eye = np.array([0.72, 0.70, 0.68])
    T = np.concatenate([synth.look_at_quat(eye, [1.5, 1.45, 1.5]), eye])
    depth = synth.render_depth(scene, T, K)
    pts = oracle.unproject(depth, K, 1)
    valid = (pts[:, 3] > 0).astype(np.int32)
    assert valid.sum() > 250
    c0 = oracle.compose_offset(T, [0.010, -0.015, 0.012, 0.02, -0.01, 0.015])
    omega = oracle.pst_uniform(1024, seed=1)
    res = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, _params(oracle))
    assert res["status"] == 0
    _, _, _, rho_pfo = v.fitness(pts, valid, res["pose"], flags=oracle.NORMALIZE)
    half = [math.sin(math.radians(2.5))] * 3 + [0.05] * 3
    rho_grid, _ = v.grid_search(pts, valid, c0, half, 7, flags=oracle.NORMALIZE)
    assert rho_pfo >= rho_grid - 1e-4
    assert np.linalg.norm(res["pose"][4:] - T[4:]) < 0.02
    assert _rot_err_deg(res["pose"], T) < 1.5
    # the trace is consistent: rho_tilde never decreases while the APS is non-empty
    tr = res["trace"]
    assert tr[0][1] == valid.sum()  # |O| without the overlap flag = all valid points
    rt = [row[4] for row in tr if row[2] > 0]
    assert all(b >= a - 1e-12 for a, b in zip(rt, rt[1:]))


def test_empty_aps_twice_stops(oracle):
    v = oracle.Volume((8, 8, 8), 0.25, (0, 0, 0), trunc=1.0)
    v.F[:] = 0.3  # every particle scores exp(-0.09): nobody is strictly better than the centre
    pts = np.zeros((50, 4))
    pts[:, :3] = np.random.default_rng(0).uniform(0.8, 1.2, size=(50, 3))
    pts[:, 3] = 1
    depth = np.ones((4, 4), np.float32)
    K = dict(fx=2.0, fy=2.0, cx=1.5, cy=1.5, z_min=0.1, z_max=8.0, width=4, height=4)
    c0 = np.array([1, 0, 0, 0, 0, 0, 0], float)
    omega = oracle.pst_uniform(64, seed=2)
    r0 = np.full(6, 0.01)
    res = v.pfo_frame(pts, depth, K, c0, c0, r0, omega, _params(oracle))
    assert res["iters"] == 2 and res["trace"][1][28] == 1  # stop reason: empty APS twice
    np.testing.assert_allclose(res["pose"], c0)
    rho = math.exp(-0.09)
    rhat = 2 * (1 - rho) / math.sqrt(6) + 1e-3  # Sec. 4 second corner case, + eps
    r1 = 0.1 * 0.01 + 0.9 * rhat
    np.testing.assert_allclose(res["r1"], r1, rtol=1e-12)
    np.testing.assert_allclose(res["trace"][1][14:20], 0.1 * r1 + 0.9 * rhat, rtol=1e-12)


def test_empty_overlap_keeps_pose(oracle):
    v = oracle.Volume((8, 8, 8), 0.25, (0, 0, 0), trunc=1.0)
    v.F[:] = 0.1
    pts = np.zeros((10, 4))  # no valid depth at all
    depth = np.zeros((4, 4), np.float32)
    K = dict(fx=2.0, fy=2.0, cx=1.5, cy=1.5, z_min=0.1, z_max=8.0, width=4, height=4)
    c0 = np.array([1, 0, 0, 0, 0.5, 0.5, 0.5])
    res = v.pfo_frame(pts, depth, K, c0, c0, np.ones(6), oracle.pst_uniform(8, 1), _params(oracle, flags=7))
    assert res["status"] == -4 and res["iters"] == 1
    np.testing.assert_allclose(res["pose"], c0)
    np.testing.assert_allclose(res["r1"], np.ones(6))


def test_template_must_start_at_origin(oracle):
    v = oracle.Volume((8, 8, 8), 0.25, (0, 0, 0), trunc=1.0)
    omega = oracle.pst_uniform(8, 1)
    omega[:, [0, 1]] = omega[:, [1, 0]]
    pts = np.zeros((4, 4))
    res = v.pfo_frame(pts, np.zeros((2, 2), np.float32), dict(fx=1, fy=1, cx=0.5, cy=0.5, z_min=0.1, z_max=8,
                                                                 width=2, height=2),
                      np.array([1, 0, 0, 0, 0, 0, 0.0]), np.array([1, 0, 0, 0, 0, 0, 0.0]), np.ones(6), omega,
                      _params(oracle))
    assert res["status"] == -1


def test_centre_particle_is_never_in_the_aps(oracle):
    # The APS holds particles better than s*_{k-1} (Sec. 3.3); particle 0 is s*_{k-1}
    # itself.  Late in this run the carried Eq. wafit threshold lies below the centre's
    # own fitness while every other particle is below it: the centre is the arg max and
    # the second-best fitness is <= rho_ref < rho_max.  Such an iteration must report
    # an empty APS, no step, and must not end on the small-step rule.
    scene, v = _scene_volume(oracle)
    K = synth.intrinsics(20, 15)
    eye = np.array([0.72, 0.70, 0.68])
    T = np.concatenate([synth.look_at_quat(eye, [1.5, 1.45, 1.5]), eye])
    depth = synth.render_depth(scene, T, K)
    pts = oracle.unproject(depth, K, 1)
    c0 = oracle.compose_offset(T, [0.004, -0.006, 0.005, 0.01, -0.01, 0.008])
    res = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.1), oracle.pst_uniform(16, seed=4), _params(oracle))
    only_centre = [row for row in res["trace"] if row[6] == 0 and row[29] <= row[3] < row[5]]
    assert only_centre  # the case occurs in this run
    for row in only_centre:
        assert row[2] == 0 and np.all(row[20:26] == 0.0) and row[28] != 2
