"""Pins for the oracle's Algorithm 1 (PFO with PST) on tiny inputs:

* brute force: on a fully observed analytic room TSDF, the pose PFO returns
  scores at least as well as the best pose of a 7^6 grid of offsets spanning
  +-5 cm / +-5 degrees around the start (117,649 candidates), and lands within
  2 cm / 1.5 degrees of the true pose;
* the empty-APS corner case and the stop rule "APS empty twice" (Sec. 4) on a
  constant volume, where no particle can beat the centre;
* an empty overlap set leaves the pose unchanged and reports EMPTY;
* the first corner case of Sec. 4 (no TSDF yet: rho = 0.5, isotropic v = 1) on
  a volume with no observed voxel, in closed form;
* the APS with and without the centre particle (flag APS_WITH_CENTRE) on a
  constant volume, in closed form;
* one iteration (or_pfo_step) replays or_pfo_frame row for row, also when
  restarted from the state stored in a trace row, and the thread count of the
  per-particle loop and of fusion does not change any result."""
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


def _state_from_row(oracle, row, k):
    """The Algorithm 1 state after trace row `row`, for iteration k."""
    return dict(c=row[oracle.T_POSE], r=row[oracle.T_SCALE], rho_carry=row[oracle.T_RHO_TILDE],
                empty_run=int(row[oracle.T_EMPTY_RUN]), k=k)


def test_step_replays_the_frame_and_the_trace_holds_the_state(oracle):
    # or_pfo_step fed its own state reproduces or_pfo_frame row for row; started
    # instead from the state read back out of trace row k-1 it reproduces row k,
    # so a trace row carries everything the next iteration needs
    v, K, T, depth, c0 = _frame_for_steps(oracle)
    pts = oracle.unproject(depth, K, 2)
    omega = oracle.pst_uniform(512, 1)
    p = _params(oracle, flags=oracle.DEFAULT_FLAGS, k_max=12)
    ref = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, p)
    assert ref["iters"] >= 3
    state = dict(c=c0, r=np.full(6, 0.05), rho_carry=0.0, empty_run=0, k=1)
    for k in range(1, ref["iters"] + 1):
        stop, state, row = v.pfo_step(pts, 512, depth, K, c0, omega, p, state)
        np.testing.assert_array_equal(row, ref["trace"][k - 1])
        assert stop == int(ref["trace"][k - 1][oracle.T_STOP])
        if k < ref["iters"]:
            _, _, row2 = v.pfo_step(pts, 512, depth, K, c0, omega, p,
                                    _state_from_row(oracle, ref["trace"][k - 1], k + 1))
            np.testing.assert_array_equal(row2, ref["trace"][k])
    assert stop != 0 or ref["iters"] == p["k_max"]


def _frame_for_steps(oracle):
    scene, v = _scene_volume(oracle)
    K = synth.intrinsics(40, 30)
    eye = np.array([0.72, 0.70, 0.68])
    T = np.concatenate([synth.look_at_quat(eye, [1.5, 1.45, 1.5]), eye])
    depth = synth.render_depth(scene, T, K)
    c0 = oracle.compose_offset(T, [0.010, -0.015, 0.012, 0.02, -0.01, 0.015])
    return v, K, T, depth, c0


def test_thread_count_does_not_change_results(oracle):
    v, K, T, depth, c0 = _frame_for_steps(oracle)
    pts = oracle.unproject(depth, K, 1)
    omega = oracle.pst_uniform(300, 1)
    p = _params(oracle, flags=oracle.DEFAULT_FLAGS, k_max=6)
    a = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, p)
    b = v.pfo_frame(pts, depth, K, c0, c0, np.full(6, 0.05), omega, p, threads=7)
    np.testing.assert_array_equal(a["trace"], b["trace"])
    np.testing.assert_array_equal(a["pose"], b["pose"])
    c = v.pfo_frame_sched([pts, oracle.unproject(depth, K, 2)], [300, 100], depth, K, c0, c0, np.full(6, 0.05),
                          omega, p, threads=5)
    d = v.pfo_frame_sched([pts, oracle.unproject(depth, K, 2)], [300, 100], depth, K, c0, c0, np.full(6, 0.05),
                          omega, p)
    np.testing.assert_array_equal(c["trace"], d["trace"])
    # fusion: slices split over threads
    w1 = oracle.Volume((16, 16, 16), 0.1, (0, 0, 0), 0.3, qmode="i16")
    w2 = oracle.Volume((16, 16, 16), 0.1, (0, 0, 0), 0.3, qmode="i16")
    scene = synth.make_scene(1.6, 0.1, seed=1)
    Kd = synth.intrinsics(32, 24)
    pose = np.concatenate([synth.look_at_quat([0.4, 0.4, 0.5], [1.0, 1.1, 0.9]), [0.4, 0.4, 0.5]])
    dep = synth.render_depth(scene, pose, Kd)
    w1.integrate(dep, Kd, pose)
    w2.integrate(dep, Kd, pose, threads=6)
    np.testing.assert_array_equal(w1.F, w2.F)
    np.testing.assert_array_equal(w1.W, w2.W)
    assert np.isfinite(w1.F).sum() > 100


def _constant_setup(oracle, value):
    v = oracle.Volume((8, 8, 8), 0.25, (0, 0, 0), trunc=1.0)
    v.F[:] = value
    pts = np.zeros((50, 4))
    pts[:, :3] = np.random.default_rng(0).uniform(0.8, 1.2, size=(50, 3))
    pts[:, 3] = 1
    depth = np.ones((4, 4), np.float32)
    K = dict(fx=2.0, fy=2.0, cx=1.5, cy=1.5, z_min=0.1, z_max=8.0, width=4, height=4)
    return v, pts, depth, K


def test_no_tsdf_corner_case(oracle):
    # Sec. 4 "PST update", first corner case: with no TSDF to sample the likelihood
    # cannot be evaluated; rho = 0.5, v = 1 (not normalised), r_hat = 0.5 v (+ eps),
    # and the state does not move.  Every voxel unobserved:
    v, pts, depth, K = _constant_setup(oracle, np.nan)
    c0 = np.array([1, 0, 0, 0, 0, 0, 0], float)
    r0 = np.array([0.01, 0.02, 0.03, 0.04, 0.05, 0.06])
    res = v.pfo_frame(pts, depth, K, c0, c0, r0, oracle.pst_uniform(64, seed=2), _params(oracle))
    tr = res["trace"]
    assert res["iters"] == 2 and tr[1][oracle.T_STOP] == 1  # counts as an empty APS twice
    r1 = 0.1 * r0 + 0.9 * (0.5 + 1e-3)
    np.testing.assert_allclose(res["r1"], r1, rtol=1e-14)
    np.testing.assert_allclose(tr[1][oracle.T_SCALE], 0.1 * r1 + 0.9 * (0.5 + 1e-3), rtol=1e-14)
    for row in tr:
        assert row[oracle.T_CORNER] == 1 and row[oracle.T_NAPS] == 0 and row[oracle.T_VALID] == 0
        assert row[oracle.T_RHO_TILDE] == 0.5
        np.testing.assert_array_equal(row[oracle.T_POSE], c0)
    # the carried 0.5 is the next threshold (k = 2), as for any Eq. wafit value
    assert tr[1][oracle.T_RHO_REF] == 0.5
    # one observed voxel in reach of one sample is enough to leave the corner case
    v2, _, _, _ = _constant_setup(oracle, np.nan)
    g = v2.grid()
    g[3:5, 3:5, 3:5] = 0.2
    res2 = v2.pfo_frame(pts, depth, K, c0, c0, r0, oracle.pst_uniform(64, seed=2), _params(oracle))
    assert res2["trace"][0][oracle.T_CORNER] != 1 and res2["trace"][0][oracle.T_VALID] > 0


def test_aps_with_centre_flag(oracle):
    # constant volume: every particle scores exp(-0.09) > the carried threshold 0.5,
    # so all candidates join the APS with equal weights and delta_bar is their mean
    # offset; with APS_WITH_CENTRE the centre (offset 0) is one more member
    v, pts, depth, K = _constant_setup(oracle, 0.3)
    N = 64
    omega = oracle.pst_uniform(N, seed=2)
    r = np.full(6, 0.01)
    c = np.array([1, 0, 0, 0, 0, 0, 0], float)
    state = dict(c=c, r=r, rho_carry=0.5, empty_run=0, k=2)
    off = (r[:, None] * omega.astype(np.float64)).T  # offsets of all particles
    base = oracle.NORMALIZE | oracle.COMPENSATED  # no overlap set: all 50 points count
    for flags, members in ((base, range(1, N)), (base | oracle.APS_WITH_CENTRE, range(0, N))):
        stop, new, row = v.pfo_step(pts, N, depth, K, c, omega, _params(oracle, flags=flags), state)
        members = list(members)
        assert row[oracle.T_NAPS] == len(members)
        dbar = off[members].mean(axis=0)
        np.testing.assert_allclose(row[oracle.T_DBAR], dbar, rtol=1e-12, atol=1e-18)
        np.testing.assert_allclose(row[oracle.T_RHO_TILDE], math.exp(-0.09), rtol=1e-14)
        w = math.exp(-0.09) - 0.5
        sens = sum(np.max(np.abs(off[i] - dbar)) for i in members) / (len(members) * w)
        np.testing.assert_allclose(row[oracle.T_SENS], sens, rtol=1e-12)
        assert row[oracle.T_CORNER] == 0 and new["empty_run"] == 0
