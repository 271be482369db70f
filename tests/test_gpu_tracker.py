"""The persistent PFO kernel (pfo_track_frame, Algorithm 1) against the FP64
oracle, plus the sequence API, the bounded-barrier failure path and the
empty-overlap corner case, through the C ABI.

Parity bar per iteration k: |O_k| and |APS| equal unless the oracle reports a
decision within tolerance of its threshold (an overlap pixel within 1e-3 px of
a rounding boundary, a particle within 1e-5 of the APS threshold); the best
state s*_k within 2e-4 (quaternion and metres) and the axis lengths r_k within
rel 2e-3 of the oracle's until the first such decision."""
import numpy as np
import pytest

from gpu_common import analytic_volume_codes, compare_traces as _compare_traces, oracle_volume, pose_f32
from paper_2105_05600_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def _oracle_params(oracle, k_max, flags=None):
    return dict(tau=1.0, beta=0.1, eps=1e-3, stop_eps=1e-6, k_max=k_max,
                flags=oracle.DEFAULT_FLAGS if flags is None else flags)


def _tiny_problem(oracle, nat, dtype="f32"):
    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype=dtype)
    gv = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), cfg["dtype"])
    gv.upload(codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 3, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    d0 = synth.render_depth(scene, traj[0], K)
    d1 = synth.render_depth(scene, traj[1], K)
    return scene, cfg, gv, ov, traj, K, d0, d1


@pytest.mark.parametrize("dtype", ["f32", "i16"])
@pytest.mark.parametrize("r0", [1.0, 0.08])
def test_tracker_parity_tiny(oracle, nat, dtype, r0):
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat, dtype)
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    params = nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"])
    tr = nat.Tracker(gv, pst, params, cfg["width"], cfg["height"])
    tr.set_scale([r0] * 6)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, prev)
    assert status == 0
    pts = oracle.unproject(d1, K, cfg["stride"])
    res = ov.pfo_frame(pts, d0, K, prev, prev, np.full(6, np.float32(r0)), oracle.pst_uniform(n, 1),
                       _oracle_params(oracle, cfg["k_max"]))
    assert res["status"] == 0
    strict = _compare_traces(gst, res["trace"])
    assert strict >= 1
    if strict == len(res["trace"]) == gst["iters"]:
        np.testing.assert_allclose(np.abs(pose[:4]), np.abs(res["pose"][:4]), atol=2e-4)
        np.testing.assert_allclose(pose[4:], res["pose"][4:], atol=2e-4)
        np.testing.assert_allclose(gst["r1"], res["r1"], rtol=2e-3, atol=2e-6)
    # the frame summary is consistent with the rows
    assert gst["lookups"] == sum(r["n_overlap"] for r in gst["it"]) * n
    assert 1 <= gst["iters"] <= cfg["k_max"]
    np.testing.assert_allclose(tr.get_scale(), gst["r1"])


def test_tracker_first_iteration_paper_scale(oracle, nat):
    """512^3 int16, 640x480 at stride 4, 20k particles: iteration 1 depends only on
    generator inputs, so the oracle recomputes it completely."""
    import torch

    scene, codes, F64, cfg = analytic_volume_codes("paper")
    gv = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), cfg["dtype"])
    gv.upload(codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    rng = np.random.default_rng(9)
    d0 = synth.render_depth(scene, traj[0], K, rng)
    d1 = synth.render_depth(scene, traj[1], K, rng)
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=1, stride=cfg["stride"]), 640, 480)
    tr.set_scale([0.05] * 6)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, prev)
    assert status == 0 and gst["iters"] == 1
    pts = oracle.unproject(d1, K, cfg["stride"])
    res = ov.pfo_frame(pts, d0, K, prev, prev, np.full(6, np.float32(0.05)), oracle.pst_uniform(n, 1),
                       _oracle_params(oracle, 1))
    _compare_traces(gst, res["trace"])


def test_tracker_timeout_hook_reports_and_recovers(oracle, nat):
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat)
    pst = nat.pst_create(256, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=5), cfg["width"], cfg["height"])
    D0, D1 = torch.from_numpy(d0).cuda(), torch.from_numpy(d1).cuda()
    tr.set_scale([0.1] * 6)
    ref_pose, ref_stats, st = nat.pfo_track_frame(tr, D1, D0, K, traj[0])
    assert st == 0
    tr.set_scale([0.1] * 6)
    tr.debug_skip_barrier(True, 50)  # block 0 never arrives: the others give up after 50 ms
    _, gst, status = nat.pfo_track_frame(tr, D1, D0, K, traj[0], check=False)
    assert status == nat.RF_ERR_TIMEOUT
    # the context is still usable and the next frame runs normally
    tr.set_scale([0.1] * 6)
    pose, gst2, status2 = nat.pfo_track_frame(tr, D1, D0, K, traj[0])
    assert status2 == 0
    np.testing.assert_array_equal(pose, ref_pose)


def test_tracker_empty_overlap(oracle, nat):
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat)
    pst = nat.pst_create(128, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=5), cfg["width"], cfg["height"])
    zeros = torch.zeros((cfg["height"], cfg["width"]), device="cuda")
    pose, gst, status = nat.pfo_track_frame(tr, zeros, torch.from_numpy(d0).cuda(), K, traj[0])
    assert status == nat.RF_ERR_EMPTY
    np.testing.assert_allclose(pose, pose_f32(traj[0]), atol=1e-7)
    assert gst["it"][0]["stop"] == 4


def test_tracker_is_deterministic(oracle, nat):
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat, "i16")
    pst = nat.pst_create(1024, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=10), cfg["width"], cfg["height"])
    out = []
    for _ in range(2):
        tr.set_scale([0.2] * 6)
        pose, gst, st = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, traj[0])
        out.append((pose, gst))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]


def test_sequence_mode_matches_explicit_calls(oracle, nat):
    import torch

    cfg = synth.CONFIGS["tiny"]
    scene = synth.make_scene(cfg["dims"] * cfg["voxel"], cfg["wall_inset"], 0)
    traj = synth.make_trajectory(scene, 4, 3.0, 3.0, 0)
    K = synth.intrinsics(cfg["width"], cfg["height"])
    depths = [synth.render_depth(scene, traj[f], K) for f in range(4)]
    pst = nat.pst_create(512, seed=1)
    params = nat.make_params(k_max=8)
    # (a) sequence API with host depth
    va = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), "f32")
    ta = nat.Tracker(va, pst, params, cfg["width"], cfg["height"])
    nat.rf_sequence_start(ta, depths[0], K, traj[0])
    poses_a = [nat.rf_sequence_step(ta, depths[f], K)[0] for f in range(1, 4)]
    # (b) sequence API with device depth
    vb = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), "f32")
    tb = nat.Tracker(vb, pst, params, cfg["width"], cfg["height"])
    nat.rf_sequence_start(tb, torch.from_numpy(depths[0]).cuda(), K, traj[0])
    poses_b = [nat.rf_sequence_step(tb, torch.from_numpy(depths[f]).cuda(), K)[0] for f in range(1, 4)]
    # (c) explicit pfo_track_frame + tsdf_integrate
    vc = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), "f32")
    tc = nat.Tracker(vc, pst, params, cfg["width"], cfg["height"])
    D = [torch.from_numpy(d).cuda() for d in depths]
    nat.tsdf_integrate(vc, D[0], K, traj[0])
    prev = pose_f32(traj[0])
    poses_c = []
    for f in range(1, 4):
        pose, _, st = nat.pfo_track_frame(tc, D[f], D[f - 1], K, prev)
        nat.tsdf_integrate(vc, D[f], K, pose)
        poses_c.append(pose)
        prev = pose
    for a, b, c in zip(poses_a, poses_b, poses_c):
        np.testing.assert_array_equal(a, b)
        np.testing.assert_array_equal(a, c)
    ca, wa = va.download()
    cc, wc = vc.download()
    np.testing.assert_array_equal(wa, wc)


def test_tracker_rejects_oversized_frames(nat):
    import torch

    v = nat.Volume(16, 0.1, 0.3, (0, 0, 0), "f32")
    pst = nat.pst_create(32, seed=1)
    tr = nat.Tracker(v, pst, nat.make_params(), 40, 30)
    K = synth.intrinsics(80, 60)
    d = torch.zeros((60, 80), device="cuda")
    with pytest.raises(nat.RfError):
        nat.pfo_track_frame(tr, d, d, K, [1, 0, 0, 0, 0, 0, 0])
    with pytest.raises(nat.RfError):
        nat.Tracker(v, pst, nat.make_params(k_max=0), 40, 30)
