"""The persistent PFO kernel (pfo_track_frame, Algorithm 1) against the FP64
oracle, plus the sequence API, the bounded-barrier failure path and the corner
cases of Sec. 4, through the C ABI.

Parity bar (gpu_common.replay_trace): EVERY iteration k of a GPU frame is
recomputed by one oracle iteration started from the state the GPU reached after
iteration k-1, and must agree: |O_k|, |APS|, corner case and stop code equal,
the fitness values within rel 1e-4, delta_bar, s*_k and r_k within the bound
the weights' FP32 error implies.  An iteration may differ only where the oracle
reports a decision inside its tie margin (an overlap pixel within 1e-3 px of a
rounding boundary, a candidate within 1e-5 of the APS threshold), and only by
the number of such decisions."""
import numpy as np
import pytest

from gpu_common import analytic_volume_codes, oracle_volume, pose_f32, replay_trace
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


def _check_frame(oracle, ov, gst, pose, levels, d_prev, K, prev, c0, r0, n, params, tr=None):
    """Replay every iteration; the frame's outputs are those of its last row."""
    res = replay_trace(oracle, ov, gst, levels, d_prev, K, prev, c0, r0, oracle.pst_uniform(n, 1), params)
    last = gst["it"][-1]
    np.testing.assert_array_equal(np.asarray(pose, np.float32), np.asarray(last["pose"], np.float32))
    if gst["it"][0]["stop"] != 4:
        np.testing.assert_array_equal(np.float32(gst["r1"]), np.float32(gst["it"][0]["scale"]))
    if tr is not None:
        np.testing.assert_array_equal(np.float32(tr.get_scale()), np.float32(gst["r1"]))
    assert gst["lookups"] == sum(r["n_overlap"] * r["n_particles"] for r in gst["it"])
    assert res["loose"] <= max(1, res["rows"] // 4), res
    return res


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
    assert status == 0 and 1 <= gst["iters"] <= cfg["k_max"]
    pts = oracle.unproject(d1, K, cfg["stride"])
    res = _check_frame(oracle, ov, gst, pose, [(pts, n)], d0, K, prev, prev, np.full(6, np.float32(r0)), n,
                       _oracle_params(oracle, cfg["k_max"]), tr)
    print("replay", dtype, r0, res)


@pytest.mark.parametrize("flags_name", ["no_cell_margin", "aps_with_centre", "rho_ref_centre_l1_right"])
def test_tracker_parity_readings(oracle, nat, flags_name):
    """The readings of the paper that are flags, each setting traced against the
    oracle: the paper-literal overlap set of Eq. validness (no cell margin), the
    centre particle as an APS candidate, and the remaining variants together."""
    import torch

    flags = {"no_cell_margin": nat.RF_DEFAULT_FLAGS & ~nat.RF_CELL_MARGIN,
             "aps_with_centre": nat.RF_DEFAULT_FLAGS | nat.RF_APS_WITH_CENTRE,
             "rho_ref_centre_l1_right": nat.RF_DEFAULT_FLAGS | nat.RF_RHO_REF_CENTER | nat.RF_L1 |
                                        nat.RF_RIGHT_MULT}[flags_name]
    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat, "i16")
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"], flags=flags), cfg["width"],
                     cfg["height"])
    tr.set_scale([0.1] * 6)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, prev)
    assert status == 0
    pts = oracle.unproject(d1, K, cfg["stride"])
    res = _check_frame(oracle, ov, gst, pose, [(pts, n)], d0, K, prev, prev, np.full(6, np.float32(0.1)), n,
                       _oracle_params(oracle, cfg["k_max"], flags), tr)
    print("replay", flags_name, res)


@pytest.mark.parametrize("group", [4, 8])
def test_tracker_parity_lookup_groups(oracle, nat, group):
    """The kernel variants with 4 and 8 lookups in flight (the default is 6), as
    the autotuner may pick them, against the oracle iteration by iteration."""
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat, "i16")
    n = cfg["n_particles"]
    tr = nat.Tracker(gv, nat.pst_create(n, seed=1), nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"]),
                     cfg["width"], cfg["height"])
    tr.set_config(ctas_per_sm=0, work_warps=1824, group=group)
    assert tr.get_config()["group"] == group
    tr.set_scale([0.1] * 6)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, prev)
    assert status == 0
    pts = oracle.unproject(d1, K, cfg["stride"])
    _check_frame(oracle, ov, gst, pose, [(pts, n)], d0, K, prev, prev, np.full(6, np.float32(0.1)), n,
                 _oracle_params(oracle, cfg["k_max"]), tr)


def test_tracker_autotune_then_parity(oracle, nat):
    """rf_tracker_autotune picks a launch configuration on one frame, restores the
    tracker's r_0, and the frame tracked with that configuration matches the
    oracle iteration by iteration."""
    import torch

    scene, cfg, gv, ov, traj, K, d0, d1 = _tiny_problem(oracle, nat, "i16")
    n = cfg["n_particles"]
    tr = nat.Tracker(gv, nat.pst_create(n, seed=1), nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"]),
                     cfg["width"], cfg["height"])
    tr.set_scale([0.1] * 6)
    prev = pose_f32(traj[0])
    D0, D1 = torch.from_numpy(d0).cuda(), torch.from_numpy(d1).cuda()
    chosen = tr.autotune(D1, D0, K, torch.from_numpy(prev.astype(np.float32)).cuda())
    assert chosen["group"] in (4, 6, 8) and chosen["ctas_per_sm"] >= 1 and chosen["ms"] > 0
    assert tr.get_config() == chosen
    np.testing.assert_array_equal(tr.get_scale(), np.float32([0.1] * 6))
    pose, gst, status = nat.pfo_track_frame(tr, D1, D0, K, prev)
    assert status == 0
    pts = oracle.unproject(d1, K, cfg["stride"])
    _check_frame(oracle, ov, gst, pose, [(pts, n)], d0, K, prev, prev, np.full(6, np.float32(0.1)), n,
                 _oracle_params(oracle, cfg["k_max"]), tr)


def _paper_problem(oracle, nat):
    scene, codes, F64, cfg = analytic_volume_codes("paper")
    gv = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), cfg["dtype"])
    gv.upload(codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 6, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    rng = np.random.default_rng(9)
    depths = [synth.render_depth(scene, traj[f], K, rng) for f in range(6)]
    return cfg, gv, ov, traj, K, depths


def test_tracker_full_frame_paper_scale(oracle, nat):
    """512^3 int16, 640x480 at stride 4, 20k particles, <= 20 iterations, the
    bench's first frame (r_0 = 1): every iteration replayed by the oracle."""
    import torch

    cfg, gv, ov, traj, K, depths = _paper_problem(oracle, nat)
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"]), 640, 480)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(depths[1]).cuda(),
                                            torch.from_numpy(depths[0]).cuda(), K, prev)
    assert status == 0
    pts = oracle.unproject(depths[1], K, cfg["stride"])
    res = _check_frame(oracle, ov, gst, pose, [(pts, n)], depths[0], K, prev, prev, np.ones(6), n,
                       _oracle_params(oracle, cfg["k_max"]), tr)
    print("replay paper frame", res, "iters", gst["iters"])


def test_tracker_sequence_handoff_paper_scale(oracle, nat):
    """Five consecutive frames on the fixed 512^3 map, GPU poses fed forward: frame
    t starts at c_0 = s*_{t-1} with r_0 = r_1 of frame t-1 (Sec. 4, PST
    initialization), and every iteration of every frame is replayed."""
    import torch

    cfg, gv, ov, traj, K, depths = _paper_problem(oracle, nat)
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=cfg["k_max"], stride=cfg["stride"]), 640, 480)
    tr.set_scale([0.3] * 6)
    prev = pose_f32(traj[0])
    r0 = np.full(6, np.float32(0.3)).astype(np.float64)
    D = [torch.from_numpy(d).cuda() for d in depths]
    total = dict(rows=0, strict=0, loose=0)
    for f in range(1, 6):
        pose, gst, status = nat.pfo_track_frame(tr, D[f], D[f - 1], K, prev)
        assert status == 0
        pts = oracle.unproject(depths[f], K, cfg["stride"])
        res = _check_frame(oracle, ov, gst, pose, [(pts, n)], depths[f - 1], K, prev, prev, r0, n,
                           _oracle_params(oracle, cfg["k_max"]), tr)
        for key in total:
            total[key] += res[key]
        prev = np.asarray(pose, np.float64)
        r0 = np.asarray(gst["r1"], np.float64)
    print("replay paper sequence", total)
    assert total["rows"] >= 5


def _flat_problem(nat, value, f32_codes=True):
    """A 64^3 f32 volume (4 cm voxels) holding `value` everywhere (NaN = never
    observed) and an 80x60 frame of a wall 1.2 m in front of the camera, well
    inside the volume; frame t-1 is the same frame at the same pose."""
    dims, voxel = 64, 0.04
    gv = nat.Volume(dims, voxel, 0.12, (0, 0, 0), "f32")
    if value is not None:
        gv.upload(np.full((dims, dims, dims), value, np.float32))
    K = synth.intrinsics(80, 60)
    depth = np.full((60, 80), 1.2, np.float32)
    pose = np.array([1, 0, 0, 0, 1.28, 1.28, 0.6])
    return gv, K, depth, pose


@pytest.mark.parametrize("case", ["empty_aps", "no_tsdf"])
def test_tracker_corner_cases(oracle, nat, case):
    """Sec. 4 "PST update": on a constant volume no particle beats the centre (empty
    APS, sphere rescale r_hat = 2 (1 - rho) / sqrt(6) + eps); on a volume with no
    observed voxel no likelihood exists (rho = 0.5, v = 1, r_hat = 0.5 + eps).
    Either way the APS is empty twice and the frame stops after two iterations at
    c_0 (Sec. 4, convergence criteria); r_1 has a closed form."""
    import math

    import torch

    value = 0.3 if case == "empty_aps" else None
    gv, K, depth, pose = _flat_problem(nat, value)
    n = 256
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=10), 80, 60)
    r0 = np.float32([0.01, 0.012, 0.014, 0.016, 0.018, 0.02])
    tr.set_scale(r0)
    D = torch.from_numpy(depth).cuda()
    out, gst, status = nat.pfo_track_frame(tr, D, D, K, pose)
    assert status == 0 and gst["iters"] == 2 and gst["it"][1]["stop"] == 1
    np.testing.assert_array_equal(np.float32(out), np.float32(pose))
    if case == "empty_aps":
        rho = math.exp(-0.09)
        assert all(r["corner"] == 2 and r["n_aps"] == 0 for r in gst["it"])
        assert abs(gst["it"][0]["rho_max"] - rho) <= 1e-6
        rhat = 2 * (1 - gst["it"][0]["rho_max"]) / math.sqrt(6) + 1e-3
    else:
        assert all(r["corner"] == 1 and r["n_aps"] == 0 and r["rho_tilde"] == 0.5 for r in gst["it"])
        rhat = 0.5 + 1e-3
    r1 = 0.1 * r0.astype(np.float64) + 0.9 * rhat
    np.testing.assert_allclose(gst["r1"], r1, rtol=1e-6)
    np.testing.assert_allclose(gst["it"][1]["scale"], 0.1 * r1 + 0.9 * rhat, rtol=1e-6)
    # and the oracle, iteration by iteration
    ov = oracle.Volume((64,) * 3, 0.04, (0, 0, 0), 0.12)
    ov.F[:] = np.nan if value is None else np.float32(value)
    pts = oracle.unproject(depth, K, 1)
    _check_frame(oracle, ov, gst, out, [(pts, n)], depth, K, pose_f32(pose), pose_f32(pose), r0.astype(np.float64),
                 n, _oracle_params(oracle, 10), tr)


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
