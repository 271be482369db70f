"""Proposal-driven tracking through the C ABI: the extended frame call (a swarm
centre c_0 apart from the previous pose, caller-held axis lengths, iteration
cap, run flag) against the FP64 oracle's Algorithm 1 with the same
initialisation, and the learned driver (rf_learned_step): its proposal, its
short PFO run and its fallback rule.  Trace parity bar as in
test_gpu_tracker.py (every iteration replayed)."""
import numpy as np
import pytest

from gpu_common import analytic_volume_codes, oracle_volume, pose_f32, replay_trace
from oracle import mlp
from paper_2105_05600_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def oracle_params(oracle, k_max, flags=None):
    return dict(tau=1.0, beta=0.1, eps=1e-3, stop_eps=1e-6, k_max=k_max,
                flags=oracle.DEFAULT_FLAGS if flags is None else flags)


@pytest.fixture(scope="module")
def tiny(oracle, nat):
    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype="f32")
    traj = synth.make_trajectory(scene, 6, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    depths = [synth.render_depth(scene, p, K) for p in traj]
    return dict(scene=scene, codes=codes, F64=F64, cfg=cfg, traj=traj, K=K, depths=depths,
                ov=oracle_volume(oracle, cfg, F64))


def gpu_volume(nat, tiny):
    cfg = tiny["cfg"]
    gv = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), cfg["dtype"])
    gv.upload(tiny["codes"])
    return gv


def test_ex_async_with_a_separate_centre(oracle, nat, tiny):
    # With c_0 != s*_{t-1} the overlap test of iteration 1 already projects to
    # generic sub-pixel positions, where a rounding boundary within the parity
    # margin is likely; the trace is compared with the overlap test off (every
    # valid point scored), where no pixel rounding takes a decision.
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    gv = gpu_volume(nat, tiny)
    n, k_max = cfg["n_particles"], 6
    flags = nat.RF_NORMALIZE | nat.RF_COMPENSATED
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=20, stride=cfg["stride"], flags=flags), cfg["width"],
                     cfg["height"])
    prev = pose_f32(traj[0])
    # centre half way to the next pose (a proposal), axis lengths held by the caller
    c0 = pose_f32(oracle.compose_offset(prev, 0.5 * mlp.offset(prev, traj[1])))
    r0 = np.array([0.02, 0.02, 0.02, 0.05, 0.05, 0.05], np.float32)
    d1, d0 = (torch.from_numpy(tiny["depths"][i]).cuda() for i in (1, 0))
    t_prev = torch.from_numpy(prev.astype(np.float32)).cuda()
    t_c0 = torch.from_numpy(c0.astype(np.float32)).cuda()
    t_r = torch.from_numpy(r0).cuda()
    out = torch.zeros(7, dtype=torch.float32, device="cuda")
    st = nat.new_stats_buffer()
    nat.pfo_track_frame_ex_async(tr, d1, d0, K, t_prev, out, st, init_pose_dev=t_c0, scale_dev=t_r, k_max=k_max)
    gst = nat.stats_dict(nat.stats_from_device(st))
    assert gst["status"] == 0 and 1 <= gst["iters"] <= k_max
    pts = oracle.unproject(tiny["depths"][1], K, cfg["stride"])
    res = replay_trace(oracle, tiny["ov"], gst, [(pts, n)], tiny["depths"][0], K, prev, c0, r0.astype(np.float64),
                       oracle.pst_uniform(n, 1), oracle_params(oracle, k_max, flags))
    assert res["loose"] <= max(1, res["rows"] // 4), res
    # outputs: the last row's pose, r_1 = the first row's axis lengths
    np.testing.assert_array_equal(out.cpu().numpy(), np.float32(gst["it"][-1]["pose"]))
    np.testing.assert_array_equal(t_r.cpu().numpy(), np.float32(gst["it"][0]["scale"]))
    # the tracker's own r_0 buffer was not touched
    np.testing.assert_allclose(tr.get_scale(), np.ones(6))


def test_run_flag_skips_the_frame(nat, tiny):
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    gv = gpu_volume(nat, tiny)
    pst = nat.pst_create(cfg["n_particles"], seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=10, stride=cfg["stride"]), cfg["width"], cfg["height"])
    d1, d0 = (torch.from_numpy(tiny["depths"][i]).cuda() for i in (1, 0))
    prev = torch.from_numpy(pose_f32(traj[0]).astype(np.float32)).cuda()
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.full((7,), 7.0, dtype=torch.float32, device="cuda")
    r = torch.full((6,), 0.05, dtype=torch.float32, device="cuda")
    st = nat.new_stats_buffer()
    nat.pfo_track_frame_ex_async(tr, d1, d0, K, prev, out, st, scale_dev=r, run_flag_dev=flag)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == 7.0) and np.all(r.cpu().numpy() == np.float32(0.05))
    assert nat.stats_dict(nat.stats_from_device(st))["iters"] == 0
    # flag set: the same call runs, with the iteration cap
    flag.fill_(1)
    nat.pfo_track_frame_ex_async(tr, d1, d0, K, prev, out, st, scale_dev=r, run_flag_dev=flag, k_max=3)
    gst = nat.stats_dict(nat.stats_from_device(st))
    assert gst["status"] == 0 and 1 <= gst["iters"] <= 3
    assert np.all(np.isfinite(out.cpu().numpy())) and not np.all(out.cpu().numpy() == 7.0)


def zero_network_params(s_value):
    """A network whose output is mu = 0 and log scale s_value on every axis."""
    theta = np.zeros(mlp.n_params(), np.float32)
    b4 = mlp.unflatten(theta)[7]
    b4[6:12] = s_value
    return theta


def test_learned_step_with_a_constant_proposal(oracle, nat, tiny):
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    gv = gpu_volume(nat, tiny)
    n, k_l = cfg["n_particles"], 4
    pst = nat.pst_create(n, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=20, stride=cfg["stride"]), cfg["width"], cfg["height"])
    net = nat.MLP(16)
    s_val = np.log(0.3)
    net.set_params(zero_network_params(s_val))
    params = nat.proposal_params(k_learned=k_l, theta=-1.0, kappa=2.0)
    lp = nat.Learned(tr, gv, net, params, cfg["width"], cfg["height"])
    prev = pose_f32(traj[0])
    lp.start(tiny["depths"][0], K, prev)
    sb = nat.new_learned_stats_buffer()
    pose, status = lp.step(tiny["depths"][1], K, stats_dev=sb)
    s = nat.learned_stats_dict(sb)
    assert status == 0 and s["status"] == 0
    assert s["used_fallback"] == 0 and s["chose_fallback"] == 0 and 1 <= s["iters_learned"] <= k_l
    # the proposal: c_0 = s*_{t-1} (no previous motion at the first frame, mu = 0),
    # r_0 = kappa e^s units
    o = np.zeros(16)
    o[6:12] = np.float32(s_val)
    c0, r0 = mlp.proposal(o, np.zeros(6), prev, kappa=2.0)
    np.testing.assert_allclose(s["init_pose"], c0, atol=1e-6)
    np.testing.assert_allclose(s["r0"], r0, rtol=2e-6)
    # the short run is Algorithm 1 from that initialisation
    pts = oracle.unproject(tiny["depths"][1], K, cfg["stride"])
    res = tiny["ov"].pfo_frame(pts, tiny["depths"][0], K, prev, c0, r0.astype(np.float32).astype(np.float64),
                               oracle.pst_uniform(n, 1), oracle_params(oracle, k_l))
    assert res["iters"] == s["iters_learned"]
    if abs(res["trace"][-1][4] - s["rho_learned"]) <= 1e-4 * res["trace"][-1][4]:
        got = np.array(pose)
        if np.dot(got[:4], res["pose"][:4]) < 0:
            got[:4] = -got[:4]
        np.testing.assert_allclose(got, res["pose"], atol=2e-4)


def test_fallback_rule_and_graph_replay(nat, tiny):
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    runs = {}
    for use_graph in (False, True):
        gv = gpu_volume(nat, tiny)
        pst = nat.pst_create(cfg["n_particles"], seed=1)
        tr = nat.Tracker(gv, pst, nat.make_params(k_max=20, stride=cfg["stride"]), cfg["width"], cfg["height"])
        tr.set_scale([0.05] * 6)
        net = nat.MLP(16)
        net.set_params(zero_network_params(np.log(0.2)))
        # theta = 2: every frame after the first (rho_prev > 0) runs the fallback
        lp = nat.Learned(tr, gv, net, nat.proposal_params(k_learned=2, theta=2.0, resume=0), cfg["width"],
                         cfg["height"])
        lp.start(tiny["depths"][0], K, pose_f32(traj[0]))
        sb = nat.new_learned_stats_buffer()
        poses, stats = [], []
        for f in range(1, 5):
            pose, status = lp.step(tiny["depths"][f], K, use_graph=use_graph, stats_dev=sb)
            assert status == 0
            poses.append(pose)
            stats.append(nat.learned_stats_dict(sb))
        runs[use_graph] = (np.array(poses), stats)
    poses, stats = runs[False]
    assert stats[0]["used_fallback"] == 0  # no previous fitness yet
    for s in stats[1:]:
        assert s["used_fallback"] == 1 and s["iters_fallback"] >= 1
        assert s["rho_prev"] > 0
        assert s["chose_fallback"] == int(s["rho_fallback"] >= s["rho_learned"])  # a tie goes to the restart
        assert s["lookups"] > 0
    # graph replay gives the same frames bit for bit
    np.testing.assert_array_equal(runs[True][0], poses)
    assert [s["chose_fallback"] for s in runs[True][1]] == [s["chose_fallback"] for s in stats]


def test_off_map_proposal_restarts_plain(nat, tiny):
    """A proposal far outside the volume: the learned run's first iteration finds
    no TSDF sample for any particle (Sec. 4's first corner case, rho_tilde = 0.5),
    so the frame restarts plain PFO from s*_{t-1} with the carried r_1 even with
    theta = 0, and that run is kept; it equals the explicit extended-frame call."""
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    n, k_fb = cfg["n_particles"], 20
    prev = pose_f32(traj[0])
    r_carry = [0.05] * 6
    d0, d1 = (torch.from_numpy(tiny["depths"][f]).cuda() for f in (0, 1))
    params = nat.make_params(k_max=20, stride=cfg["stride"])
    theta = zero_network_params(np.log(0.3))
    mlp.unflatten(theta)[7][3] = 100.0  # mu_x = 100 units (10 m): c_0 beyond the 2.56 m volume
    net = nat.MLP(16)
    net.set_params(theta)

    gv = gpu_volume(nat, tiny)
    tr = nat.Tracker(gv, nat.pst_create(n, seed=1), params, cfg["width"], cfg["height"])
    tr.set_scale(r_carry)
    lp = nat.Learned(tr, gv, net, nat.proposal_params(k_learned=3, k_fallback=k_fb, theta=0.0), cfg["width"],
                     cfg["height"])
    lp.start(tiny["depths"][0], K, prev)
    sb = nat.new_learned_stats_buffer()
    pose, status = lp.step(tiny["depths"][1], K, stats_dev=sb)
    s = nat.learned_stats_dict(sb)
    assert status == 0 and s["status"] == 0
    assert abs(s["init_pose"][4] - (prev[4] + 10.0)) < 1e-3
    assert s["iters_learned"] >= 1 and s["rho_learned"] == 0.5
    assert s["used_fallback"] == 1 and s["chose_fallback"] == 1 and s["iters_fallback"] >= 1

    gv2 = gpu_volume(nat, tiny)
    nat.tsdf_integrate(gv2, d0, K, prev)
    tr2 = nat.Tracker(gv2, nat.pst_create(n, seed=1), params, cfg["width"], cfg["height"])
    prev_dev = torch.tensor(prev, dtype=torch.float32, device="cuda")
    pose_f = torch.zeros(7, dtype=torch.float32, device="cuda")
    st_f = nat.new_stats_buffer()
    nat.pfo_track_frame_ex_async(tr2, d1, d0, K, prev_dev, pose_f, st_f, init_pose_dev=prev_dev.clone(),
                                 scale_dev=torch.tensor(r_carry, dtype=torch.float32, device="cuda"), k_max=k_fb)
    sf = nat.stats_dict(nat.stats_from_device(st_f))
    assert s["iters_fallback"] == sf["iters"] and s["rho_fallback"] == sf["it"][-1]["rho_tilde"] > 0.5
    np.testing.assert_array_equal(np.asarray(pose, dtype=np.float32), pose_f.cpu().numpy())
    assert np.linalg.norm(np.asarray(pose[4:]) - traj[1][4:]) < 0.2  # back on the map, not 10 m away


def test_resume_continues_the_learned_run(nat, tiny):
    # theta = 0 never judges the proposal poor, so a learned run that used its one
    # iteration without converging is resumed from its own s* and axis lengths:
    # the step must equal the two explicit extended-frame calls it stands for.
    import torch

    cfg, K, traj = tiny["cfg"], tiny["K"], tiny["traj"]
    n, k_fb = cfg["n_particles"], 20
    prev = pose_f32(traj[0])
    d0, d1 = (torch.from_numpy(tiny["depths"][f]).cuda() for f in (0, 1))
    params = nat.make_params(k_max=20, stride=cfg["stride"])

    gv = gpu_volume(nat, tiny)
    tr = nat.Tracker(gv, nat.pst_create(n, seed=1), params, cfg["width"], cfg["height"])
    net = nat.MLP(16)
    net.set_params(zero_network_params(np.log(0.3)))
    lp = nat.Learned(tr, gv, net, nat.proposal_params(k_learned=1, k_fallback=k_fb, theta=0.0, resume=1, stuck=0),
                     cfg["width"], cfg["height"])
    lp.start(tiny["depths"][0], K, prev)
    sb = nat.new_learned_stats_buffer()
    pose, status = lp.step(tiny["depths"][1], K, stats_dev=sb)
    s = nat.learned_stats_dict(sb)
    assert status == 0 and s["iters_learned"] == 1

    # the same frame by hand: frame 0 fused at prev, the learned run, then the resumed run
    gv2 = gpu_volume(nat, tiny)
    nat.tsdf_integrate(gv2, d0, K, prev)
    tr2 = nat.Tracker(gv2, nat.pst_create(n, seed=1), params, cfg["width"], cfg["height"])
    prev_dev = torch.tensor(prev, dtype=torch.float32, device="cuda")
    c0 = torch.tensor(s["init_pose"], dtype=torch.float32, device="cuda")
    r = torch.tensor(s["r0"], dtype=torch.float32, device="cuda")
    pose_l = torch.zeros(7, dtype=torch.float32, device="cuda")
    st_l = nat.new_stats_buffer()
    nat.pfo_track_frame_ex_async(tr2, d1, d0, K, prev_dev, pose_l, st_l, init_pose_dev=c0, scale_dev=r, k_max=1)
    sl = nat.stats_dict(nat.stats_from_device(st_l))
    assert sl["iters"] == 1
    if sl["it"][0]["stop"] != 3:  # converged (small step) in one iteration: nothing to resume
        assert s["used_fallback"] == 0
        return
    assert s["used_fallback"] == 2
    r1 = torch.tensor(sl["it"][0]["scale"], dtype=torch.float32, device="cuda")
    pose_f = torch.zeros(7, dtype=torch.float32, device="cuda")
    st_f = nat.new_stats_buffer()
    nat.pfo_track_frame_ex_async(tr2, d1, d0, K, prev_dev, pose_f, st_f, init_pose_dev=pose_l.clone(),
                                 scale_dev=r1, k_max=k_fb)
    sf = nat.stats_dict(nat.stats_from_device(st_f))
    assert s["iters_fallback"] == sf["iters"] >= 1
    assert s["rho_fallback"] == sf["it"][-1]["rho_tilde"] and s["rho_learned"] == sl["it"][-1]["rho_tilde"]
    want = (pose_f if s["rho_fallback"] > s["rho_learned"] else pose_l).cpu().numpy().astype(np.float64)
    assert s["chose_fallback"] == int(s["rho_fallback"] > s["rho_learned"])
    np.testing.assert_array_equal(np.asarray(pose, dtype=np.float32), want.astype(np.float32))


def test_stuck_rule_resumes_from_the_proposal(nat):
    """A learned run whose every iteration has an empty APS never leaves c_0; with
    stuck = 1 the second run resumes PFO from c_0 with the carried r_1 of the
    Sec. 4 initialisation.  On a constant volume every APS is empty, so the
    learned run stops after two iterations at c_0, the second run starts there
    with the tracker's r_0 and also stops after two empty iterations.  (Frame 0
    is an all-invalid depth map, so fusing it leaves the volume constant; the
    overlap test is off, every valid point is scored.)"""
    import math

    from test_gpu_tracker import _flat_problem

    flags = nat.RF_NORMALIZE | nat.RF_COMPENSATED
    r_carry = np.float32([0.011, 0.012, 0.013, 0.021, 0.022, 0.023])
    net = nat.MLP(16)
    net.set_params(zero_network_params(np.log(0.3)))
    sb = nat.new_learned_stats_buffer()
    runs = {}
    for stuck in (1, 0):
        gv, K, depth, pose = _flat_problem(nat, 0.3)
        tr = nat.Tracker(gv, nat.pst_create(256, seed=1), nat.make_params(k_max=20, flags=flags), 80, 60)
        tr.set_scale(r_carry)
        params = nat.proposal_params(k_learned=5, k_fallback=20, theta=0.0, resume=1, stuck=stuck)
        lp = nat.Learned(tr, gv, net, params, 80, 60)
        lp.start(np.zeros_like(depth), K, pose)
        out, status = lp.step(depth, K, stats_dev=sb)
        runs[stuck] = (nat.learned_stats_dict(sb), out, status, pose)
    s, out, status, pose = runs[1]
    assert status == 0 and s["status"] == 0
    assert s["iters_learned"] == 2 and s["used_fallback"] == 3 and s["iters_fallback"] == 2
    # zero previous motion: c_0 = s*_{t-1}, and the kept pose is c_0 either way
    np.testing.assert_array_equal(np.float32(s["init_pose"]), np.float32(pose))
    np.testing.assert_array_equal(np.float32(out), np.float32(pose))
    assert abs(s["rho_fallback"] - math.exp(-0.09)) <= 1e-6
    # with stuck = 0 the learned run is kept and nothing else runs
    s0 = runs[0][0]
    assert s0["used_fallback"] == 0 and s0["iters_learned"] == 2 and s0["iters_fallback"] == 0
