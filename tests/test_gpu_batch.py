"""Multi-resolution PST alternation (Sec. 4) and batched sequences in one
persistent kernel, through the C ABI.

* multi-resolution: every iteration (level, particles, |O_k|, |APS|, best
  state, axis lengths) replayed by the FP64 oracle's one-iteration step;
* batch: the first frame of every sequence of a batch (different volumes,
  frame sizes, particle counts, schedules, iteration limits), stepped in one
  persistent launch, is replayed by the oracle iteration by iteration, with
  and without CUDA-graph replay and with the autotuned launch and work split;
  stepping several sequences together gives bit for bit the poses and
  statistics of each sequence stepped alone; one sequence with an empty
  overlap set does not disturb the others."""
import numpy as np
import pytest

from gpu_common import analytic_volume_codes, oracle_volume, pose_f32, replay_trace
from paper_2105_05600_gb300 import synth
from test_gpu_tracker import _oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def test_multires_parity_tiny(oracle, nat):
    import torch

    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype="i16")
    gv = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), "i16")
    gv.upload(codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    d0 = synth.render_depth(scene, traj[0], K)
    d1 = synth.render_depth(scene, traj[1], K)
    levels_n, levels_s = [256, 512, 1024], [3, 2, 1]
    pst = nat.pst_create(1024, seed=1)
    tr = nat.Tracker(gv, pst, nat.make_params(k_max=9), cfg["width"], cfg["height"])
    tr.set_schedule(levels_n, levels_s)
    tr.set_scale([0.1] * 6)
    prev = pose_f32(traj[0])
    pose, gst, status = nat.pfo_track_frame(tr, torch.from_numpy(d1).cuda(), torch.from_numpy(d0).cuda(), K, prev)
    assert status == 0
    sets = [oracle.unproject(d1, K, s) for s in levels_s]
    res = replay_trace(oracle, ov, gst, list(zip(sets, levels_n)), d0, K, prev, prev, np.full(6, np.float32(0.1)),
                       oracle.pst_uniform(1024, 1), _oracle_params(oracle, 9))
    assert res["loose"] <= max(1, res["rows"] // 4), res
    assert gst["lookups"] == sum(r["n_overlap"] * r["n_particles"] for r in gst["it"])


def _sequences(nat, specs):
    """Per spec: (volume, tracker, intrinsics, depth frames, poses)."""
    out = []
    for sp in specs:
        dims, voxel, trunc = sp["dims"], sp["voxel"], 3 * sp["voxel"]
        scene = synth.make_scene(dims * voxel, 0.2, sp["seed"])
        traj = synth.make_trajectory(scene, sp["frames"], 1.5, 1.5, sp["seed"])
        K = synth.intrinsics(sp["w"], sp["h"])
        depths = [synth.render_depth(scene, traj[f], K) for f in range(sp["frames"])]
        vol = nat.Volume(dims, voxel, trunc, (0, 0, 0), "i16")
        pst = nat.pst_create(sp["n"], seed=sp["seed"] + 1)
        tr = nat.Tracker(vol, pst, nat.make_params(k_max=sp["k_max"], stride=sp["stride"]), sp["w"], sp["h"])
        if "levels" in sp:
            tr.set_schedule(*sp["levels"])
        out.append(dict(vol=vol, tr=tr, K=K, depths=depths, traj=traj, pst=pst))
    return out


SPECS = [dict(dims=64, voxel=0.04, w=80, h=60, n=1024, k_max=8, stride=1, seed=0, frames=4),
         dict(dims=96, voxel=0.03, w=96, h=72, n=700, k_max=3, stride=2, seed=1, frames=4),
         dict(dims=64, voxel=0.05, w=64, h=48, n=1500, k_max=9, stride=1, seed=2, frames=4,
              levels=([256, 700, 1500], [3, 2, 1]))]


def _run_alone(nat, specs):
    import torch

    poses, stats = [], []
    for s in _sequences(nat, specs):
        nat.rf_sequence_start(s["tr"], torch.from_numpy(s["depths"][0]).cuda(), s["K"], s["traj"][0])
        ps, ss = [], []
        for f in range(1, len(s["depths"])):
            sd = nat.new_stats_buffer()
            p, st = nat.rf_sequence_step(s["tr"], torch.from_numpy(s["depths"][f]).cuda(), s["K"], stats_dev=sd)
            ps.append(p)
            ss.append(nat.stats_dict(nat.stats_from_device(sd)))
        poses.append(ps)
        stats.append(ss)
    return poses, stats


def _run_batch(nat, specs, use_graph, autotune=False, blank=None):
    import torch

    seqs = _sequences(nat, specs)
    b = nat.Batch([s["tr"] for s in seqs], [s["K"] for s in seqs])
    for i, s in enumerate(seqs):
        b.depth_slot(i, 0).copy_(torch.from_numpy(s["depths"][0]).cuda())
    b.start([s["traj"][0] for s in seqs])
    poses = [[] for _ in seqs]
    stats = [[] for _ in seqs]
    chosen = None
    for f in range(1, len(seqs[0]["depths"])):
        parity = f % 2
        for i, s in enumerate(seqs):
            d = torch.from_numpy(s["depths"][f]).cuda()
            if blank is not None and i == blank:
                d.zero_()
            b.depth_slot(i, parity).copy_(d)
        if autotune and f == 1:
            chosen = b.autotune(parity)
        b.step(parity, use_graph=use_graph)
        torch.cuda.synchronize()
        for i, st in enumerate(b.stats()):
            poses[i].append(b.pose_dev(i, parity).cpu().numpy().astype(np.float64))
            stats[i].append(st)
    return poses, stats, chosen


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_sequences_alone(nat, use_graph):
    pa, sa = _run_alone(nat, SPECS)
    pb, sb, _ = _run_batch(nat, SPECS, use_graph)
    for i in range(len(SPECS)):
        for f in range(len(pa[i])):
            np.testing.assert_array_equal(pa[i][f], pb[i][f])
            assert sa[i][f] == sb[i][f]


def _analytic_batch(oracle, nat, specs, use_graph, autotune):
    """Each spec's volume holds its room's analytic TSDF (also given to the oracle);
    frame 0 is fused as an all-invalid depth map, which changes no voxel, so the
    first batched frame (overlap test off: every valid point scored) runs on
    exactly the oracle's volume."""
    import torch

    flags = nat.RF_NORMALIZE | nat.RF_COMPENSATED
    seqs, ovs = [], []
    for sp in specs:
        dims, voxel, trunc = sp["dims"], sp["voxel"], 3 * sp["voxel"]
        scene = synth.make_scene(dims * voxel, 0.2, sp["seed"])
        F = synth.analytic_tsdf(scene.sdf, (dims,) * 3, voxel, (0, 0, 0), trunc, observed_band=trunc)
        codes = synth.encode_values(F, "i16")
        vol = nat.Volume(dims, voxel, trunc, (0, 0, 0), "i16")
        vol.upload(codes)
        ov = oracle.Volume((dims,) * 3, voxel, (0, 0, 0), trunc)
        ov.F[:] = synth.decode_values(codes).reshape(-1)
        traj = synth.make_trajectory(scene, 2, 1.5, 1.5, sp["seed"])
        K = synth.intrinsics(sp["w"], sp["h"])
        pst = nat.pst_create(sp["n"], seed=sp["seed"] + 1)
        tr = nat.Tracker(vol, pst, nat.make_params(k_max=sp["k_max"], stride=sp["stride"], flags=flags), sp["w"],
                         sp["h"])
        tr.set_scale([0.05] * 6)
        levels = sp.get("levels", ([sp["n"]], [sp["stride"]]))
        if "levels" in sp:
            tr.set_schedule(*sp["levels"])
        seqs.append(dict(vol=vol, tr=tr, K=K, traj=traj, depth1=synth.render_depth(scene, traj[1], K), levels=levels,
                         seed=sp["seed"], n=sp["n"], k_max=sp["k_max"]))
        ovs.append(ov)
    b = nat.Batch([s["tr"] for s in seqs], [s["K"] for s in seqs])
    for i, s in enumerate(seqs):
        b.depth_slot(i, 0).zero_()
    b.start([pose_f32(s["traj"][0]) for s in seqs])
    for i, s in enumerate(seqs):
        b.depth_slot(i, 1).copy_(torch.from_numpy(s["depth1"]).cuda())
    chosen = b.autotune(1) if autotune else None
    b.step(1, use_graph=use_graph)
    torch.cuda.synchronize()
    stats = b.stats()
    for i, s in enumerate(seqs):
        gst = stats[i]
        assert gst["status"] == 0
        sets = [(oracle.unproject(s["depth1"], s["K"], st), n_l) for n_l, st in zip(*s["levels"])]
        prev = pose_f32(s["traj"][0])
        res = replay_trace(oracle, ovs[i], gst, sets, np.zeros((s["K"]["height"], s["K"]["width"]), np.float32),
                           s["K"], prev, prev, np.full(6, np.float32(0.05)), oracle.pst_uniform(s["n"], s["seed"] + 1),
                           _oracle_params(oracle, s["k_max"], flags))
        assert res["loose"] <= max(1, res["rows"] // 4), (i, res)
        np.testing.assert_array_equal(b.pose_dev(i, 1).cpu().numpy(), np.float32(gst["it"][-1]["pose"]))
    return chosen


@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_first_frame_matches_oracle(oracle, nat, use_graph):
    _analytic_batch(oracle, nat, SPECS, use_graph, autotune=False)


def test_batch_autotuned_matches_oracle(oracle, nat):
    chosen = _analytic_batch(oracle, nat, SPECS, use_graph=True, autotune=True)
    assert chosen["ctas_per_sm"] >= 1 and chosen["ms"] > 0 and chosen["group"] in (4, 6, 8)


def test_batch_with_an_empty_sequence(nat):
    pa, sa = _run_alone(nat, SPECS)
    pb, sb, _ = _run_batch(nat, SPECS, use_graph=False, blank=1)
    assert all(st["status"] == nat.RF_ERR_EMPTY for st in sb[1])
    for i in (0, 2):
        for f in range(len(pa[i])):
            np.testing.assert_array_equal(pa[i][f], pb[i][f])
