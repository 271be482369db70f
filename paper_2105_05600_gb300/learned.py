"""Learned swarm proposal: training data from the plain tracker, training with the
library's network kernels, and proposal-driven tracking (include/rf_proposal.h).

Orchestration only -- seeds, loops and buffers.  Every arithmetic step of the
method runs in librosefusion's kernels: the plain PFO that labels the frames
(Algorithm 1 with the Sec. 4 initialisation), the feature and target kernels,
the network's forward / backward products and Adam, the proposal and the short
PFO run with its fallback.  Depth frames come from the synthetic input module.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import metrics, synth

LAYERS = [(256, 832), (256, 256), (256, 256), (16, 256)]  # (out, in) per layer
N_RES, N_USED_IN, N_USED_OUT = 768, 774, 12


# ----------------------------------------------------------------------------- inputs
def make_sequence(spec: dict, seed: int, n_frames: int, substeps: int = 1):
    """(scene, ground-truth trajectory, intrinsics, depth frames (F, H, W) float32
    on the device) of one seeded synthetic sequence at 30 Hz x substeps (the same
    motion statistics; F = (n_frames - 1) * substeps + 1)."""
    scene = synth.make_scene(spec["dims"] * spec["voxel"], spec["wall_inset"], seed)
    traj = synth.make_trajectory(scene, (n_frames - 1) * substeps + 1, spec["speed"], spec["ang_speed"], seed,
                                 fps=30.0 * substeps, walk_sigma=0.05 / math.sqrt(substeps))
    K = synth.intrinsics(spec["width"], spec["height"])
    depths = synth.render_depth_batch(scene, traj, K, seed=50_000 + seed, noise=spec.get("noise", True))
    return scene, traj, K, depths


def _tracker(nat, spec, k_max=None, flags=None):
    vol = nat.Volume(spec["dims"], spec["voxel"], spec["trunc"], (0, 0, 0), spec["dtype"])
    pst = nat.pst_create(spec["n_particles"], seed=1)
    params = nat.make_params(k_max=k_max or spec["k_max"], stride=spec["stride"],
                             flags=nat.RF_DEFAULT_FLAGS if flags is None else flags)
    tr = nat.Tracker(vol, pst, params, spec["width"], spec["height"])
    tr.set_scale(spec.get("r_first", [1.0] * 6))  # r_0 of the first tracked frame
    return vol, pst, tr


# ----------------------------------------------------------------------------- data
def generate_dataset(nat, spec: dict, seeds, n_frames: int, substeps: int = 2, group: int = 16,
                     use_graph: bool = True, start: str = "tracked", speeds=None):
    """Training pairs from the plain tracker (Algorithm 1 with the Sec. 4
    initialisation, fusion of every frame; up to `group` sequences per batched
    step).  The samples are the network input of (D_t, D_{t-1}, s_{t-2},
    s_{t-1}) and the target offset(s_{t-1}, s*_t), s*_t the pose the tracker
    converges to for frame t.
      start="tracked": each seeded sequence is rendered at 30 Hz x substeps and
        tracked frame by frame, which keeps its per-frame motion small enough to
        converge; s_{t} are the tracker's own poses at the 30 Hz frames
        (s_{-1} = s_0).
      start="truth": rendered at 30 Hz; each frame is tracked from the true pose
        of frame t-1 (one sequence at a time, pfo_track_frame_async) and the
        map is fused at the true poses, so s*_t is what plain PFO converges to
        from there on a correct map, and one failed frame does not spoil the
        frames after it; s_{t-1}, s_{t-2} are the true poses.
    Returns dict(X: (N, 832) bfloat16, Y: (N, 6) float32 on the device, seq: (N,)
    sequence index, tracked / truth: per-sequence 30 Hz poses, seconds)."""
    import torch

    if start == "truth":
        return _dataset_from_truth(nat, spec, seeds, n_frames, speeds)
    seeds = list(seeds)
    n_rows = len(seeds) * (n_frames - 1)
    X = torch.zeros((n_rows, 832), dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros((n_rows, 6), dtype=torch.float32, device="cuda")
    seq = np.zeros(n_rows, np.int64)
    tracked, truth = [], []
    t0 = time.perf_counter()
    row = 0
    F = (n_frames - 1) * substeps + 1
    for g0 in range(0, len(seeds), group):
        gs = seeds[g0:g0 + group]
        seqs = [make_sequence(spec, s, n_frames, substeps) for s in gs]
        objs = [_tracker(nat, spec) for _ in gs]
        batch = nat.Batch([o[2] for o in objs], [sq[2] for sq in seqs])
        n = len(gs)
        for i, sq in enumerate(seqs):
            batch.depth_slot(i, 0).copy_(sq[3][0])
        batch.start([sq[1][0] for sq in seqs])
        poses = torch.zeros((n, F, 7), dtype=torch.float32, device="cuda")
        for i in range(n):
            poses[i, 0].copy_(batch.pose_dev(i, 0))
        for f in range(1, F):
            par = f % 2
            for i, sq in enumerate(seqs):
                batch.depth_slot(i, par).copy_(sq[3][f])
            batch.step(par, use_graph=use_graph)
            for i in range(n):
                poses[i, f].copy_(batch.pose_dev(i, par))
        del batch, objs
        base = poses
        for i, sq in enumerate(seqs):
            K, D = sq[2], sq[3]
            for t in range(1, n_frames):
                a, b = (t - 1) * substeps, t * substeps
                c = max(a - substeps, 0)
                nat.rf_proposal_features(D[b], D[a], K, base[i, c], base[i, a], x_out=X[row])
                nat.rf_proposal_target(base[i, a], poses[i, b], y_out=Y[row])
                seq[row] = g0 + i
                row += 1
        torch.cuda.synchronize()
        sub = poses[:, ::substeps].cpu().numpy().astype(np.float64)
        tracked += [p for p in sub]
        truth += [sq[1][::substeps] for sq in seqs]
        del seqs
    return dict(X=X, Y=Y, seq=seq, tracked=tracked, truth=truth, seconds=time.perf_counter() - t0)


def _dataset_from_truth(nat, spec, seeds, n_frames, speeds=None):
    """generate_dataset(start="truth"): per sequence, frame 0 fused at its true
    pose; every frame t tracked by plain PFO from the true pose of frame t-1
    (with the tracker's carried r_1) and fused at its true pose.  speeds: an
    optional list of (m/s, rad/s) pairs taken in turn by the sequences (default:
    the spec's speed for all)."""
    import torch

    seeds = list(seeds)
    n_rows = len(seeds) * (n_frames - 1)
    X = torch.zeros((n_rows, 832), dtype=torch.bfloat16, device="cuda")
    Y = torch.zeros((n_rows, 6), dtype=torch.float32, device="cuda")
    seq = np.zeros(n_rows, np.int64)
    tracked, truth = [], []
    t0 = time.perf_counter()
    row = 0
    for si, s in enumerate(seeds):
        spec_s = spec if not speeds else dict(spec, speed=speeds[si % len(speeds)][0],
                                                ang_speed=speeds[si % len(speeds)][1])
        _, traj, K, D = make_sequence(spec_s, s, n_frames)
        vol, pst, tr = _tracker(nat, spec)
        gt = torch.as_tensor(traj, dtype=torch.float32, device="cuda")
        poses = torch.zeros_like(gt)
        poses[0].copy_(gt[0])
        nat.tsdf_integrate(vol, D[0], K, traj[0])
        for t in range(1, n_frames):
            nat.pfo_track_frame_async(tr, D[t], D[t - 1], K, gt[t - 1], poses[t], None)
            nat.tsdf_integrate_dev(vol, D[t], K, gt[t])
        for t in range(1, n_frames):
            nat.rf_proposal_features(D[t], D[t - 1], K, gt[max(t - 2, 0)], gt[t - 1], x_out=X[row])
            nat.rf_proposal_target(gt[t - 1], poses[t], y_out=Y[row])
            seq[row] = si
            row += 1
        torch.cuda.synchronize()
        tracked.append(poses.cpu().numpy().astype(np.float64))
        truth.append(traj)
        del vol, pst, tr, D
    return dict(X=X, Y=Y, seq=seq, tracked=tracked, truth=truth, seconds=time.perf_counter() - t0)


# ----------------------------------------------------------------------------- training
def init_params(seed: int) -> np.ndarray:
    """He-uniform weights on the used block of every layer (the output layer
    scaled by 0.1), zero biases, zero padding; the flat layout of rf_proposal.h."""
    rng = np.random.default_rng(seed)
    parts = []
    for l, (o, i) in enumerate(LAYERS):
        W = np.zeros((o, i), np.float32)
        rows = N_USED_OUT if l == 3 else o
        cols = N_USED_IN if l == 0 else i
        lim = math.sqrt(6.0 / cols) * (0.1 if l == 3 else 1.0)
        W[:rows, :cols] = rng.uniform(-lim, lim, size=(rows, cols))
        parts += [W.ravel(), np.zeros(o, np.float32)]
    return np.concatenate(parts)


def train(nat, X, Y, train_rows, val_rows, epochs: int = 30, batch: int = 512, lr: float = 1e-3,
          lr_final: float = 2e-5, seed: int = 0):
    """Adam on the mean + log-scale loss over train_rows (cosine learning-rate
    decay).  After every epoch the held-out rows give the loss and the squared
    error of the predicted offset; the network keeps the parameters of the epoch
    with the lowest offset error (the log-scale head overfits long before the
    offset does, so the loss itself would stop too early), then its scale head is
    calibrated on the held-out rows (rf_mlp_calibrate_scale).  Returns (MLP,
    history)."""
    import torch

    net = nat.MLP(batch)
    net.set_params(init_params(seed))
    tr_idx = torch.as_tensor(np.asarray(train_rows, np.int32), device="cuda")
    va_idx = torch.as_tensor(np.asarray(val_rows, np.int32), device="cuda")
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    per_epoch = len(train_rows) // batch
    total = epochs * per_epoch
    losses = torch.zeros(max(total, 1), dtype=torch.float32, device="cuda")
    hist = dict(train=[], val=[], val_offset_err=[])
    step = 0
    best, best_theta = float("inf"), None
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = tr_idx[torch.randperm(len(train_rows), generator=gen, device="cuda")]
        for b in range(per_epoch):
            a = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / max(total, 1)))
            net.train_step(X, Y, batch, a, idx=perm[b * batch:(b + 1) * batch].contiguous(),
                           loss_out=losses[step:step + 1])
            step += 1
        hist["train"].append(float(losses[step - per_epoch:step].mean().item()))
        hist["val"].append(validation_loss(net, X, Y, va_idx, batch))
        _, stats = net.evaluate(X, Y, idx=va_idx)
        hist["val_offset_err"].append(float(stats[0].item()))
        if hist["val_offset_err"][-1] < best:
            best, best_theta = hist["val_offset_err"][-1], net.get_params()
            hist["best_epoch"] = ep
    torch.cuda.synchronize()
    hist["seconds"] = time.perf_counter() - t0
    hist["steps"] = step
    if best_theta is not None:
        net.set_params(best_theta)
    hist["scale_calibration"] = net.calibrate_scale(X, Y, idx=va_idx)
    _, stats = net.evaluate(X, Y, idx=va_idx)
    hist["zero_offset_err"] = float(stats[7:13].sum().item())
    st = net.status()
    if st != 0:
        raise nat.RfError(st, "network kernels reported an error during training")
    return net, hist


def predict(net, X, Y, idx):
    """(mean offset mu = previous offset + correction (rows, 6), targets (rows, 6))
    of the dataset rows idx (rf_mlp_evaluate)."""
    mu, _ = net.evaluate(X, Y, idx=idx)
    return mu, Y[idx.long()]


def validation_loss(net, X, Y, va_idx, batch: int) -> float:
    tot, n = 0.0, 0
    for b in range(0, len(va_idx) - batch + 1, batch):
        _, loss, _ = net.gradient(X, Y, batch, idx=va_idx[b:b + batch].contiguous())
        tot += float(loss.item()) * batch
        n += batch
    return tot / max(n, 1)


# ----------------------------------------------------------------------------- evaluation
class _FrameTimer:
    """CUDA events around each timed frame (frames >= `warmup`); with `flush`
    (a device buffer larger than L2) the buffer is rewritten before each timed
    frame, outside the events."""

    def __init__(self, n, warmup=0, flush=None):
        import torch

        self.ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
        self.warmup, self.flush = warmup, flush

    def begin(self, f):
        if f > self.warmup:
            if self.flush is not None:
                self.flush.fill_(f & 0xFF)
            self.ev[f][0].record()

    def end(self, f):
        if f > self.warmup:
            self.ev[f][1].record()

    def seconds(self, n):
        return sum(self.ev[f][0].elapsed_time(self.ev[f][1]) for f in range(self.warmup + 1, n)) / 1e3


def run_plain(nat, spec, traj, K, depths, k_max=None, warmup=0, flush=None, flags=None):
    """Plain PFO over a sequence (rf_sequence_step).  Returns (poses, seconds of the
    frames after `warmup` measured with CUDA events, their lookups)."""
    import torch

    vol, pst, tr = _tracker(nat, spec, k_max, flags)
    nat.rf_sequence_start(tr, depths[0], K, traj[0])
    n = len(depths)
    out = torch.zeros((n, 7), dtype=torch.float32, device="cuda")
    pose_buf = torch.zeros(7, dtype=torch.float32, device="cuda")
    stats = nat.new_stats_buffer()
    lookups = torch.zeros(n, dtype=torch.int64, device="cuda")
    out[0] = torch.as_tensor(traj[0], dtype=torch.float32)
    tm = _FrameTimer(n, warmup, flush)
    torch.cuda.synchronize()
    for f in range(1, n):
        tm.begin(f)
        nat.rf_sequence_step(tr, depths[f], K, want_host_pose=False, out_pose_dev=pose_buf, stats_dev=stats)
        tm.end(f)
        out[f].copy_(pose_buf)
        lookups[f] = stats[16:24].view(torch.int64)[0]  # rf_frame_stats.lookups
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), tm.seconds(n), int(lookups[warmup + 1:].sum().item())


def run_learned(nat, spec, traj, K, depths, net, params, use_graph=True, warmup=0, flush=None):
    """Proposal-driven tracking over a sequence (rf_learned_step).  Returns dict(poses,
    seconds and lookups of the frames after `warmup`, fallback runs / kept, mean
    learned iterations, frames with a non-zero status)."""
    import torch

    vol, pst, tr = _tracker(nat, spec)
    lp = nat.Learned(tr, vol, net, params, spec["width"], spec["height"])
    lp.start(depths[0], K, traj[0])
    n = len(depths)
    out = torch.zeros((n, 7), dtype=torch.float32, device="cuda")
    out[0] = torch.as_tensor(traj[0], dtype=torch.float32)
    pose_buf = torch.zeros(7, dtype=torch.float32, device="cuda")
    sb = nat.new_learned_stats_buffer()
    rec = torch.zeros((n, sb.numel()), dtype=torch.uint8, device="cuda")
    tm = _FrameTimer(n, warmup, flush)
    torch.cuda.synchronize()
    for f in range(1, n):
        tm.begin(f)
        lp.step(depths[f], K, use_graph=use_graph, want_host_pose=False, out_pose_dev=pose_buf, stats_dev=sb)
        tm.end(f)
        out[f].copy_(pose_buf)
        rec[f].copy_(sb)
    torch.cuda.synchronize()
    st = [nat.learned_stats_dict(rec[f]) for f in range(1, n)]
    timed = st[warmup:]
    return dict(poses=out.cpu().numpy().astype(np.float64), seconds=tm.seconds(n),
                lookups=sum(s["lookups"] for s in timed), fallbacks=sum(s["used_fallback"] == 1 for s in st),
                resumed=sum(s["used_fallback"] == 2 for s in st), unstuck=sum(s["used_fallback"] == 3 for s in st),
                fallback_kept=sum(s["chose_fallback"] for s in st),
                iters=float(np.mean([s["iters_learned"] for s in st])),
                failed=sum(1 for s in st if s["status"] != 0))


def evaluate(nat, spec, seeds, n_frames, net, params, use_graph=True, warmup=0, flush=None, plain=True):
    """A/B on held-out sequences: plain PFO (spec k_max) against the learned
    proposal + k_learned iterations, same frames.  Per sequence: frames/s of the
    frames after `warmup`, ATE over all tracked frames, lookups, fallbacks
    (plain=False skips the plain arm; its entries are then placeholders)."""
    rows = []
    for s in seeds:
        _, traj, K, depths = make_sequence(spec, s, n_frames)
        if plain:
            pp, tp, lkp = run_plain(nat, spec, traj, K, depths, warmup=warmup, flush=flush)
        else:
            pp, tp, lkp = np.tile(traj[:1], (len(traj), 1)), 1.0, 0
        rl = run_learned(nat, spec, traj, K, depths, net, params, use_graph, warmup=warmup, flush=flush)
        ap, _ = metrics.ate(pp, traj)
        al, _ = metrics.ate(rl["poses"], traj)
        nf = n_frames - 1 - warmup
        rows.append(dict(seed=s, frames=nf, plain_s=tp, learned_s=rl["seconds"], plain_fps=nf / tp,
                         learned_fps=nf / rl["seconds"], plain_ate_cm=100 * ap, learned_ate_cm=100 * al,
                         plain_lookups=lkp, learned_lookups=rl["lookups"], fallbacks=rl["fallbacks"],
                         resumed=rl["resumed"], unstuck=rl["unstuck"],
                         fallback_kept=rl["fallback_kept"], learned_iters=rl["iters"], failed_frames=rl["failed"]))
    return rows
