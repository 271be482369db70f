"""Shared set-up for the GPU parity tests: seeded inputs from the synthetic
generators, handed identically to the CUDA path and to the FP64 oracle."""
import numpy as np

from paper_2105_05600_gb300 import synth

DTYPE_TOL = {"f32": 1e-4, "f16": 1e-4, "i16": 1e-4}  # relative tolerance on per-particle fitness


def analytic_volume_codes(cfg_name="tiny", dtype=None, dims=None):
    """(scene, codes (dz,dy,dx), F64 decoded values, cfg): a room TSDF sampled
    analytically and stored in the volume dtype; unobserved behind one
    truncation distance."""
    cfg = dict(synth.CONFIGS[cfg_name])
    if dims is not None:
        cfg["dims"] = dims
    if dtype is not None:
        cfg["dtype"] = dtype
    extent = cfg["dims"] * cfg["voxel"]
    scene = synth.make_scene(extent, cfg["wall_inset"], cfg["seed"])
    F = synth.analytic_tsdf(scene.sdf, (cfg["dims"],) * 3, cfg["voxel"], (0, 0, 0), cfg["trunc"],
                            observed_band=cfg["trunc"])
    codes = synth.encode_values(F, cfg["dtype"])
    return scene, codes, synth.decode_values(codes), cfg


def oracle_volume(oracle, cfg, F64):
    v = oracle.Volume((cfg["dims"],) * 3, cfg["voxel"], (0, 0, 0), cfg["trunc"])
    v.F[:] = F64.reshape(-1)
    return v


def frame_points(oracle, scene, cfg, pose, noise_seed=None):
    """Valid unprojected points (float32-rounded, as the GPU receives them) of a
    rendered frame, plus the depth image and intrinsics."""
    K = synth.intrinsics(cfg["width"], cfg["height"])
    rng = np.random.default_rng(noise_seed) if noise_seed is not None else None
    depth = synth.render_depth(scene, pose, K, rng)
    pts = oracle.unproject(depth, K, cfg["stride"])
    pts = pts[pts[:, 3] > 0].astype(np.float32).astype(np.float64)
    return pts, depth, K


def to_gpu_points(pts):
    import torch

    return torch.from_numpy(pts.astype(np.float32)).cuda().contiguous()


def pose_f32(p):
    """A pose as the GPU holds it (float32), back in float64 for the oracle."""
    return np.asarray(p, np.float64).astype(np.float32).astype(np.float64)


# FP32 error of one APS weight w_i = rho_i - rho_ref on the GPU (rho to ~1e-6
# absolute).  The oracle's trace columns T_SENS (all errors one way) and T_SENS2
# (independent errors, added in quadrature; errors proportional to the weights
# cancel in the normalised average) turn it into a bound on delta_bar.
EPS_W = 2e-6
RHO_RTOL = 1e-4  # per-particle fitness tolerance (relative)


def dbar_tolerance(o, oracle):
    return 1e-6 + min(EPS_W * o[oracle.T_SENS], 10 * EPS_W * o[oracle.T_SENS2])


def _aligned(q_gpu, q_ref):
    q = np.array(q_gpu, np.float64)
    if np.dot(q[:4], q_ref[:4]) < 0:
        q[:4] = -q[:4]
    return q


def gpu_state(row, k_next, empty_run):
    """The Algorithm 1 state the GPU holds after stats row `row` (float32 values)."""
    return dict(c=np.array(row["pose"], np.float64), r=np.array(row["scale"], np.float64),
                rho_carry=float(row["rho_tilde"]), empty_run=empty_run, k=k_next)


def replay_trace(oracle, ov, gst, levels, prev_depth, K, prev_pose, c0, r0, omega, params, threads=None):
    """Per-iteration parity of a GPU frame trace with the FP64 oracle.

    Iteration k of the GPU's stats is recomputed by one oracle iteration
    (or_pfo_step) started from the state the GPU itself reached after iteration
    k-1 (from c0, r0 at k = 1), so every iteration of the persistent kernel is
    checked, not only those before the first near-tie.  levels = [(points, n)]
    per multi-resolution level (one entry for the plain algorithm).
    Strict rows: |O_k|, |APS|, corner case, stop code, argmax (when the best two
    fitness values are apart) equal; rho_ref / rho_tilde / rho_max within
    RHO_RTOL; delta_bar, s*_k and r_k within the bound the oracle's weight
    sensitivity gives for EPS_W per weight.  A row may be loose only when the
    oracle reports a decision within its tie margin that the GPU took the other
    way: |O_k| differing by at most the fragile points, or |APS| by at most the
    tied candidates; the next row restarts from the GPU's state either way.
    Returns dict(rows, strict, loose, worst) (worst = largest error / tolerance)."""
    import os

    threads = threads or max(1, min(32, os.cpu_count() or 1))
    rows = gst["it"]
    assert len(rows) == gst["iters"] >= 1
    L = len(levels)
    state = dict(c=np.asarray(c0, np.float64), r=np.asarray(r0, np.float64), rho_carry=0.0, empty_run=0, k=1)
    strict = loose = 0
    worst = 0.0
    empty_run = 0
    for k, g in enumerate(rows, start=1):
        pts, n_l = levels[(k - 1) % L]
        stop, _, o = ov.pfo_step(pts, n_l, prev_depth, K, prev_pose, omega, params, state, centre_ref=L > 1,
                                 threads=threads)
        assert g["k"] == k and g["level"] == (k - 1) % L and g["n_particles"] == n_l
        ok = True
        if g["n_overlap"] != int(o[oracle.T_NO]):
            assert abs(g["n_overlap"] - int(o[oracle.T_NO])) <= int(o[oracle.T_FRAGILE_PX]), (k, g["n_overlap"], o[1])
            ok = False
        elif g["n_aps"] != int(o[oracle.T_NAPS]):
            assert abs(g["n_aps"] - int(o[oracle.T_NAPS])) <= int(o[oracle.T_TIES]), (k, g["n_aps"], o[2], o[36])
            ok = False
        if ok and int(o[oracle.T_STOP]) != 4:
            assert g["corner"] == int(o[oracle.T_CORNER]), (k, g["corner"], o[oracle.T_CORNER])
            for key, col in (("rho_ref", oracle.T_RHO_REF), ("rho_tilde", oracle.T_RHO_TILDE),
                             ("rho_max", oracle.T_RHO_MAX)):
                err = abs(g[key] - o[col])
                tol = RHO_RTOL * abs(o[col]) + 1e-7
                assert err <= tol, (k, key, g[key], o[col])
                worst = max(worst, err / tol)
            if o[oracle.T_RHO_MAX] - o[oracle.T_RHO_2ND] > 4e-6:
                assert g["argmax"] == int(o[oracle.T_ARGMAX]), (k, g["argmax"], o[oracle.T_ARGMAX])
            tol_d = dbar_tolerance(o, oracle)
            err = np.max(np.abs(np.array(g["offset"]) - o[oracle.T_DBAR]))
            assert err <= tol_d, (k, "delta_bar", err, tol_d)
            worst = max(worst, err / tol_d)
            # s*_k = c_{k-1} (+) delta_bar and r_k from Eq. rsinter / momentum, by the
            # oracle's own routines applied to the GPU's delta_bar and rho_tilde: tight
            c_prev = np.asarray(state["c"], np.float64)
            want = oracle.compose_offset(c_prev, np.asarray(g["offset"], np.float64), params["flags"])
            err = np.max(np.abs(_aligned(g["pose"], want) - want))
            assert err <= 2e-6, (k, "pose from delta_bar", err)
            err = np.max(np.abs(_aligned(g["pose"], o[oracle.T_POSE]) - o[oracle.T_POSE]))
            assert err <= 2e-6 + 2 * tol_d, (k, "pose", err, tol_d)
            beta, eps = params["beta"], params["eps"]
            r_prev = np.asarray(state["r"], np.float64)
            if g["corner"] == 0:
                _, _, _, r_want = oracle.pst_update([g["rho_tilde"]], np.asarray(g["offset"], np.float64),
                                                   g["rho_tilde"] - 1.0, r_prev, beta, eps)
            elif g["corner"] == 2:
                _, _, _, r_want = oracle.pst_update([0.0], np.zeros(6), g["rho_ref"], r_prev, beta, eps)
            else:
                r_want = beta * r_prev + (1 - beta) * (0.5 + eps)
            err_r = np.abs(np.array(g["scale"]) - r_want)
            assert np.all(err_r <= 1e-5 * np.abs(r_want) + 1e-7), (k, "scale", g["scale"], r_want)
            nv = np.linalg.norm(o[oracle.T_DBAR])
            dir_err = 2 * np.sqrt(6) * tol_d / nv if nv > 1e-9 else 2.0
            tol_r = 1e-7 + 1e-5 * np.abs(o[oracle.T_SCALE]) + (1 - beta) * (RHO_RTOL + dir_err)
            err_r = np.abs(np.array(g["scale"]) - o[oracle.T_SCALE])
            assert np.all(err_r <= tol_r), (k, "scale vs oracle", g["scale"], o[oracle.T_SCALE])
            worst = max(worst, float(np.max(err_r / tol_r)))
            if g["stop"] != int(o[oracle.T_STOP]):
                # only the small-step rule can flip, for a step at the threshold
                assert {g["stop"], int(o[oracle.T_STOP])} <= {0, 2, 3}, (k, g["stop"], o[oracle.T_STOP])
                assert abs(o[oracle.T_STEP] - params["stop_eps"]) <= tol_d, (k, o[oracle.T_STEP])
            strict += 1
        elif ok:
            assert g["stop"] == 4
            strict += 1
        else:
            loose += 1
        empty_run = empty_run + 1 if g["n_aps"] == 0 else 0
        state = gpu_state(g, k + 1, empty_run)
    last = rows[-1]
    assert last["stop"] != 0, "the GPU frame ended without a stop reason"
    assert len(rows) == params["k_max"] or last["stop"] in (1, 2, 4)
    return dict(rows=len(rows), strict=strict, loose=loose, worst=worst)
