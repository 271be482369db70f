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


def compare_traces(gst, otr, n_pts_margin=None):
    """Compare GPU stats rows with oracle trace rows; returns #iterations compared strictly."""
    strict = 0
    for k, (g, o) in enumerate(zip(gst["it"], otr)):
        ambiguous_overlap = o[27] < 1e-3
        ambiguous_aps = o[26] < 1e-5
        if not ambiguous_overlap:
            assert g["n_overlap"] == int(o[1]), (k, g["n_overlap"], o[1])
        else:
            assert abs(g["n_overlap"] - int(o[1])) <= 3
        if ambiguous_overlap or ambiguous_aps:
            break
        assert g["n_aps"] == int(o[2]), (k, g["n_aps"], o[2])
        assert abs(g["rho_ref"] - o[3]) <= 1e-4 * o[3]
        assert abs(g["rho_tilde"] - o[4]) <= 1e-4 * o[4]
        gp, op = np.array(g["pose"]), o[7:14]
        if np.dot(gp[:4], op[:4]) < 0:
            gp[:4] = -gp[:4]
        np.testing.assert_allclose(gp, op, atol=2e-4)
        np.testing.assert_allclose(g["scale"], o[14:20], rtol=2e-3, atol=2e-6)
        strict += 1
    return strict
