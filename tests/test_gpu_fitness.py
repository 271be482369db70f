"""GPU fitness (Eq. normallh) against the FP64 oracle and closed forms, through
the C ABI (fitness_eval).  Bar: per-particle fitness within rel 1e-4; a
particle may differ by more only through samples whose validity flips within
1e-3 voxel of the FP64 position (counted by the oracle), each worth at most 1
in the sum."""
import math

import numpy as np
import pytest

from gpu_common import analytic_volume_codes, frame_points, oracle_volume, pose_f32, to_gpu_points

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def _gpu_volume(nat, cfg, codes):
    v = nat.Volume(cfg["dims"], cfg["voxel"], cfg["trunc"], (0, 0, 0), cfg["dtype"])
    v.upload(codes)
    return v


def _compare(oracle, ov, pts, pst_np, idx, centre, scale, flags, tau, rho, S, nv, rtol=1e-4):
    ones = np.ones(len(pts), np.int32)
    worst = 0.0
    for i in idx:
        pose = oracle.particle_pose(centre, scale, pst_np[:, i].astype(np.float64), flags)
        So, no, nO, rho_o, fr = ov.fitness_fragile(pts, ones, pose, tau=tau, flags=flags)
        assert nO == len(pts)
        assert abs(S[i] - So) <= rtol * So + 1e-6 * len(pts) + fr, (i, S[i], So, fr)
        assert abs(int(nv[i]) - no) <= fr, (i, nv[i], no, fr)
        if fr == 0:
            assert abs(rho[i] - rho_o) <= rtol * rho_o + 1e-30, (i, rho[i], rho_o)
            worst = max(worst, abs(S[i] - So) / max(So, 1e-30))
    return worst


@pytest.mark.parametrize("dtype", ["f32", "f16", "i16"])
def test_fitness_parity_tiny(oracle, nat, dtype):
    import torch

    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype=dtype)
    gv = _gpu_volume(nat, cfg, codes)
    ov = oracle_volume(oracle, cfg, F64)
    from paper_2105_05600_gb300 import synth

    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    pts, _, _ = frame_points(oracle, scene, cfg, traj[1])
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    pst_np = pst.cpu().numpy()
    np.testing.assert_array_equal(pst_np, oracle.pst_uniform(n, 1))
    centre = pose_f32(traj[0])
    scale = pose_f32([0.03, 0.03, 0.03, 0.05, 0.05, 0.05])[:6]
    params = nat.make_params(flags=nat.RF_DEFAULT_FLAGS)
    rho, S, nv = nat.fitness_eval(gv, to_gpu_points(pts), pst, centre, scale, params)
    torch.cuda.synchronize()
    _compare(oracle, ov, pts, pst_np, range(n), centre, scale, oracle.DEFAULT_FLAGS, 1.0, rho.cpu().numpy(),
             S.cpu().numpy(), nv.cpu().numpy())


@pytest.mark.parametrize("flags_name", ["nearest", "l1", "plain_sum", "right_mult", "no_normalize_tau"])
def test_fitness_parity_flags(oracle, nat, flags_name):
    from paper_2105_05600_gb300 import synth

    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype="i16")
    gv = _gpu_volume(nat, cfg, codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    pts, _, _ = frame_points(oracle, scene, cfg, traj[1])
    extra = {"nearest": nat.RF_NEAREST, "l1": nat.RF_L1, "plain_sum": -nat.RF_COMPENSATED,
             "right_mult": nat.RF_RIGHT_MULT, "no_normalize_tau": -nat.RF_NORMALIZE}[flags_name]
    flags = nat.RF_DEFAULT_FLAGS + extra
    tau = 2000.0 if flags_name == "no_normalize_tau" else 1.0
    n = 96
    pst = nat.pst_create(n, seed=5)
    centre = pose_f32(traj[0])
    scale = pose_f32([0.02, 0.04, 0.02, 0.05, 0.03, 0.05])[:6]
    rho, S, nv = nat.fitness_eval(gv, to_gpu_points(pts), pst, centre, scale,
                                  nat.make_params(tau=tau, flags=flags))
    rtol = 1e-4 if flags_name != "plain_sum" else 2e-4
    _compare(oracle, ov, pts, pst.cpu().numpy(), range(n), centre, scale, flags, tau, rho.cpu().numpy(),
             S.cpu().numpy(), nv.cpu().numpy(), rtol=rtol)


@pytest.mark.parametrize("m,n", [(1, 1), (1, 33), (257, 1), (300, 65), (4099, 31)])
def test_fitness_ragged_sizes(oracle, nat, m, n):
    from paper_2105_05600_gb300 import synth

    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype="f32")
    gv = _gpu_volume(nat, cfg, codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    pts, _, _ = frame_points(oracle, scene, cfg, traj[1])
    pts = np.resize(pts, (m, 4))
    pst = nat.pst_create(n, seed=3)
    centre = pose_f32(traj[0])
    scale = pose_f32([0.02] * 3 + [0.04] * 3)[:6]
    rho, S, nv = nat.fitness_eval(gv, to_gpu_points(pts), pst, centre, scale, nat.make_params())
    _compare(oracle, ov, pts, pst.cpu().numpy(), range(n), centre, scale, oracle.DEFAULT_FLAGS, 1.0,
             rho.cpu().numpy(), S.cpu().numpy(), nv.cpu().numpy())


@pytest.mark.parametrize("dtype,code,value", [("f32", 0.25, 0.25), ("f16", 0.25, 0.25), ("i16", 8192, 8192 / 32767)])
def test_constant_volume_closed_form(nat, dtype, code, value):
    import torch

    dims = 64
    codes = np.full((dims,) * 3, code, dtype={"f32": np.float32, "f16": np.float16, "i16": np.int16}[dtype])
    v = nat.Volume(dims, 0.05, 0.15, (0, 0, 0), dtype)
    v.upload(codes)
    rng = np.random.default_rng(0)
    pts = np.zeros((5000, 4), np.float32)
    pts[:, :3] = rng.uniform(-0.5, 0.5, size=(5000, 3))
    pst = nat.pst_create(300, seed=2)
    centre = [1, 0, 0, 0, 1.6, 1.6, 1.6]
    rho, S, nv = nat.fitness_eval(v, to_gpu_points(pts), pst, centre, [0.05] * 6, nat.make_params())
    torch.cuda.synchronize()
    assert np.all(nv.cpu().numpy() == 5000)
    np.testing.assert_allclose(S.cpu().numpy(), 5000 * value * value, rtol=1e-6)
    np.testing.assert_allclose(rho.cpu().numpy(), math.exp(-value * value), rtol=1e-6)


def test_binary_volume_counts_points(nat):
    # points at voxel centres (power-of-two voxel) with every particle on the centre (r = 0)
    dims, voxel = 64, 0.0625
    codes = np.zeros((dims,) * 3, np.float32)
    codes[:, :, 20:] = 1.0  # x index >= 20
    v = nat.Volume(dims, voxel, 0.2, (0, 0, 0), "f32")
    v.upload(codes)
    rng = np.random.default_rng(1)
    idx = rng.integers(1, 62, size=(3000, 3))
    pts = np.zeros((3000, 4), np.float32)
    pts[:, :3] = voxel * (idx + 0.5)
    pst = nat.pst_create(64, seed=4)
    rho, S, nv = nat.fitness_eval(v, to_gpu_points(pts), pst, [1, 0, 0, 0, 0, 0, 0], [0.0] * 6, nat.make_params())
    assert np.all(S.cpu().numpy() == float((idx[:, 0] >= 20).sum()))
    assert np.all(nv.cpu().numpy() == 3000)


def test_fitness_parity_paper_scale_sampled(oracle, nat):
    """512^3 int16 volume, 160x120 points of a noisy 640x480 frame, 20k particles:
    the GPU scores all of them; the oracle re-scores a sample one by one."""
    from paper_2105_05600_gb300 import synth

    scene, codes, F64, cfg = analytic_volume_codes("paper")
    gv = _gpu_volume(nat, cfg, codes)
    ov = oracle_volume(oracle, cfg, F64)
    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    pts, _, _ = frame_points(oracle, scene, cfg, traj[1], noise_seed=11)
    assert len(pts) > 15000
    n = cfg["n_particles"]
    pst = nat.pst_create(n, seed=1)
    centre = pose_f32(traj[0])
    scale = pose_f32([0.02, 0.02, 0.02, 0.04, 0.04, 0.04])[:6]
    rho, S, nv = nat.fitness_eval(gv, to_gpu_points(pts), pst, centre, scale, nat.make_params())
    rng = np.random.default_rng(7)
    idx = sorted(set([0, 1, n - 1] + list(rng.choice(n, 45, replace=False))))
    _compare(oracle, ov, pts, pst.cpu().numpy(), idx, centre, scale, oracle.DEFAULT_FLAGS, 1.0,
             rho.cpu().numpy(), S.cpu().numpy(), nv.cpu().numpy())
    assert np.all(np.isfinite(rho.cpu().numpy())) and rho.cpu().numpy().max() <= 1.0


def test_fitness_is_deterministic(nat):
    from paper_2105_05600_gb300 import synth

    scene, codes, F64, cfg = analytic_volume_codes("tiny", dtype="i16")
    gv = _gpu_volume(nat, cfg, codes)
    import oracle as o

    traj = synth.make_trajectory(scene, 2, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    pts, _, _ = frame_points(o, scene, cfg, traj[1])
    pst = nat.pst_create(1024, seed=1)
    a = nat.fitness_eval(gv, to_gpu_points(pts), pst, traj[0], [0.03] * 6, nat.make_params())[1].cpu().numpy()
    b = nat.fitness_eval(gv, to_gpu_points(pts), pst, traj[0], [0.03] * 6, nat.make_params())[1].cpu().numpy()
    np.testing.assert_array_equal(a, b)


def test_fitness_rejects_bad_arguments(nat):
    import torch

    v = nat.Volume(8, 0.1, 0.3, (0, 0, 0), "f32")
    pts = torch.zeros((4, 4), device="cuda")
    pst = nat.pst_create(4, seed=1)
    with pytest.raises(nat.RfError):
        nat.fitness_eval(v, pts[:0], pst, [1, 0, 0, 0, 0, 0, 0], [0.1] * 6, nat.make_params())
    with pytest.raises(nat.RfError):
        nat.fitness_eval(v, pts, pst, [1, 0, 0, 0, 0, 0, 0], [0.1] * 6, nat.make_params(tau=0.0))
