"""fitness_eval_noalloc: the fitness entry point for callers that cannot let the
library allocate device memory (real-time loops that must not stall on the
allocator's device-wide synchronisation, hosts with a fixed memory budget).  It must give the same per-particle fitness as fitness_eval (within
the rel 1e-4 bar of the fitness parity tests) on two calls in a row, reject
sizes beyond its 32 MiB static scratch with an error, and work both in a fresh
process and after every other test.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2105_05600_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def _problem(nat, n, stride):
    import torch

    cfg = dict(synth.CONFIGS["tiny"])
    dims, voxel, trunc = cfg["dims"], cfg["voxel"], cfg["trunc"]
    scene = synth.make_scene(dims * voxel, cfg["wall_inset"], cfg["seed"])
    F = synth.analytic_tsdf(scene.sdf, (dims,) * 3, voxel, (0, 0, 0), trunc, observed_band=trunc)
    vol = nat.Volume(dims, voxel, trunc, (0, 0, 0), "i16")
    vol.upload(synth.encode_values(F, "i16"))
    traj = synth.make_trajectory(scene, 3, cfg["speed"], cfg["ang_speed"], cfg["seed"])
    K = synth.intrinsics(cfg["width"], cfg["height"])
    depth = torch.from_numpy(synth.render_depth(scene, traj[1], K)).cuda()
    pts = nat.rf_depth_to_points(depth, K, stride)
    pts = pts[pts[:, 3] > 0].contiguous()
    pst = nat.pst_create(n, seed=9)
    return vol, pts, pst, traj


def _check_same(a, b):
    rho_a, S_a, n_a = (t.cpu().numpy() for t in a)
    rho_b, S_b, n_b = (t.cpu().numpy() for t in b)
    np.testing.assert_allclose(rho_a, rho_b, rtol=1e-4)
    np.testing.assert_allclose(S_a, S_b, rtol=1e-4)
    np.testing.assert_array_equal(n_a, n_b)


def test_noalloc_matches_fitness_eval_twice(nat):
    vol, pts, pst, traj = _problem(nat, 3000, 1)
    params = nat.make_params()
    # two calls in a row with different centres and scales: the second must not
    # see anything the first left in the shared scratch
    for centre, scale in ((traj[0], [0.03] * 3 + [0.05] * 3), (traj[2], [0.01] * 3 + [0.02] * 3)):
        want = nat.fitness_eval(vol, pts, pst, centre, scale, params)
        got = nat.fitness_eval_noalloc(vol, pts, pst, centre, scale, params)
        _check_same(got, want)


def test_noalloc_rejects_oversized_problems(nat):
    vol, pts, pst, traj = _problem(nat, 64, 1)
    big_pst = nat.pst_create(60000, seed=1)
    import torch

    many = pts.repeat(40, 1).contiguous()  # ceil(m / 256) * 60000 * 12 B > 32 MiB
    with pytest.raises(nat.RfError):
        nat.fitness_eval_noalloc(vol, many, big_pst, traj[0], [0.02] * 6, nat.make_params())
    torch.cuda.synchronize()
    # and the library keeps working afterwards
    got = nat.fitness_eval_noalloc(vol, pts, pst, traj[0], [0.02] * 6, nat.make_params())
    _check_same(got, nat.fitness_eval(vol, pts, pst, traj[0], [0.02] * 6, nat.make_params()))
