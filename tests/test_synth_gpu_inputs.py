"""The device-side input generators of the synthetic module (used for large
training sets) reproduce the numpy generators: closed-form ray casting and the
analytic TSDF, evaluated with torch on the CPU here."""
import numpy as np
import pytest

from paper_2105_05600_gb300 import synth


def test_render_depth_batch_matches_render_depth():
    pytest.importorskip("torch")
    scene = synth.make_scene(5.12, 0.2, 3)
    traj = synth.make_trajectory(scene, 4, 4.0, 3.0, 3)
    K = synth.intrinsics(80, 60)
    got = synth.render_depth_batch(scene, traj, K, seed=1, noise=False, device="cpu").numpy()
    want = np.stack([synth.render_depth(scene, p, K) for p in traj])
    np.testing.assert_array_equal(got, want)
    noisy = synth.render_depth_batch(scene, traj, K, seed=1, noise=True, device="cpu").numpy()
    m = (want > 0) & (noisy > 0)
    z = want[m].astype(np.float64)
    # N(0, (1 mm z^2)^2): the normalised residual has unit spread
    r = (noisy[m] - want[m]) / (0.001 * z * z)
    assert abs(r.mean()) < 0.05 and abs(r.std() - 1.0) < 0.05


def test_analytic_tsdf_torch_matches_numpy():
    pytest.importorskip("torch")
    scene = synth.make_scene(1.28, 0.2, 5)
    a = synth.analytic_tsdf(scene.sdf, (32, 32, 32), 0.04, (0, 0, 0), 0.12, observed_band=0.12)
    b = synth.analytic_tsdf_torch(scene, (32, 32, 32), 0.04, (0, 0, 0), 0.12, observed_band=0.12,
                                  device="cpu").double().numpy()
    assert np.array_equal(np.isnan(a), np.isnan(b))
    np.testing.assert_allclose(b[~np.isnan(b)], a[~np.isnan(a)], atol=1e-7)


def test_substep_trajectory_keeps_the_motion_statistics():
    scene = synth.make_scene(5.12, 0.2, 7)
    t30 = synth.make_trajectory(scene, 301, 2.0, 1.0, 7)
    t60 = synth.make_trajectory(scene, 601, 2.0, 1.0, 7, fps=60.0, walk_sigma=0.05 / np.sqrt(2))
    s30 = np.linalg.norm(np.diff(t30[:, 4:], axis=0), axis=1)
    s60 = np.linalg.norm(np.diff(t60[::2, 4:], axis=0), axis=1)
    assert abs(np.median(s30) - 2.0 / 30) < 2e-3 and abs(np.median(s60) - 2.0 / 30) < 4e-3


def test_trajectory_speeds_and_scanning():
    # every frame turns by exactly ang_speed / fps and moves by speed / fps (unless
    # clipped at the camera box); the scanning bias keeps the optical axis on the
    # room's interior: the camera looks towards the centre far more often than a
    # plain random walk of the same seed, and stays inside the camera box
    scene = synth.make_scene(5.12, 0.2, 11)
    m = synth.camera_margin(scene)
    centre = 0.5 * (scene.lo + scene.hi)
    facing = {}
    for gain in (0.0, 3.0):
        tr = synth.make_trajectory(scene, 400, 2.0, 1.5, 11, scan_gain=gain)
        dq = np.abs(np.sum(tr[1:, :4] * tr[:-1, :4], axis=1))
        np.testing.assert_allclose(2 * np.arccos(np.minimum(1.0, dq)), 1.5 / 30, rtol=1e-6, atol=1e-7)
        step = np.linalg.norm(np.diff(tr[:, 4:], axis=0), axis=1)
        assert np.all(step <= 2.0 / 30 + 1e-12) and np.median(step) == pytest.approx(2.0 / 30)
        assert np.all(tr[:, 4:] >= scene.lo + m - 1e-12) and np.all(tr[:, 4:] <= scene.hi - m + 1e-12)
        z = np.stack([synth._qrot(q)[:, 2] for q in tr[:, :4]])
        to = centre - tr[:, 4:]
        far = np.linalg.norm(to, axis=1) > 0.5
        cosang = np.sum(z[far] * to[far], axis=1) / np.linalg.norm(to[far], axis=1)
        facing[gain] = float(np.mean(cosang > 0.0))
    assert facing[3.0] > 0.9 and facing[3.0] > facing[0.0] + 0.2
