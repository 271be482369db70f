"""Pins for the oracle's TSDF sampling and fitness (Eq. normallh / Eq. ourlh):
trilinear interpolation reproduces linear fields exactly, a constant volume
gives rho = exp(-c^2), a plane at the true pose gives rho = 1 and a known
offset exp(-(delta/mu)^2), a binary volume sampled at voxel centres gives a
brute-force count, invalid samples weigh psi = 1 (reading 2)."""
import math

import numpy as np
import pytest


def make_vol(oracle, dims, voxel, origin, fill):
    v = oracle.Volume(dims, voxel, origin, trunc=1.0)
    dx, dy, dz = dims
    k, j, i = np.meshgrid(np.arange(dz), np.arange(dy), np.arange(dx), indexing="ij")
    v.F[:] = fill(i, j, k).reshape(-1)
    return v


def test_trilinear_reproduces_linear_field(oracle):
    dims, voxel, origin = (6, 5, 4), 0.1, np.array([-0.2, 0.1, 0.3])
    a, b, c, d = 0.05, -0.03, 0.07, -0.1
    v = make_vol(oracle, dims, voxel, origin, lambda i, j, k: a * i + b * j + c * k + d)
    rng = np.random.default_rng(0)
    for _ in range(200):
        g = rng.uniform(0, 1, size=3) * (np.array(dims) - 1)  # voxel-centre coordinates inside the grid
        p = origin + voxel * (g + 0.5)
        val = v.sample(p)
        assert val is not None
        assert abs(val - (a * g[0] + b * g[1] + c * g[2] + d)) < 1e-12
    # outside the span of the voxel centres the sample is invalid
    assert v.sample(origin + voxel * (np.array([-0.1, 1.0, 1.0]) + 0.5)) is None
    assert v.sample(origin + voxel * (np.array([1.0, 4.2, 1.0]) + 0.5)) is None  # y beyond dims[1]-1 = 4
    assert v.sample(origin + voxel * (np.array([1.0, 1.0, 3.01]) + 0.5)) is None  # z beyond dims[2]-1 = 3


def test_trilinear_axis_order_is_x_fastest(oracle):
    # a field varying along x only: swapping axes in the sampler would break this
    dims, voxel = (8, 3, 2), 0.5
    v = make_vol(oracle, dims, voxel, np.zeros(3), lambda i, j, k: 0.1 * i + 0.0 * j + 0.0 * k)
    assert abs(v.sample(voxel * (np.array([5.25, 0.5, 0.5]) + 0.5)) - 0.525) < 1e-12


def test_unobserved_corner_invalidates_neighbouring_cells(oracle):
    dims, voxel = (6, 6, 6), 0.25
    v = make_vol(oracle, dims, voxel, np.zeros(3), lambda i, j, k: 0.0 * i + 0.2)
    v.grid()[3, 3, 3] = np.nan
    for gx in (2.5, 3.5):
        assert v.sample(voxel * (np.array([gx, 3.2, 2.7]) + 0.5)) is None
    assert v.sample(voxel * (np.array([1.5, 3.2, 2.7]) + 0.5)) == pytest.approx(0.2, abs=1e-15)
    # nearest mode only needs its own voxel
    assert v.sample(voxel * (np.array([2.6, 3.2, 2.7]) + 0.5), flags=oracle.NEAREST) is None
    assert v.sample(voxel * (np.array([2.4, 3.2, 2.7]) + 0.5), flags=oracle.NEAREST) == pytest.approx(0.2)


def _points_in(rng, lo, hi, n):
    pts = np.zeros((n, 4))
    pts[:, :3] = rng.uniform(lo, hi, size=(n, 3))
    pts[:, 3] = 1
    return pts


def test_constant_volume_closed_form(oracle):
    c = 0.25
    v = make_vol(oracle, (8, 8, 8), 0.25, np.zeros(3), lambda i, j, k: 0.0 * i + c)
    pts = _points_in(np.random.default_rng(1), 0.3, 1.6, 500)
    ident = np.array([1, 0, 0, 0, 0, 0, 0], float)
    ones = np.ones(500, np.int32)
    S, n, nO, rho = v.fitness(pts, ones, ident)
    assert (n, nO) == (500, 500)
    assert S == pytest.approx(500 * c * c, rel=1e-12)
    assert rho == pytest.approx(math.exp(-c * c), rel=1e-12)
    S, _, _, rho = v.fitness(pts, ones, ident, flags=oracle.NORMALIZE | oracle.L1)
    assert rho == pytest.approx(math.exp(-c), rel=1e-12)
    S, _, _, rho = v.fitness(pts, ones, ident, tau=200.0, flags=0)  # Eq. ourlh: no normalisation
    assert rho == pytest.approx(math.exp(-500 * c * c / 200.0), rel=1e-12)
    S, _, _, rho = v.fitness(pts, ones, ident, tau=2.0)  # temperature
    assert rho == pytest.approx(math.exp(-c * c / 2.0), rel=1e-12)


def test_plane_true_pose_and_known_offset(oracle):
    # psi(p) = (z0 - z) / mu: a linear field, so trilinear sampling is exact.
    mu, voxel, z0 = 0.5, 0.1, 1.0
    dims = (20, 20, 20)
    v = make_vol(oracle, dims, voxel, np.zeros(3), lambda i, j, k: (z0 - voxel * (k + 0.5)) / mu + 0.0 * i)
    rng = np.random.default_rng(2)
    # a camera at (1, 1, 0.2) looking along +z (identity rotation); points on the plane z = z0
    T = np.array([1, 0, 0, 0, 1.0, 1.0, 0.2])
    world = np.column_stack([rng.uniform(0.6, 1.4, 300), rng.uniform(0.6, 1.4, 300), np.full(300, z0)])
    pts = np.zeros((300, 4))
    pts[:, :3] = world - T[4:]
    pts[:, 3] = 1
    ones = np.ones(300, np.int32)
    S, n, nO, rho = v.fitness(pts, ones, T)
    assert S < 1e-24 and rho == pytest.approx(1.0, abs=1e-15)
    for delta in (0.01, -0.03, 0.08):
        Td = T.copy()
        Td[6] += delta  # every point moves by delta along z: psi = -delta / mu
        S, n, nO, rho = v.fitness(pts, ones, Td)
        assert S == pytest.approx(300 * (delta / mu) ** 2, rel=1e-9)
        assert rho == pytest.approx(math.exp(-(delta / mu) ** 2), rel=1e-9)


def test_binary_volume_counts_points(oracle):
    # points exactly at voxel centres (power-of-two voxel: no rounding) sample their own voxel
    voxel = 0.25
    v = make_vol(oracle, (8, 8, 8), voxel, np.zeros(3), lambda i, j, k: (i >= 3).astype(float) + 0.0 * j)
    rng = np.random.default_rng(3)
    idx = rng.integers(0, 7, size=(400, 3))  # centres 0..6 in each axis (cell interior)
    pts = np.zeros((400, 4))
    pts[:, :3] = voxel * (idx + 0.5)
    pts[:, 3] = 1
    ident = np.array([1, 0, 0, 0, 0, 0, 0], float)
    S, n, nO, rho = v.fitness(pts, np.ones(400, np.int32), ident)
    assert S == float((idx[:, 0] >= 3).sum()) and n == 400
    # the in-set mask removes points from both the sum and |O|
    m = (np.arange(400) % 2).astype(np.int32)
    S2, n2, nO2, _ = v.fitness(pts, m, ident)
    assert nO2 == 200 and S2 == float(((idx[:, 0] >= 3) & (m == 1)).sum())


def test_invalid_samples_count_as_one(oracle):
    v = make_vol(oracle, (8, 8, 8), 0.25, np.zeros(3), lambda i, j, k: 0.0 * i + 0.1)
    pts = _points_in(np.random.default_rng(4), 5.0, 6.0, 50)  # far outside the volume
    S, n, nO, rho = v.fitness(pts, np.ones(50, np.int32), np.array([1, 0, 0, 0, 0, 0, 0], float))
    assert (S, n, nO) == (50.0, 0, 50) and rho == pytest.approx(math.exp(-1.0))
    v.grid()[:, :, 4:] = np.nan  # unobserved half
    pts2 = _points_in(np.random.default_rng(5), 0.2, 1.75, 300)
    S2, n2, _, _ = v.fitness(pts2, np.ones(300, np.int32), np.array([1, 0, 0, 0, 0, 0, 0], float))
    assert S2 == pytest.approx((300 - n2) * 1.0 + n2 * 0.01, rel=1e-12)
    assert 0 < n2 < 300
