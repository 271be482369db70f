"""Pins for the oracle's geometry: quaternions, MovePST composition, unprojection
(Eq. unproj) and the overlap set (Eq. validness).  Every expected value comes
from a textbook routine (Rodrigues' formula) or a closed form, never from the
oracle itself."""
import math

import numpy as np
import pytest


def rodrigues(axis, theta):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + math.sin(theta) * K + (1 - math.cos(theta)) * K @ K


def q_axis_angle(axis, theta):
    a = np.asarray(axis, float) / np.linalg.norm(axis)
    return np.concatenate([[math.cos(theta / 2)], math.sin(theta / 2) * a])


def test_quat_to_rot_matches_rodrigues(oracle):
    rng = np.random.default_rng(0)
    for _ in range(50):
        axis = rng.normal(size=3)
        theta = rng.uniform(-math.pi, math.pi)
        R = oracle.quat_to_rot(q_axis_angle(axis, theta))
        np.testing.assert_allclose(R, rodrigues(axis, theta), atol=1e-12)
    # 90 degrees about z maps x to y (catches a transposed matrix)
    R = oracle.quat_to_rot(q_axis_angle([0, 0, 1], math.pi / 2))
    np.testing.assert_allclose(R @ [1, 0, 0], [0, 1, 0], atol=1e-12)


def test_quat_mul_composes_rotations(oracle):
    rng = np.random.default_rng(1)
    for _ in range(20):
        a = q_axis_angle(rng.normal(size=3), rng.uniform(-3, 3))
        b = q_axis_angle(rng.normal(size=3), rng.uniform(-3, 3))
        ab = oracle.quat_mul(a, b)
        np.testing.assert_allclose(oracle.quat_to_rot(ab), oracle.quat_to_rot(a) @ oracle.quat_to_rot(b), atol=1e-12)
        conj = a * np.array([1, -1, -1, -1])
        np.testing.assert_allclose(oracle.quat_mul(a, conj), [1, 0, 0, 0], atol=1e-12)


def _random_pose(rng):
    q = q_axis_angle(rng.normal(size=3), rng.uniform(-2, 2))
    if q[0] < 0:
        q = -q
    return np.concatenate([q, rng.normal(size=3)])


def test_compose_offset_closed_forms(oracle):
    rng = np.random.default_rng(2)
    for _ in range(20):
        c = _random_pose(rng)
        Rc = oracle.quat_to_rot(c[:4])
        # zero offset is the centre itself
        np.testing.assert_allclose(oracle.compose_offset(c, np.zeros(6)), c, atol=1e-12)
        # a translation offset moves t only
        d = rng.normal(size=3) * 0.1
        out = oracle.compose_offset(c, np.concatenate([[0, 0, 0], d]))
        np.testing.assert_allclose(out[:4], c[:4], atol=1e-12)
        np.testing.assert_allclose(out[4:], c[4:] + d, atol=1e-12)
        # a rotation offset dq = sin(theta/2) axis rotates about the camera centre in world axes
        axis, theta = rng.normal(size=3), rng.uniform(-0.5, 0.5)
        dq = math.sin(theta / 2) * axis / np.linalg.norm(axis)
        out = oracle.compose_offset(c, np.concatenate([dq, [0, 0, 0]]))
        np.testing.assert_allclose(oracle.quat_to_rot(out[:4]), rodrigues(axis, theta) @ Rc, atol=1e-12)
        np.testing.assert_allclose(out[4:], c[4:], atol=1e-12)
        assert out[0] >= 0 and abs(np.linalg.norm(out[:4]) - 1) < 1e-12
        # RIGHT_MULT: T_c * T_delta
        out = oracle.compose_offset(c, np.concatenate([dq, d]), flags=oracle.RIGHT_MULT)
        np.testing.assert_allclose(oracle.quat_to_rot(out[:4]), Rc @ rodrigues(axis, theta), atol=1e-12)
        np.testing.assert_allclose(out[4:], c[4:] + Rc @ d, atol=1e-12)


def test_compose_offset_clamps_long_rotation(oracle):
    c = np.array([1, 0, 0, 0, 0, 0, 0], float)
    out = oracle.compose_offset(c, [3.0, 0, 0, 0, 0, 0])  # |dq| > 1 -> half-turn about x
    np.testing.assert_allclose(oracle.quat_to_rot(out[:4]), np.diag([1, -1, -1]), atol=1e-12)


def test_particle_pose_scaling(oracle):
    rng = np.random.default_rng(3)
    c = _random_pose(rng)
    om = rng.uniform(-0.4, 0.4, size=6)
    np.testing.assert_allclose(oracle.particle_pose(c, np.zeros(6), om), c, atol=1e-12)
    om_t = np.concatenate([[0, 0, 0], om[3:]])
    r = np.array([9, 9, 9, 0.5, 2.0, 0.25])
    out = oracle.particle_pose(c, r, om_t)
    np.testing.assert_allclose(out[4:], c[4:] + r[3:] * om[3:], atol=1e-12)


def _cam(W, H):
    return dict(fx=3.1, fy=2.6, cx=2.9, cy=1.7, z_min=0.1, z_max=8.0, width=W, height=H)


@pytest.mark.parametrize("stride", [1, 2, 3])
def test_unproject_reprojects_to_pixels(oracle, stride):
    W, H = 7, 5
    K = _cam(W, H)
    rng = np.random.default_rng(4)
    depth = rng.uniform(0.5, 3.0, size=(H, W)).astype(np.float32)
    depth[0, 2] = 0.0
    depth[1, 0] = 9.0  # beyond z_max
    depth[2, 2] = np.nan
    depth[4, 6] = 0.1  # not above z_min
    pts = oracle.unproject(depth, K, stride)
    nw, nh = -(-W // stride), -(-H // stride)
    assert pts.shape == (nw * nh, 4)
    for b in range(nh):
        for a in range(nw):
            p = pts[b * nw + a]
            u, v = a * stride, b * stride
            z = float(depth[v, u])
            if np.isfinite(z) and 0.1 < z <= 8.0:
                assert p[3] == 1.0 and p[2] == z
                assert abs(K["fx"] * p[0] / p[2] + K["cx"] - u) < 1e-12
                assert abs(K["fy"] * p[1] / p[2] + K["cy"] - v) < 1e-12
            else:
                assert list(p) == [0, 0, 0, 0]


def _plane_frame(W=40, H=30, z=2.0):
    K = dict(fx=20.0, fy=20.0, cx=19.5, cy=14.5, z_min=0.1, z_max=8.0, width=W, height=H)
    return K, np.full((H, W), z, np.float32)


def test_overlap_identity_keeps_all_valid(oracle):
    K, depth = _plane_frame()
    depth[3, 4] = 0.0
    pts = oracle.unproject(depth, K, 1)
    I = np.array([1, 0, 0, 0, 0, 0, 0], float)
    mask, margin, n = oracle.overlap(pts, depth, K, I, I)
    assert n == int((pts[:, 3] > 0).sum()) == 40 * 30 - 1
    assert np.array_equal(mask, (pts[:, 3] > 0).astype(np.int32))


def test_overlap_translation_shift(oracle):
    # Fronto-parallel plane at z = 2, the previous camera 0.3 m along +x: a point
    # lands fx * 0.3 / 2 = 3 px further left, so columns u < 3 fall outside.
    K, depth = _plane_frame()
    pts = oracle.unproject(depth, K, 1)
    cur = np.array([1, 0, 0, 0, 0, 0, 0], float)
    prev = np.array([1, 0, 0, 0, 0.3, 0, 0], float)
    mask, _, n = oracle.overlap(pts, depth, K, cur, prev)
    assert n == (40 - 3) * 30
    prev_depth = depth.copy()
    prev_depth[:, 10] = 0.0  # pixels of frame t-1 without depth drop the points mapping there (u = 13)
    mask2, _, n2 = oracle.overlap(pts, prev_depth, K, cur, prev)
    assert n2 == (40 - 3) * 30 - 30
    u = np.arange(len(pts)) % 40
    assert np.all(mask2[u == 13] == 0) and np.all(mask2[u == 14] == 1)


def test_overlap_cell_margin_hand_count(oracle):
    # cell_m = 0.225 m at z = 2 m and fx = fy = 20 px: a footprint of 2.25 px, so
    # u must lie in [1.75, 40 - 0.5 - 2.25) -> columns 2..37 (36), rows 2..27 (26)
    K, depth = _plane_frame()
    pts = oracle.unproject(depth, K, 1)
    I = np.array([1, 0, 0, 0, 0, 0, 0], float)
    mask, margin, n = oracle.overlap(pts, depth, K, I, I, cell_m=0.225)
    assert n == 36 * 26
    u, v = np.arange(len(pts)) % 40, np.arange(len(pts)) // 40
    assert np.array_equal(mask.astype(bool), (u >= 2) & (u <= 37) & (v >= 2) & (v <= 27))
    assert np.min(margin) == pytest.approx(0.25)  # u = 2 lies 0.25 px inside the inset edge 1.75
    # at z = 4 m the footprint halves (1.125 px): columns 1..38, rows 1..28
    K4, d4 = _plane_frame(z=4.0)
    p4 = oracle.unproject(d4, K4, 1)
    assert oracle.overlap(p4, d4, K4, I, I, cell_m=0.225)[2] == 38 * 28
    # with the 0.3 m shift of the previous camera (3 px), u - 3 must lie in [1.75, 37.25): columns 5..39
    prev = np.array([1, 0, 0, 0, 0.3, 0, 0], float)
    mask, _, n = oracle.overlap(pts, depth, K, I, prev, cell_m=0.225)
    assert n == 35 * 26
    assert np.all(mask[(u == 4)] == 0) and np.all(mask[(u == 5) & (v == 10)] == 1)


def test_overlap_behind_previous_camera(oracle):
    K, depth = _plane_frame()
    pts = oracle.unproject(depth, K, 1)
    cur = np.array([1, 0, 0, 0, 0, 0, 0], float)
    prev = np.concatenate([q_axis_angle([0, 1, 0], math.pi), [0, 0, 0]])  # looking the other way
    _, _, n = oracle.overlap(pts, depth, K, cur, prev)
    assert n == 0
