"""Pins for the oracle's volumetric fusion (Sec. 3 overview: Curless-Levoy /
KinectFusion running average of the truncated projective distance) and the
storage rounding of each dtype (reading 14)."""
import math

import numpy as np
import pytest

I_POSE = np.array([1, 0, 0, 0, 0, 0, 0], float)


def _setup(oracle, qmode="f64", w_max=255):
    # camera at the origin looking along +z, a 32x24 image with a wide field of view
    K = dict(fx=8.0, fy=8.0, cx=15.5, cy=11.5, z_min=0.1, z_max=8.0, width=32, height=24)
    v = oracle.Volume((16, 16, 16), 0.1, (-0.8, -0.8, 0.0), trunc=0.3, w_max=w_max, qmode=qmode)
    return K, v


def _centres(v):
    d = v.dims
    k, j, i = np.meshgrid(np.arange(d[2]), np.arange(d[1]), np.arange(d[0]), indexing="ij")
    return (v.origin[0] + v.voxel * (i + 0.5), v.origin[1] + v.voxel * (j + 0.5), v.origin[2] + v.voxel * (k + 0.5))


def test_fronto_parallel_plane(oracle):
    K, v = _setup(oracle)
    d = 1.0
    v.integrate(np.full((24, 32), d, np.float32), K, I_POSE)
    x, y, z = _centres(v)
    F = v.grid()
    W = v.W.reshape(F.shape)
    inside = (z >= 0.45) & (np.abs(x) <= 0.75) & (np.abs(y) <= 0.6)  # |x/z| <= 1.67 < 16/8, |y/z| <= 1.33 < 12/8
    band = inside & (d - z >= -0.3)
    expect = np.minimum(1.0, (d - z) / 0.3)
    np.testing.assert_allclose(F[band], expect[band], atol=1e-12)
    assert np.all(W[band] == 1)
    behind = inside & (d - z < -0.3)  # more than one truncation distance behind the surface: untouched
    assert np.all(np.isnan(F[behind])) and np.all(W[behind] == 0)
    assert np.all(W <= 1) and np.nanmax(np.abs(F)) <= 1.0


def test_running_average_and_weight(oracle):
    K, v = _setup(oracle)
    v.integrate(np.full((24, 32), 1.0, np.float32), K, I_POSE)
    v.integrate(np.full((24, 32), 1.1, np.float32), K, I_POSE)
    x, y, z = _centres(v)
    F = v.grid()
    W = v.W.reshape(F.shape)
    both = (z >= 0.45) & (np.abs(x) <= 0.75) & (np.abs(y) <= 0.6) & (1.0 - z >= -0.3)
    f1 = np.minimum(1.0, (1.0 - z) / 0.3)
    f2 = np.minimum(1.0, (float(np.float32(1.1)) - z) / 0.3)  # the depth image holds float32(1.1)
    np.testing.assert_allclose(F[both], 0.5 * (f1 + f2)[both], atol=1e-12)
    assert np.all(W[both] == 2)
    only2 = (z >= 0.45) & (np.abs(x) <= 0.75) & (np.abs(y) <= 0.6) & (1.0 - z < -0.3) & (1.1 - z >= -0.3)
    np.testing.assert_allclose(F[only2], f2[only2], atol=1e-12)
    assert np.all(W[only2] == 1)


def test_weight_saturates(oracle):
    K, v = _setup(oracle, w_max=3)
    for _ in range(5):
        v.integrate(np.full((24, 32), 1.0, np.float32), K, I_POSE)
    assert v.W.max() == 3


def test_pose_moves_the_surface(oracle):
    # the same depth seen from a camera 0.2 m further along +z puts the plane at z = 1.2
    K, v = _setup(oracle)
    v.integrate(np.full((24, 32), 1.0, np.float32), K, np.array([1, 0, 0, 0, 0, 0, 0.2]))
    x, y, z = _centres(v)
    F = v.grid()
    band = (z >= 0.65) & (np.abs(x) <= 0.75) & (np.abs(y) <= 0.6) & (1.2 - z >= -0.3)
    np.testing.assert_allclose(F[band], np.minimum(1.0, (1.2 - z) / 0.3)[band], atol=1e-12)


def test_storage_rounding(oracle):
    assert oracle.quantize(0.1, "f32") == float(np.float32(0.1))
    assert oracle.quantize(0.1, "f16") == float(np.float16(0.1))
    # int16 code round(F * 32767), ties to even: 0.5 * 32767 = 16383.5 -> 16384
    assert oracle.quantize(0.5, "i16") == 16384 / 32767
    assert oracle.quantize(-1.0, "i16") == -1.0
    assert oracle.quantize(2.0, "i16") == 1.0
    assert oracle.quantize(0.123456789, "f64") == 0.123456789


def test_int16_volume_holds_codes(oracle):
    K, v = _setup(oracle, qmode="i16")
    v.integrate(np.full((24, 32), 1.0, np.float32), K, I_POSE)
    F = v.F[np.isfinite(v.F)]
    codes = F * 32767
    np.testing.assert_allclose(codes, np.round(codes), atol=1e-9)
