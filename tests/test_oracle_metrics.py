"""Pins for the oracle's ATE (Sec. 5.1, mean error after rigid alignment) and TE
(Eq. te), and a cross-check of the host metrics module against them."""
import math

import numpy as np
import pytest


def _traj(rng, T=40):
    out = np.zeros((T, 7))
    for f in range(T):
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        th = rng.uniform(-1, 1)
        out[f, :4] = [math.cos(th / 2), *(math.sin(th / 2) * a)]
        out[f, 4:] = rng.normal(size=3)
    return out


def test_ate_zero_for_rigidly_moved_copy(oracle):
    rng = np.random.default_rng(0)
    gt = _traj(rng)
    ax = np.array([0.3, -0.5, 0.8])
    th = 0.9
    K = np.array([[0, -ax[2], ax[1]], [ax[2], 0, -ax[0]], [-ax[1], ax[0], 0]]) / np.linalg.norm(ax)
    R = np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    est = gt.copy()
    est[:, 4:] = gt[:, 4:] @ R.T + np.array([1.0, -2.0, 0.5])
    mean, rmse = oracle.ate(est, gt)
    assert mean < 1e-9 and rmse < 1e-9


def test_ate_scaled_square(oracle):
    # corners of a square of half-width 1 scaled by 1.1 about its centre: the
    # best rigid fit is the identity and every corner is off by 0.1 * sqrt(2)
    gt = np.zeros((4, 7))
    gt[:, 0] = 1
    gt[:, 4:6] = [[1, 1], [-1, 1], [-1, -1], [1, -1]]
    est = gt.copy()
    est[:, 4:] *= 1.1
    mean, rmse = oracle.ate(est, gt)
    assert mean == pytest.approx(0.1 * math.sqrt(2), rel=1e-12)
    assert rmse == pytest.approx(0.1 * math.sqrt(2), rel=1e-12)


def test_te(oracle):
    gt = np.array([math.cos(0.3), 0, math.sin(0.3), 0, 1.0, 2.0, 3.0])
    assert oracle.te(gt, gt) == 0.0
    est = gt.copy()
    est[4:] += [3.0, 4.0, 0.0]
    assert oracle.te(est, gt) == pytest.approx(5.0, rel=1e-14)


def test_host_metrics_agree_with_oracle(oracle):
    from paper_2105_05600_gb300 import metrics

    rng = np.random.default_rng(1)
    gt = _traj(rng, 60)
    est = gt.copy()
    est[:, 4:] += rng.normal(size=(60, 3)) * 0.02
    m1, r1 = metrics.ate(est, gt)
    m2, r2 = oracle.ate(est, gt)
    assert m1 == pytest.approx(m2, rel=1e-9) and r1 == pytest.approx(r2, rel=1e-9)
    assert metrics.te(est[3], gt[3]) == pytest.approx(oracle.te(est[3], gt[3]), rel=1e-12)
