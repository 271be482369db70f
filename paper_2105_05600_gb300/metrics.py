"""Trajectory metrics on the host (evaluation, not part of the tracking path).

ATE: the estimated camera positions are rigidly aligned to the ground truth
(Umeyama 1991 least-squares rotation + translation, no scale, via an SVD of the
3x3 cross-covariance) and the mean (the paper's Sec. 5.1 definition) and RMS of
the remaining position errors are reported.  TE (Eq. te) is the norm of the
translation of T_G^-1 T_E for one frame.
"""
from __future__ import annotations

import numpy as np


def _rot(q):
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                     [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                     [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def ate(est, gt):
    """(mean, rmse) in metres; est, gt: (T, 7) poses (q w,x,y,z then t)."""
    P = np.asarray(est, np.float64)[:, 4:7]
    Q = np.asarray(gt, np.float64)[:, 4:7]
    mp, mq = P.mean(0), Q.mean(0)
    C = (Q - mq).T @ (P - mp) / len(P)
    U, _, Vt = np.linalg.svd(C)
    S = np.eye(3)
    if np.linalg.det(U) * np.linalg.det(Vt) < 0:
        S[2, 2] = -1.0
    R = U @ S @ Vt
    err = np.linalg.norm((P - mp) @ R.T + mq - Q, axis=1)
    return float(err.mean()), float(np.sqrt((err ** 2).mean()))


def te(est, gt):
    """Eq. te for one frame."""
    est = np.asarray(est, np.float64)
    gt = np.asarray(gt, np.float64)
    return float(np.linalg.norm(_rot(gt[:4]).T @ (est[4:7] - gt[4:7])))


def rotation_error_deg(est, gt):
    """Angle of R_G^T R_E in degrees."""
    d = abs(float(np.dot(np.asarray(est)[:4], np.asarray(gt)[:4])))
    return float(np.degrees(2.0 * np.arccos(min(1.0, d))))
