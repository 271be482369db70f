"""The per-iteration replay used by the GPU parity tests (gpu_common.replay_trace),
checked on the CPU: a trace that the oracle itself produced, stored in FP32 as
the GPU stores its statistics rows, passes; the same trace with one planted
mistake (a moved best state, a wrong axis length, a wrong APS count, a missing
stop reason) is rejected."""
import copy

import numpy as np
import pytest

from gpu_common import replay_trace
from paper_2105_05600_gb300 import synth
from test_oracle_pfo import _params, _scene_volume


def _as_gpu_stats(oracle, res, n):
    rows = []
    for o in res["trace"]:
        f = lambda x: [float(np.float32(v)) for v in np.atleast_1d(x)]
        rows.append(dict(k=int(o[oracle.T_K]), n_overlap=int(o[oracle.T_NO]), n_aps=int(o[oracle.T_NAPS]),
                         argmax=int(o[oracle.T_ARGMAX]), rho_ref=f(o[oracle.T_RHO_REF])[0],
                         rho_tilde=f(o[oracle.T_RHO_TILDE])[0], rho_max=f(o[oracle.T_RHO_MAX])[0],
                         rho_second=f(o[oracle.T_RHO_2ND])[0], pose=f(o[oracle.T_POSE]), scale=f(o[oracle.T_SCALE]),
                         offset=f(o[oracle.T_DBAR]), stop=int(o[oracle.T_STOP]), level=int(o[oracle.T_LEVEL]),
                         n_particles=int(o[oracle.T_NL]), corner=int(o[oracle.T_CORNER])))
    return dict(iters=res["iters"], status=res["status"], it=rows, r1=[float(np.float32(v)) for v in res["r1"]])


def _frame(oracle):
    scene, v = _scene_volume(oracle)
    K = synth.intrinsics(40, 30)
    eye = np.array([0.72, 0.70, 0.68])
    T = np.concatenate([synth.look_at_quat(eye, [1.5, 1.45, 1.5]), eye])
    depth = synth.render_depth(scene, T, K)
    c0 = oracle.compose_offset(T, [0.010, -0.015, 0.012, 0.02, -0.01, 0.015]).astype(np.float32).astype(np.float64)
    pts = oracle.unproject(depth, K, 1)
    return v, K, depth, c0, pts


@pytest.fixture(scope="module")
def run(oracle):
    v, K, depth, c0, pts = _frame(oracle)
    n = 400
    omega = oracle.pst_uniform(n, 1)
    p = _params(oracle, flags=oracle.DEFAULT_FLAGS, k_max=12)
    r0 = np.full(6, np.float32(0.05)).astype(np.float64)
    res = v.pfo_frame(pts, depth, K, c0, c0, r0, omega, p)
    assert res["iters"] >= 4
    return v, K, depth, c0, pts, n, omega, p, r0, res


def test_replay_accepts_the_oracles_own_trace(oracle, run):
    v, K, depth, c0, pts, n, omega, p, r0, res = run
    gst = _as_gpu_stats(oracle, res, n)
    out = replay_trace(oracle, v, gst, [(pts, n)], depth, K, c0, c0, r0, omega, p, threads=2)
    assert out["rows"] == res["iters"] and out["loose"] == 0 and out["strict"] == out["rows"]
    assert out["worst"] < 0.5


@pytest.mark.parametrize("mistake", ["pose", "scale", "n_aps", "stop", "rho_tilde", "offset"])
def test_replay_rejects_a_planted_mistake(oracle, run, mistake):
    v, K, depth, c0, pts, n, omega, p, r0, res = run
    gst = _as_gpu_stats(oracle, res, n)
    bad = copy.deepcopy(gst)
    row = bad["it"][2]
    if mistake == "pose":
        row["pose"][5] += 1e-3
    elif mistake == "scale":
        row["scale"][1] *= 1.01
    elif mistake == "n_aps":
        row["n_aps"] += 3
    elif mistake == "stop":
        bad["it"][-1]["stop"] = 0
    elif mistake == "rho_tilde":
        row["rho_tilde"] *= 1.001
    else:
        row["offset"][0] += 1e-4
    with pytest.raises(AssertionError):
        replay_trace(oracle, v, bad, [(pts, n)], depth, K, c0, c0, r0, omega, p, threads=2)
