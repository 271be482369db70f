"""What the trained network gains over the method without it, on a small version
of the learned workload (4 m/s + 3 rad/s, 10k particles; own-kernel training on
~1,200 samples whose labels are plain PFO started from the true previous pose
on a map fused at the true poses; held-out seeds):

  * its proposal is closer to the tracker's converged offset than the paper's
    initialisation (c_0 = s*_{t-1}, i.e. a zero offset) on held-out samples;
  * proposal + 5 PFO iterations (with the library's default second-run rules)
    tracks the same held-out frames at least as fast as plain PFO with up to
    20 iterations, at an equal or lower ATE (mean over the sequences).
"""
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


def test_trained_proposal_beats_the_zero_offset_and_plain_pfo(nat):
    import torch

    from paper_2105_05600_gb300 import learned

    spec = dict(synth.CONFIGS["learned"])
    ds = learned.generate_dataset(nat, spec, list(range(100, 108)), 151, start="truth")
    seq = ds["seq"]
    train_rows, val_rows = np.flatnonzero(seq < 7), np.flatnonzero(seq >= 7)
    net, hist = learned.train(nat, ds["X"], ds["Y"], train_rows, val_rows, epochs=30, batch=256)
    assert net.status() == 0
    # proposal quality on the held-out sequence's samples (rf_mlp_evaluate)
    rows = torch.as_tensor(val_rows.astype(np.int32), device="cuda")
    _, stats = net.evaluate(ds["X"], ds["Y"], idx=rows)
    err_net, err_zero = float(stats[0]), float(stats[7:13].sum())
    assert err_net < 0.5 * err_zero, (err_net, err_zero)
    # tracking A/B on held-out sequences with the default proposal parameters
    p = nat.proposal_params()
    rows_ab = learned.evaluate(nat, spec, [1000, 1001], 200, net, p, use_graph=True, warmup=3)
    for r in rows_ab:
        assert r["failed_frames"] <= 3, r
    learned_fps = sum(r["frames"] for r in rows_ab) / sum(r["learned_s"] for r in rows_ab)
    plain_fps = sum(r["frames"] for r in rows_ab) / sum(r["plain_s"] for r in rows_ab)
    learned_ate = float(np.mean([r["learned_ate_cm"] for r in rows_ab]))
    plain_ate = float(np.mean([r["plain_ate_cm"] for r in rows_ab]))
    print("gain", dict(learned_fps=learned_fps, plain_fps=plain_fps, learned_ate=learned_ate, plain_ate=plain_ate,
                       err_net=err_net, err_zero=err_zero))
    assert learned_fps >= plain_fps, (learned_fps, plain_fps)
    assert learned_ate <= plain_ate, (learned_ate, plain_ate, rows_ab)
