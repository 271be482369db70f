"""What the trained network gains over the method without it, on a small
version of the learned workload at the paper's FastCaMo-Synth mean speeds
(1.5 m/s, 0.75 rad/s; held-out seeds, own-kernel training on ~700 samples):

  * its proposal is closer to the tracker's converged offset than the paper's
    initialisation (c_0 = s*_{t-1}, i.e. a zero offset) on held-out samples;
  * proposal + 5 PFO iterations tracks the same frames at least 1.5x faster
    than plain PFO with up to 20 iterations.
The ATE comparison needs long sequences (bench.py --config learned); here one
150-frame sequence only guards against a tracking failure.
"""
import numpy as np
import pytest

from paper_2105_05600_gb300 import metrics, synth

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

    spec = dict(synth.CONFIGS["learned"], speed=1.5, ang_speed=0.75)
    ds = learned.generate_dataset(nat, spec, list(range(100, 108)), 120, substeps=2)
    seq = ds["seq"]
    train_rows, val_rows = np.flatnonzero(seq < 6), np.flatnonzero(seq >= 6)
    net, hist = learned.train(nat, ds["X"], ds["Y"], train_rows, val_rows, epochs=20, batch=256)
    assert net.status() == 0
    # proposal quality on the held-out sequences' samples
    rows = torch.as_tensor(val_rows.astype(np.int32), device="cuda")
    mu, y = learned.predict(net, ds["X"], ds["Y"], rows)
    mu, y = mu.cpu().numpy(), y.cpu().numpy()
    err_net = np.mean(np.sum((mu - y) ** 2, axis=1))
    err_zero = np.mean(np.sum(y ** 2, axis=1))
    assert err_net < 0.8 * err_zero, (err_net, err_zero)
    # tracking A/B on one held-out sequence
    p = nat.proposal_params(k_learned=5, kappa=2.0, theta=0.9)
    r = learned.evaluate(nat, spec, [1000], 150, net, p, use_graph=True, warmup=3)[0]
    assert r["failed_frames"] <= 3
    assert r["learned_fps"] >= 1.5 * r["plain_fps"], r
    assert r["learned_ate_cm"] <= 2.0 * r["plain_ate_cm"] + 10.0, r
