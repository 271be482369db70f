"""The learned proposal's network and geometry kernels (rf_proposal.h) against the
FP64 oracle (oracle/mlp.py), through the C ABI.

Parity bars:
  * dyadic network (inputs k/8, weights j/8, biases multiples of 2^-6): every
    product of every layer is a multiple of a layer quantum q and the sum of
    their magnitudes stays below 2^24 q, so every FP32 partial sum is exact in
    any order and the bfloat16 roundings see the exact value: the GPU forward
    output equals the oracle's bit for bit (the test asserts the premise);
  * general inputs: FP32 sums round differently from exact ones, so a stored
    bfloat16 activation can land one step (2^-7 relative) away from the
    oracle's; the output, a weighted sum of such values, is held to one step
    of its own scale in RMS and four steps at worst;
  * gradient (dyadic forward): per element <= 4 x 2^-7 x the magnitude
    gradient (the backward pass run on |values|), which covers a one-step
    disagreement in every rounded gradient entry, cascaded through the layers;
  * Adam's first step: the update is -lr g / (|g| + eps), so each parameter
    moves by at most lr and by exactly -lr sign(g) where the gradient is
    clearly nonzero;
  * features: bfloat16 codes equal to the oracle's rounding of its FP64 value.
"""
import numpy as np
import pytest

from oracle import mlp

pytestmark = pytest.mark.gpu

U = 2.0 ** -7  # one bfloat16 step, relative


@pytest.fixture(scope="module")
def nat():
    from paper_2105_05600_gb300 import build

    build.build()
    from paper_2105_05600_gb300 import _native

    return _native


def to_bf16(a):
    """numpy float64 values (bfloat16-exact) -> CUDA bfloat16 tensor."""
    import torch

    t = torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16)
    assert np.array_equal(t.float().numpy(), np.asarray(a, np.float32)), "values must be bfloat16-exact"
    return t.cuda()


def dyadic_problem(seed, B):
    rng = np.random.default_rng(seed)
    theta = np.zeros(mlp.n_params())
    W = mlp.unflatten(theta)
    for l, (o, i) in enumerate(mlp.LAYERS):
        rows = mlp.D_OUT if l == 3 else o
        cols = mlp.D_IN if l == 0 else i
        W[2 * l][:rows, :cols] = rng.choice([-1, 0, 0, 1], size=(rows, cols)) / 8.0
        W[2 * l + 1][:rows] = rng.integers(-8, 9, size=rows) / 64.0
    X = np.zeros((B, mlp.D_IN_PAD))
    X[:, :mlp.D_IN] = rng.integers(-4, 5, size=(B, mlp.D_IN)) / 8.0
    return theta, X


def assert_exact_premise(theta, X):
    """Every partial sum of every forward product is exact in FP32."""
    O, acts = mlp.forward(theta, X, round_bf16=True)
    Ws = mlp.unflatten(theta)[0::2]
    for l, q in enumerate((2.0 ** -6, 2.0 ** -9, 2.0 ** -12, 2.0 ** -15)):
        A, Wl = acts[l], Ws[l]
        prod_mag = np.abs(A) @ np.abs(Wl).T
        assert prod_mag.max() < 2.0 ** 24 * q
        assert np.all(np.mod(A / (q / 2.0 ** -3), 1.0) == 0.0)  # A is a multiple of q / (1/8)
    return O


# ----------------------------------------------------------------------------- forward
@pytest.mark.parametrize("B", [1, 200])
def test_forward_dyadic_is_exact(nat, B):
    import torch

    theta, X = dyadic_problem(1, B)
    O = assert_exact_premise(theta, X)
    net = nat.MLP(256)
    net.set_params(theta.astype(np.float32))
    out = net.forward(to_bf16(X))
    torch.cuda.synchronize()
    assert net.status() == 0
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), O)


def test_forward_general_within_one_step(nat):
    rng = np.random.default_rng(2)
    theta = mlp.init_params(3)
    for b in mlp.unflatten(theta)[1::2]:
        b[:] = rng.normal(size=b.shape) * 0.05
    B = 333
    X = np.zeros((B, mlp.D_IN_PAD))
    X[:, :mlp.D_IN] = np.clip(rng.normal(size=(B, mlp.D_IN)) * 2.0, -8, 8)
    X = mlp.bf16(X)
    net = nat.MLP(512)
    net.set_params(theta.astype(np.float32))
    theta32 = theta.astype(np.float32).astype(np.float64)  # the GPU holds FP32 parameters
    O, _ = mlp.forward(theta32, X, round_bf16=True)
    out = net.forward(to_bf16(X)).cpu().numpy().astype(np.float64)
    assert net.status() == 0
    err = np.abs(out - O)
    assert err.max() <= 4 * U * np.abs(O).max()
    assert np.sqrt(np.mean(err ** 2)) <= U * np.sqrt(np.mean(O ** 2))


def test_forward_rejects_bad_batches(nat):
    import torch

    net = nat.MLP(16)
    x = torch.zeros((17, 832), dtype=torch.bfloat16, device="cuda")
    with pytest.raises(nat.RfError):
        net.forward(x)


# ----------------------------------------------------------------------------- backward
def magnitude_gradient(theta, acts, G):
    """The backward pass on magnitudes (|G|, |W|, |activations|, masks kept)."""
    Ws = [np.abs(mlp.bf16(w)) for w in mlp.unflatten(theta)[0::2]]
    out = np.zeros(mlp.n_params())
    ov = mlp.unflatten(out)
    dA = np.abs(mlp.bf16(G))
    for l in (3, 2, 1, 0):
        ov[2 * l][:] = dA.T @ np.abs(acts[l])
        ov[2 * l + 1][:] = dA.sum(axis=0)
        if l > 0:
            dA = (dA @ Ws[l]) * (acts[l] > 0)
    return out


def test_gradient_matches_oracle(nat):
    import torch

    B = 256
    theta, X = dyadic_problem(4, B)
    assert_exact_premise(theta, X)
    # targets as the device holds them (FP32)
    Y = (np.random.default_rng(5).normal(size=(B, 6)) * 0.5).astype(np.float32).astype(np.float64)
    L, g_or, O = mlp.loss_and_grad(theta, X, Y, round_bf16=True)
    _, acts = mlp.forward(theta, X, round_bf16=True)
    Gm = magnitude_gradient(theta, acts, mlp.loss_and_grad_out(O, Y, mlp.velocity(acts))[1])
    net = nat.MLP(B)
    net.set_params(theta.astype(np.float32))
    grad, loss, out = net.gradient(to_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda(), B)
    torch.cuda.synchronize()
    assert net.status() == 0
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), O)  # forward exact
    assert abs(float(loss.item()) - L) <= 1e-6 * abs(L)
    g = grad.cpu().numpy().astype(np.float64)
    tol = 4 * U * Gm + 1e-30
    bad = np.abs(g - g_or) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:10], g[bad][:5], g_or[bad][:5], tol[bad][:5])
    # padding stays exactly zero
    gv = mlp.unflatten(g)
    assert np.all(gv[0][:, mlp.D_IN:] == 0.0) and np.all(gv[6][mlp.D_OUT:] == 0.0)
    assert np.all(gv[7][mlp.D_OUT:] == 0.0)


def test_gradient_with_index_gather(nat):
    # a permuted batch of a larger dataset gives the gradient of those rows
    import torch

    n_all, B = 96, 64
    theta, X = dyadic_problem(6, n_all)
    Y = np.random.default_rng(7).normal(size=(n_all, 6)).astype(np.float32).astype(np.float64)
    idx = np.random.default_rng(8).permutation(n_all)[:B].astype(np.int32)
    net = nat.MLP(B)
    net.set_params(theta.astype(np.float32))
    grad, loss, out = net.gradient(to_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda(), B,
                                   idx=torch.from_numpy(idx).cuda())
    assert net.status() == 0
    L, g_or, O = mlp.loss_and_grad(theta, X[idx], Y[idx], round_bf16=True)
    np.testing.assert_array_equal(out.cpu().numpy().astype(np.float64), O)
    assert abs(float(loss.item()) - L) <= 1e-6 * abs(L)
    _, acts = mlp.forward(theta, X[idx], round_bf16=True)
    Gm = magnitude_gradient(theta, acts, mlp.loss_and_grad_out(O, Y[idx], mlp.velocity(acts))[1])
    assert np.all(np.abs(grad.cpu().numpy() - g_or) <= 4 * U * Gm + 1e-30)
    # an index outside the dataset is reported, not read
    bad = torch.from_numpy(np.r_[idx[:-1], n_all].astype(np.int32)).cuda()
    net.gradient(to_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda(), B, idx=bad)
    assert net.status() == nat.RF_ERR_ARG
    assert net.status() == 0  # reset by the read


# ----------------------------------------------------------------------------- Adam
def test_adam_first_step(nat):
    import torch

    B = 128
    theta, X = dyadic_problem(9, B)
    Y = np.random.default_rng(10).normal(size=(B, 6)).astype(np.float32).astype(np.float64)
    _, g_or, O = mlp.loss_and_grad(theta, X, Y, round_bf16=True)
    _, acts = mlp.forward(theta, X, round_bf16=True)
    Gm = magnitude_gradient(theta, acts, mlp.loss_and_grad_out(O, Y, mlp.velocity(acts))[1])
    net = nat.MLP(B)
    net.set_params(theta.astype(np.float32))
    lr = 1e-3
    net.train_step(to_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda(), B, lr)
    assert net.status() == 0
    t1 = net.get_params().astype(np.float64)
    t0 = theta.astype(np.float32).astype(np.float64)
    step = t1 - t0
    assert np.all(np.abs(step) <= lr * (1 + 1e-5) + np.abs(t0) * 2.0 ** -23)
    # where the gradient's sign is certain (|g| above the parity bound) and |g| >> eps
    clear = (np.abs(g_or) > 4 * U * Gm) & (np.abs(g_or) > 1e-3)
    assert clear.sum() > 1000
    np.testing.assert_allclose(step[clear], -lr * np.sign(g_or[clear]), rtol=1e-4,
                               atol=np.abs(t0[clear]).max() * 2.0 ** -22)
    assert np.all(step[g_or == 0.0] == 0.0)


def test_training_follows_the_oracle(nat):
    # 120 Adam steps on a smooth regression problem: the GPU's loss curve follows
    # the oracle's (same batches, same initialisation)
    import torch

    rng = np.random.default_rng(11)
    n_all, B, steps, lr = 2048, 128, 120, 2e-3
    X = np.zeros((n_all, mlp.D_IN_PAD))
    X[:, :mlp.D_IN] = mlp.bf16(np.clip(rng.normal(size=(n_all, mlp.D_IN)), -8, 8))
    A = rng.normal(size=(6, 6)) * 0.5
    Y = np.tanh(X[:, 768:774] @ A.T) + 0.3 * X[:, :6]
    Y = Y.astype(np.float32).astype(np.float64)
    theta0 = mlp.init_params(12).astype(np.float32).astype(np.float64)
    batches = [rng.choice(n_all, B, replace=False).astype(np.int32) for _ in range(steps)]

    net = nat.MLP(B)
    net.set_params(theta0.astype(np.float32))
    xg, yg = to_bf16(X), torch.from_numpy(Y.astype(np.float32)).cuda()
    loss_buf = torch.zeros(steps, dtype=torch.float32, device="cuda")
    for s, idx in enumerate(batches):
        net.train_step(xg, yg, B, lr, idx=torch.from_numpy(idx).cuda(), loss_out=loss_buf[s:s + 1])
    gpu_loss = loss_buf.cpu().numpy().astype(np.float64)
    assert net.status() == 0

    opt = mlp.Adam(mlp.n_params())
    th = theta0.copy()
    or_loss = []
    for idx in batches:
        L, g, _ = mlp.loss_and_grad(th, X[idx], Y[idx], round_bf16=True)
        or_loss.append(L)
        th = opt.step(th, g, lr)
    or_loss = np.array(or_loss)
    assert gpu_loss[0] == pytest.approx(or_loss[0], rel=1e-3)
    assert or_loss[-10:].mean() < 0.5 * or_loss[:10].mean()  # the problem is learnable
    # same curve (moving averages): rounding differences grow through Adam's
    # normalised steps, so the bar is 1 % of the loss range over the first 30
    # steps and 5 % over all of them
    k = 10
    ga = np.convolve(gpu_loss, np.ones(k) / k, "valid")
    oa = np.convolve(or_loss, np.ones(k) / k, "valid")
    span = oa.max() - oa.min()
    assert np.all(np.abs(ga - oa)[:30 - k + 1] <= 0.01 * span), np.abs(ga - oa)[:30].max() / span
    assert np.all(np.abs(ga - oa) <= 0.05 * span), np.abs(ga - oa).max() / span


# ----------------------------------------------------------------------------- geometry
def rand_pose(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    q = q if q[0] >= 0 else -q
    return np.concatenate([q, rng.normal(size=3)])


@pytest.mark.parametrize("shape", [(480, 640), (61, 83)])
def test_features_match_oracle(nat, shape):
    import torch
    from oracle import compose_offset

    rng = np.random.default_rng(13)
    H, W = shape
    cur = rng.uniform(0.3, 6.0, size=(H, W)).astype(np.float32)
    prev = (cur + rng.normal(size=(H, W)) * 0.05).astype(np.float32)
    cur[rng.random((H, W)) < 0.2] = 0.0
    prev[rng.random((H, W)) < 0.2] = 0.0
    cur[: H // 5, : W // 5] = 0.0  # empty cells
    prev[-3:, :] = 9.0  # beyond z_max
    from paper_2105_05600_gb300 import synth

    K = synth.intrinsics(W, H)
    p2 = rand_pose(rng).astype(np.float32).astype(np.float64)
    p1 = compose_offset(p2, np.r_[rng.uniform(-0.05, 0.05, 3), rng.uniform(-0.1, 0.1, 3)])
    p1 = p1.astype(np.float32).astype(np.float64)
    x = nat.rf_proposal_features(torch.from_numpy(cur).cuda(), torch.from_numpy(prev).cuda(), K,
                                 torch.from_numpy(p2.astype(np.float32)).cuda(),
                                 torch.from_numpy(p1.astype(np.float32)).cuda())
    got = x.float().cpu().numpy().astype(np.float64)
    want = mlp.bf16(mlp.features(cur, prev, K["z_min"], K["z_max"], p2, p1))
    assert np.count_nonzero(want[:768] == 0.0) > 0 and np.count_nonzero(want[:768]) > 100
    diff = got != want
    assert diff.sum() <= 1, np.flatnonzero(diff)
    if diff.any():  # a rounding tie at most: one bfloat16 step apart
        i = np.flatnonzero(diff)[0]
        assert abs(got[i] - want[i]) <= U * abs(want[i])


def test_target_and_proposal_match_oracle(nat):
    import torch
    from oracle import compose_offset

    rng = np.random.default_rng(14)
    for trial in range(5):
        prev = rand_pose(rng).astype(np.float32).astype(np.float64)
        cur = compose_offset(prev, np.r_[rng.uniform(-0.08, 0.08, 3), rng.uniform(-0.2, 0.2, 3)])
        cur = cur.astype(np.float32).astype(np.float64)
        tp = torch.from_numpy(prev.astype(np.float32)).cuda()
        tc = torch.from_numpy(cur.astype(np.float32)).cuda()
        y = nat.rf_proposal_target(tp, tc).cpu().numpy()
        np.testing.assert_allclose(y, mlp.target(prev, cur), rtol=1e-6, atol=1e-6)
        o = np.zeros(16, np.float32)
        o[:6] = rng.normal(size=6)
        o[6:12] = rng.uniform(-8, 3, size=6)  # some clamped at -6, some clipped at r_min / r_max
        p = nat.proposal_params(kappa=1.5)
        x = np.zeros(832)
        x[768:774] = mlp.bf16(rng.normal(size=6) * 0.5)  # previous offset: the base of mu
        c0, r0 = nat.rf_proposal_apply(torch.from_numpy(o).cuda(), to_bf16(x), tp, p)
        oc, orr = mlp.proposal(o.astype(np.float64), x[768:774], prev, kappa=1.5)
        c0 = c0.cpu().numpy()
        if np.dot(c0[:4], oc[:4]) < 0:
            c0[:4] = -c0[:4]
        np.testing.assert_allclose(c0, oc, atol=2e-6)
        np.testing.assert_allclose(r0.cpu().numpy(), orr, rtol=2e-6)


# ----------------------------------------------------------------------------- evaluation / calibration
def test_evaluate_and_calibrate_match_oracle(nat):
    """rf_mlp_evaluate over gathered rows in several forward batches, and
    rf_mlp_calibrate_scale, against the oracle.  With dyadic weights, inputs and
    targets the forward pass and mu are exact (asserted premise), so mu must be
    equal and the FP64 statistics agree to the rounding of exp."""
    import torch

    theta, X = dyadic_problem(5, 300)
    O = assert_exact_premise(theta, X)
    rng = np.random.default_rng(6)
    Y = rng.integers(-16, 17, size=(300, 6)) / 16.0
    idx = rng.permutation(300)[:217].astype(np.int32)
    net = nat.MLP(64)  # 217 rows in four forward batches
    net.set_params(theta.astype(np.float32))
    Xg = to_bf16(X)
    Yg = torch.from_numpy(Y.astype(np.float32)).cuda()
    ig = torch.from_numpy(idx).cuda()
    mu, stats = net.evaluate(Xg, Yg, idx=ig)
    assert net.status() == 0
    mu_o, stats_o = mlp.evaluate(theta, X[idx], Y[idx])
    np.testing.assert_array_equal(mu.cpu().numpy().astype(np.float64), mu_o)
    np.testing.assert_allclose(stats.cpu().numpy(), stats_o, rtol=1e-12)
    # calibration: same k, the log-scale biases moved by log k, nothing else changed
    k = net.calibrate_scale(Xg, Yg, idx=ig)
    theta_o, k_o = mlp.calibrate_scale(theta.astype(np.float32).astype(np.float64), X[idx], Y[idx])
    np.testing.assert_allclose(k, k_o, rtol=1e-6)
    got = net.get_params().astype(np.float64)
    np.testing.assert_allclose(got, theta_o, rtol=1e-6, atol=1e-7)
    changed = np.flatnonzero(got != theta.astype(np.float32))
    assert set(changed) <= set(range(len(theta) - 10, len(theta) - 4))
    # without an index: the first n rows
    mu2, stats2 = net.evaluate(Xg, Yg, n_rows=90)
    theta32 = got
    mu2_o, stats2_o = mlp.evaluate(theta32, X[:90], Y[:90])
    np.testing.assert_allclose(mu2.cpu().numpy(), mu2_o, rtol=0, atol=1e-6)
    np.testing.assert_allclose(stats2.cpu().numpy(), stats2_o, rtol=1e-5)
