"""Pins of the learned-proposal oracle (oracle/mlp.py) against facts that do not
come from the oracle itself: bfloat16 rounding against a library cast, the
pose offset against the C oracle's MovePST composition, block means against a
reshape-based mean, closed-form networks, finite differences of the FP64 loss,
the closed form of the first Adam steps (Kingma & Ba 2015, Algorithm 1)."""
import numpy as np
import pytest

from oracle import compose_offset
from oracle import mlp


def rand_pose(rng, scale=1.0):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return np.concatenate([q, rng.normal(size=3) * scale])


def small_step(rng, pose, rot=0.05, trans=0.1):
    d = np.concatenate([rng.uniform(-rot, rot, 3), rng.uniform(-trans, trans, 3)])
    return compose_offset(pose, d), d


# ----------------------------------------------------------------------------- bf16
def test_bf16_matches_library_cast():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=20000) * 10.0 ** rng.integers(-20, 20, 20000),
                        [0.0, 1.0, -1.0, 3.0, 1e-30, -7.5e12]]).astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), ref)


def test_bf16_ties_to_even():
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: the even neighbour is 1
    assert mlp.bf16(1.0 + 2.0 ** -8) == 1.0
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    assert mlp.bf16(1.0 + 3 * 2.0 ** -8) == 1.0 + 2.0 ** -6
    assert mlp.bf16(-(1.0 + 3 * 2.0 ** -8)) == -(1.0 + 2.0 ** -6)
    # a value just above the midpoint rounds up
    assert mlp.bf16(1.0 + 2.0 ** -8 + 2.0 ** -30) == 1.0 + 2.0 ** -7


# ----------------------------------------------------------------------------- offsets
def test_offset_inverts_the_movepst_composition():
    rng = np.random.default_rng(1)
    for _ in range(50):
        a = rand_pose(rng)
        b, d = small_step(rng, a)
        np.testing.assert_allclose(mlp.offset(a, b), d, atol=1e-12)
        np.testing.assert_allclose(compose_offset(a, mlp.offset(a, b)), b, atol=1e-12)
    a = rand_pose(rng)
    np.testing.assert_allclose(mlp.offset(a, a), np.zeros(6), atol=1e-15)


def test_offset_of_a_pure_translation():
    a = np.array([1.0, 0, 0, 0, 1.0, 2.0, 3.0])
    b = np.array([1.0, 0, 0, 0, 1.5, 2.0, 2.0])
    np.testing.assert_allclose(mlp.offset(a, b), [0, 0, 0, 0.5, 0.0, -1.0], atol=1e-15)


# ----------------------------------------------------------------------------- features
def test_block_means_against_reshape_mean():
    rng = np.random.default_rng(2)
    D = rng.uniform(0.3, 5.0, size=(480, 640)).astype(np.float32)
    D[rng.random(D.shape) < 0.2] = 0.0
    D[:40, :60] = 0.0  # whole cells empty
    means, counts = mlp.block_means(D, 0.1, 8.0)
    blocks = D.astype(np.float64).reshape(24, 20, 32, 20)
    valid = (blocks > 0.1) & (blocks <= 8.0)
    n = valid.sum(axis=(1, 3))
    s = np.where(valid, blocks, 0.0).sum(axis=(1, 3))
    np.testing.assert_array_equal(counts, n)
    np.testing.assert_allclose(means, np.where(n > 0, s / np.maximum(n, 1), 0.0), rtol=1e-13)


def test_block_means_partition_a_ragged_image():
    rng = np.random.default_rng(3)
    D = rng.uniform(0.3, 5.0, size=(61, 83)).astype(np.float32)
    D[rng.random(D.shape) < 0.3] = 0.0
    means, counts = mlp.block_means(D, 0.1, 8.0)
    valid = (D > 0.1) & (D <= 8.0)
    assert counts.sum() == valid.sum()
    np.testing.assert_allclose((means * counts).sum(), D[valid].astype(np.float64).sum(), rtol=1e-12)


def test_features_of_a_constant_depth_pair():
    cur = np.full((60, 80), 2.0, np.float32)
    prev = np.full((60, 80), 1.9, np.float32)
    prev[:, :10] = 0.0  # cells with no previous depth give 0
    a = np.array([1.0, 0, 0, 0, 0, 0, 0])
    b = np.array([1.0, 0, 0, 0, 0.02, 0, -0.01])
    x = mlp.features(cur, prev, 0.1, 8.0, a, b)
    res = x[:768].reshape(24, 32)
    want = (np.float64(np.float32(2.0)) - np.float64(np.float32(1.9))) / 0.1
    np.testing.assert_allclose(res[:, 4:], want, rtol=1e-12)
    assert np.all(res[:, :4] == 0.0)
    np.testing.assert_allclose(x[768:774], [0, 0, 0, 0.2, 0.0, -0.1], atol=1e-15)
    assert np.all(x[774:] == 0.0) and x.shape == (mlp.D_IN_PAD,)


def test_residual_features_are_clipped():
    cur = np.full((48, 64), 5.0, np.float32)
    prev = np.full((48, 64), 1.0, np.float32)
    p = np.array([1.0, 0, 0, 0, 0, 0, 0])
    assert np.all(mlp.features(cur, prev, 0.1, 8.0, p, p)[:768] == mlp.RES_CLIP)
    assert np.all(mlp.features(prev, cur, 0.1, 8.0, p, p)[:768] == -mlp.RES_CLIP)


# ----------------------------------------------------------------------------- network
def test_zero_weights_give_the_output_bias():
    theta = np.zeros(mlp.n_params())
    b4 = mlp.unflatten(theta)[7]
    b4[:] = np.arange(16) * 0.25
    X = np.random.default_rng(4).normal(size=(5, mlp.D_IN_PAD))
    O, _ = mlp.forward(theta, X)
    np.testing.assert_array_equal(O, np.tile(b4, (5, 1)))


def test_selector_network_is_the_identity_on_positive_inputs():
    # W1 copies inputs 0..5, W2 = W3 = identity on them, W4 copies them to outputs
    # 0..5 and to outputs 6..11 negated; with bf16-exact inputs every value is exact
    theta = np.zeros(mlp.n_params())
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unflatten(theta)
    for i in range(6):
        W1[i, i] = W2[i, i] = W3[i, i] = 1.0
        W4[i, i] = 1.0
        W4[6 + i, i] = -2.0
    b4[:12] = 0.5
    X = np.zeros((3, mlp.D_IN_PAD))
    X[:, :6] = np.array([[0.5, 1.0, 2.0, 0.25, 3.0, 1.5]] * 3) * np.array([[1], [2], [4]])
    for rnd in (True, False):
        O, acts = mlp.forward(theta, X, round_bf16=rnd)
        np.testing.assert_array_equal(O[:, :6], X[:, :6] + 0.5)
        np.testing.assert_array_equal(O[:, 6:12], -2 * X[:, :6] + 0.5)
        np.testing.assert_array_equal(acts[3][:, :6], X[:, :6])


def test_loss_closed_forms():
    B = 4
    Y = np.random.default_rng(5).normal(size=(B, 6))
    O = np.zeros((B, 16))
    O[:, :6] = Y
    V = np.zeros((B, 6))
    L, G = mlp.loss_and_grad_out(O, Y, V)
    assert L == 0.0
    np.testing.assert_array_equal(G[:, :6], 0.0)
    np.testing.assert_allclose(G[:, 6:12], 1.0 / B)  # dL/ds = (1 - 0) / B
    O[:, :6] = Y - 1.0
    O[:, 6:12] = np.log(2.0)
    L, G = mlp.loss_and_grad_out(O, Y, V)
    np.testing.assert_allclose(L, 6 * (0.5 * 1.0 * (1 + 0.25) + np.log(2.0)), rtol=1e-14)
    np.testing.assert_allclose(G[:, :6], -1.25 / B, rtol=1e-14)
    np.testing.assert_allclose(G[:, 6:12], (1 - 0.25) / B, rtol=1e-14)
    assert np.all(G[:, 12:] == 0.0)
    O[:, 6] = 7.0  # clamped: value uses s = 6, gradient is zero
    L2, G2 = mlp.loss_and_grad_out(O, Y, V)
    assert np.all(G2[:, 6] == 0.0)
    # the mean is the previous offset plus the correction: shifting V by d and O
    # by -d changes nothing
    d = np.random.default_rng(6).normal(size=(B, 6))
    O2 = O.copy()
    O2[:, :6] -= d
    L3, G3 = mlp.loss_and_grad_out(O2, Y, V + d)
    assert L3 == pytest.approx(L2, rel=1e-12) and np.allclose(G3, G2, rtol=1e-12, atol=1e-15)


@pytest.fixture(scope="module")
def net():
    rng = np.random.default_rng(6)
    theta = mlp.init_params(7)
    W = mlp.unflatten(theta)
    for b in W[1::2]:
        b[:] = rng.normal(size=b.shape) * 0.1
    X = np.zeros((6, mlp.D_IN_PAD))
    X[:, :mlp.D_IN] = rng.normal(size=(6, mlp.D_IN))
    Y = rng.normal(size=(6, 6))
    return theta, X, Y


def test_gradient_matches_finite_differences(net):
    theta, X, Y = net
    L, g, _ = mlp.loss_and_grad(theta, X, Y, round_bf16=False)
    rng = np.random.default_rng(8)
    h = 1e-6
    # whole-gradient directional derivatives
    for _ in range(4):
        u = rng.normal(size=theta.shape)
        fd = (mlp.loss(theta + h * u, X, Y) - mlp.loss(theta - h * u, X, Y)) / (2 * h)
        np.testing.assert_allclose(fd, g @ u, rtol=1e-6)
    # single components of every layer (weights in the used block, all output biases)
    offs, p = [], 0
    for o, i in mlp.LAYERS:
        offs.append((p, o, i))
        p += o * i + o
    idx = []
    for l, (p0, o, i) in enumerate(offs):
        rows = mlp.D_OUT if l == 3 else o
        cols = mlp.D_IN if l == 0 else i
        for r, c in zip(rng.integers(0, rows, 12), rng.integers(0, cols, 12)):
            idx.append(p0 + r * i + c)
        idx += list(p0 + o * i + rng.integers(0, rows, 4))
    for k in idx:
        e = np.zeros_like(theta)
        e[k] = h
        fd = (mlp.loss(theta + e, X, Y) - mlp.loss(theta - e, X, Y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_padding_gradients_are_zero(net):
    theta, X, Y = net
    _, g, _ = mlp.loss_and_grad(theta, X, Y, round_bf16=True)
    W1, b1, W2, b2, W3, b3, W4, b4 = mlp.unflatten(g)
    assert np.all(W1[:, mlp.D_IN:] == 0.0)
    assert np.all(W4[mlp.D_OUT:] == 0.0) and np.all(b4[mlp.D_OUT:] == 0.0)


def test_rounded_gradient_is_close_to_exact(net):
    # bf16 operands perturb each product by ~2^-8 relative; the gradient stays close
    theta, X, Y = net
    _, g64, _ = mlp.loss_and_grad(theta, X, Y, round_bf16=False)
    _, g16, _ = mlp.loss_and_grad(theta, X, Y, round_bf16=True)
    assert np.linalg.norm(g16 - g64) <= 0.05 * np.linalg.norm(g64)


# ----------------------------------------------------------------------------- Adam
def test_adam_first_steps_closed_form():
    g1 = np.array([1e-3, -2.0, 0.0, 5e-9])
    theta0 = np.array([1.0, 2.0, 3.0, 4.0])
    opt = mlp.Adam(4)
    lr = 0.01
    t1 = opt.step(theta0, g1, lr)
    # step 1: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)
    np.testing.assert_allclose(t1, theta0 - lr * g1 / (np.abs(g1) + 1e-8), rtol=1e-15)
    g2 = np.array([3e-3, 1.0, 1.0, 0.0])
    t2 = opt.step(t1, g2, lr)
    m = 0.9 * 0.1 * g1 + 0.1 * g2
    v = 0.999 * 0.001 * g1 ** 2 + 0.001 * g2 ** 2
    np.testing.assert_allclose(t2, t1 - lr * (m / (1 - 0.81)) / (np.sqrt(v / (1 - 0.999 ** 2)) + 1e-8),
                               rtol=1e-13)


def test_adam_fits_a_linear_least_squares_problem():
    # Adam on a least-squares objective converges to the solution of a library
    # least-squares routine
    rng = np.random.default_rng(9)
    A = rng.uniform(0.5, 1.5, size=(64, 4))
    w_true = np.array([0.3, -0.2, 0.5, 0.1])
    y = A @ w_true + 0.01 * rng.normal(size=64)
    w_ls, *_ = np.linalg.lstsq(A, y, rcond=None)
    w = np.zeros(4)
    opt = mlp.Adam(4)
    for it in range(4000):
        g = A.T @ (A @ w - y) / 64
        w = opt.step(w, g, 0.01 if it < 3000 else 0.001)
    np.testing.assert_allclose(w, w_ls, atol=2e-4)


# ----------------------------------------------------------------------------- proposal
def test_proposal_of_a_zero_output_is_the_previous_pose():
    prev = np.array([0.9, 0.1, -0.3, 0.2, 1.0, 2.0, 0.5])
    prev[:4] /= np.linalg.norm(prev[:4])
    c0, r0 = mlp.proposal(np.zeros(16), np.zeros(6), prev, kappa=2.0)
    np.testing.assert_allclose(c0, prev, atol=1e-15)
    np.testing.assert_allclose(r0, 2.0 * mlp.OFFSET_UNITS)


def test_proposal_moves_by_the_predicted_offset():
    rng = np.random.default_rng(10)
    prev = rand_pose(rng)
    cur, d = small_step(rng, prev)
    v = rng.normal(size=6) * 0.3  # previous offset; the network predicts the rest
    o = np.zeros(16)
    o[:6] = mlp.target(prev, cur) - v
    o[6:12] = np.log(0.01)  # tiny scale: clipped to r_min
    c0, r0 = mlp.proposal(o, v, prev)
    np.testing.assert_allclose(c0, cur, atol=1e-12)
    np.testing.assert_allclose(r0, [2e-3, 2e-3, 2e-3, 4e-3, 4e-3, 4e-3])


# ----------------------------------------------------------------------------- evaluation / calibration
def _const_head_network(rng, b_mu, b_s):
    """A network whose output does not depend on the input: zero weights, output
    bias (b_mu, b_s) -- mu = previous offset + b_mu, s = b_s on every row."""
    theta = np.zeros(mlp.n_params())
    b4 = mlp.unflatten(theta)[7]
    b4[0:6] = b_mu
    b4[6:12] = b_s
    return theta


def _rows(rng, B):
    X = np.zeros((B, mlp.D_IN_PAD))
    X[:, :mlp.D_IN] = mlp.bf16(rng.normal(size=(B, mlp.D_IN)))
    Y = rng.normal(size=(B, 6)) * 0.7
    return X, Y


def test_evaluate_agrees_with_the_pinned_loss():
    # with a constant log scale s, the loss (pinned by finite differences and closed
    # forms above) is 1/2 stats[0] + 1/2 sum_d stats[1 + d] + sum_d s_d
    rng = np.random.default_rng(11)
    X, Y = _rows(rng, 57)
    b_s = np.array([-0.4, 0.1, 0.3, -1.2, 0.8, 0.05])
    theta = _const_head_network(rng, rng.normal(size=6) * 0.2, b_s)
    mu, stats = mlp.evaluate(theta, X, Y)
    L = mlp.loss(theta, X, Y, round_bf16=True)
    assert abs(L - (0.5 * stats[0] + 0.5 * stats[1:7].sum() + b_s.sum())) <= 1e-12 * abs(L)
    # an exact fit: targets equal to mu give zero error
    mu_fit, stats_fit = mlp.evaluate(theta, X, mu)
    assert stats_fit[0] == 0.0 and np.all(stats_fit[1:7] == 0.0)
    np.testing.assert_array_equal(mu_fit, mu)
    # the zero-offset error of the Sec. 4 initialisation depends on the targets only
    _, stats_zero = mlp.evaluate(np.zeros(mlp.n_params()), X, Y)
    np.testing.assert_array_equal(stats_zero[7:13], stats[7:13])


def test_calibration_makes_the_moments_one():
    # k_d^2 = mean e_d^2 exp(-2 s_d); after s_d += log k_d the same mean is exactly 1
    # (the errors e do not depend on the scale head); a scale head that already fits
    # gets k = 1
    rng = np.random.default_rng(12)
    X, Y = _rows(rng, 200)
    theta = mlp.init_params(4)
    b4 = mlp.unflatten(theta)[7]
    b4[6:12] = rng.normal(size=6) * 0.3
    theta2, k = mlp.calibrate_scale(theta, X, Y)
    _, st = mlp.evaluate(theta2, X, Y)
    np.testing.assert_allclose(st[1:7], 1.0, rtol=1e-12)
    _, st_before = mlp.evaluate(theta, X, Y)
    np.testing.assert_allclose(st[0], st_before[0], rtol=1e-15)  # mu unchanged
    _, k_again = mlp.calibrate_scale(theta2, X, Y)
    np.testing.assert_allclose(k_again, 1.0, rtol=1e-12)
    np.testing.assert_array_equal(np.delete(theta2, np.arange(len(theta) - 10, len(theta) - 4)),
                                  np.delete(theta, np.arange(len(theta) - 10, len(theta) - 4)))
