"""FP64 oracle of the learned swarm proposal: feature map, 4-layer MLP forward and
backward, loss, Adam update and the proposal that seeds the PST.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s cpu_baseline / reference leg may import this module.  It shares
no code with the CUDA library.

The paper has no learned component: Sec. 6 names combining its random
optimisation with learned priors as future work, and Sec. 4 seeds each frame's
PST with c_0 = s*_{t-1} and r_0 = r_1 of the previous frame.  This module
defines the extension the library implements: a network predicts the swarm
centre offset and per-axis scale that replace that initialisation.

    features ........ 32 x 24 block-mean depth residual of (D_t, D_{t-1}) + the
                      previous frame-to-frame offset (6 values)
    forward ......... 832 -> 256 -> 256 -> 256 -> 16 (12 used), ReLU between
                      layers; optional bfloat16 rounding of weights, inputs and
                      hidden activations (the kernels' storage types) with
                      exact (FP64) sums
    loss ............ per output axis 1/2 r^2 (1 + e^{-2s}) + s: squared error
                      on the mean plus a Gaussian negative log-likelihood for
                      the log scale s (clamped to [-6, 6]); the mean offset is
                      the previous offset (an input) plus the first 6 outputs
    backward ........ hand-written reverse mode of the above; in pure FP64 mode
                      it is the exact gradient (checked by finite differences)
    adam ............ Kingma & Ba 2015, Algorithm 1 (bias-corrected moments)
    proposal ........ c_0 = s*_{t-1} (+) mean offset (the MovePST composition of
                      Sec. 3.3), r_0 = kappa * e^s per axis, clipped
"""
from __future__ import annotations

import numpy as np

from . import compose_offset, quat_mul

GRID_W, GRID_H = 32, 24
N_RES = GRID_W * GRID_H          # 768 residual features
D_IN = N_RES + 6                 # + previous offset
D_IN_PAD = 832                   # padded to a multiple of 64 (zeros)
D_H = 256
D_OUT = 12                       # 6 mean offsets + 6 log scales
D_OUT_PAD = 16
S_Z = 0.1                        # residual unit (m)
RES_CLIP = 8.0                   # residual features clipped to +-8 units
S_Q = 0.05                       # quaternion vector unit (about 0.1 rad of rotation)
S_T = 0.1                        # translation unit (m)
S_CLAMP = 6.0                    # log-scale clamp
OFFSET_UNITS = np.array([S_Q, S_Q, S_Q, S_T, S_T, S_T])

LAYERS = [(D_H, D_IN_PAD), (D_H, D_H), (D_H, D_H), (D_OUT_PAD, D_H)]  # (out, in) per layer


# ----------------------------------------------------------------------------- parameters
def n_params():
    return sum(o * i + o for o, i in LAYERS)


def unflatten(theta):
    """Views (W1, b1, W2, b2, W3, b3, W4, b4) into the flat parameter vector, in
    that order, each W row-major (out, in)."""
    out, p = [], 0
    for o, i in LAYERS:
        out.append(theta[p:p + o * i].reshape(o, i))
        p += o * i
        out.append(theta[p:p + o])
        p += o
    return out


def init_params(seed):
    """He-uniform weights, zero biases; input columns >= D_IN and output rows
    >= D_OUT stay zero (padding)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(n_params())
    views = unflatten(theta)
    for l, (o, i) in enumerate(LAYERS):
        fan_in = D_IN if l == 0 else i
        lim = np.sqrt(6.0 / fan_in) if l < 3 else np.sqrt(3.0 / fan_in) * 0.1
        W = views[2 * l]
        rows = D_OUT if l == 3 else o
        cols = D_IN if l == 0 else i
        W[:rows, :cols] = rng.uniform(-lim, lim, size=(rows, cols))
    return theta


# ----------------------------------------------------------------------------- bfloat16
def bf16(x):
    """Round to the nearest bfloat16 value (8 significant bits, ties to even),
    directly from the FP64 value: x = m 2^E with m in [0.5, 1) -> round(256 m) 2^(E-8)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0), e - 8)


# ----------------------------------------------------------------------------- features
def offset(pose_a, pose_b):
    """The 6-vector delta with pose_b = pose_a (+) delta under the default MovePST
    composition (left-multiplied rotation, world-frame translation, Sec. 3.3):
    delta[0:3] = vector part of q_b q_a^-1 (scalar part made >= 0),
    delta[3:6] = t_b - t_a.  Poses are (qw, qx, qy, qz, tx, ty, tz)."""
    a = np.asarray(pose_a, np.float64)
    b = np.asarray(pose_b, np.float64)
    qa_inv = np.array([a[0], -a[1], -a[2], -a[3]]) / np.dot(a[:4], a[:4])
    qd = quat_mul(b[:4] / np.linalg.norm(b[:4]), qa_inv)
    if qd[0] < 0:
        qd = -qd
    return np.concatenate([qd[1:], b[4:] - a[4:]])


def block_means(depth, z_min, z_max):
    """Mean of the valid depths (z_min < z <= z_max) in each of the 32 x 24 cells,
    cell (i, j) covering columns [floor(iW/32), floor((i+1)W/32)) and rows
    [floor(jH/24), floor((j+1)H/24)); returns (means, counts), shape (24, 32)."""
    H, W = depth.shape
    means = np.zeros((GRID_H, GRID_W))
    counts = np.zeros((GRID_H, GRID_W), np.int64)
    for j in range(GRID_H):
        r0, r1 = (j * H) // GRID_H, ((j + 1) * H) // GRID_H
        for i in range(GRID_W):
            c0, c1 = (i * W) // GRID_W, ((i + 1) * W) // GRID_W
            z = depth[r0:r1, c0:c1].astype(np.float64).ravel()
            z = z[(z > z_min) & (z <= z_max)]
            counts[j, i] = len(z)
            means[j, i] = z.sum() / len(z) if len(z) else 0.0
    return means, counts


def features(depth, prev_depth, z_min, z_max, pose_prev2, pose_prev):
    """Network input x (D_IN_PAD values): clip((mean_t - mean_{t-1}) / S_Z, +-8) per
    cell where both cells hold valid depth (else 0), row-major over (j, i); then the
    offset from s*_{t-2} to s*_{t-1} in units (S_Q, S_Q, S_Q, S_T, S_T, S_T); zeros."""
    mc, nc = block_means(depth, z_min, z_max)
    mp, npv = block_means(prev_depth, z_min, z_max)
    res = np.where((nc > 0) & (npv > 0), np.clip((mc - mp) / S_Z, -RES_CLIP, RES_CLIP), 0.0)
    x = np.zeros(D_IN_PAD)
    x[:N_RES] = res.ravel()
    x[N_RES:D_IN] = offset(pose_prev2, pose_prev) / OFFSET_UNITS
    return x


def target(pose_prev, pose_cur):
    """Training target: the offset from s*_{t-1} to s*_t in offset units."""
    return offset(pose_prev, pose_cur) / OFFSET_UNITS


# ----------------------------------------------------------------------------- network
def forward(theta, X, round_bf16=True):
    """Outputs O (B x 16) and the stored activations [x, h1, h2, h3] of a batch
    X (B x 832).  With round_bf16 the weights, the input and each hidden
    activation are rounded to bfloat16 (the kernels' operand type); every sum is
    exact in FP64 (the kernels accumulate in FP32)."""
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    W1, b1, W2, b2, W3, b3, W4, b4 = unflatten(np.asarray(theta, np.float64))
    acts = [R(X)]
    for W, b in ((W1, b1), (W2, b2), (W3, b3)):
        acts.append(R(np.maximum(acts[-1] @ R(W).T + b, 0.0)))
    O = acts[-1] @ R(W4).T + b4
    return O, acts


def mean_offset(O, V):
    """mu = V + O[:, 0:6]: the previous offset (input columns 768..773, as the
    network sees them) plus the network's correction."""
    return np.asarray(V, np.float64) + O[:, 0:6]


def loss_and_grad_out(O, Y, V):
    """Mean over the batch of sum_d [1/2 r_d^2 (1 + e^{-2 s_d}) + s_d], r = y - mu,
    mu = V + O[:, 0:6], s = clamp(O[:, 6:12], -6, 6); returns (L, dL/dO) with dL/dO
    zero in the padding columns and where the clamp is active."""
    B = O.shape[0]
    mu, s_raw = mean_offset(O, V), O[:, 6:12]
    s = np.clip(s_raw, -S_CLAMP, S_CLAMP)
    r = Y - mu
    e = np.exp(-2.0 * s)
    L = float(np.sum(0.5 * r * r * (1.0 + e) + s)) / B
    G = np.zeros_like(O)
    G[:, 0:6] = -r * (1.0 + e) / B
    inside = (s_raw > -S_CLAMP) & (s_raw < S_CLAMP)
    G[:, 6:12] = np.where(inside, (1.0 - r * r * e) / B, 0.0)
    return L, G


def backward(theta, acts, G, round_bf16=True):
    """Flat gradient of the loss given dL/dO = G (B x 16) and the activations of
    forward().  With round_bf16 the output gradient and each masked hidden
    gradient are rounded to bfloat16 before they enter a product (the kernels'
    operand type); the bias gradient sums the same rounded values."""
    R = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    Ws = unflatten(np.asarray(theta, np.float64))[0::2]
    grad = np.zeros(n_params())
    gv = unflatten(grad)
    dA = R(G)
    for l in (3, 2, 1, 0):
        gv[2 * l][:] = dA.T @ acts[l]
        gv[2 * l + 1][:] = dA.sum(axis=0)
        if l > 0:
            dH = dA @ R(Ws[l])
            dA = R(dH * (acts[l] > 0))
    return grad


def velocity(acts):
    """The previous-offset inputs of a batch as the network holds them."""
    return acts[0][:, N_RES:D_IN]


def evaluate(theta, X, Y, round_bf16=True):
    """The quantities the training selects and calibrates with, over the rows of X
    (the network's output O, mu = previous offset + correction, s = clamp(O[:,
    6:12], -6, 6), e = Y - mu): returns (mu, stats) with stats the means over the
    rows of [sum_d e_d^2, e_d^2 exp(-2 s_d) (d = 0..5), y_d^2 (d = 0..5)]."""
    O, acts = forward(theta, X, round_bf16)
    mu = mean_offset(O, velocity(acts))
    s = np.clip(O[:, 6:12], -S_CLAMP, S_CLAMP)
    e = np.asarray(Y, np.float64) - mu
    stats = np.concatenate([[np.mean(np.sum(e * e, axis=1))], np.mean(e * e * np.exp(-2.0 * s), axis=0),
                            np.mean(np.asarray(Y, np.float64) ** 2, axis=0)])
    return mu, stats


def calibrate_scale(theta, X, Y, round_bf16=True):
    """Per-axis calibration of the log-scale head: k_d^2 = mean over the rows of
    e_d^2 exp(-2 s_d) (evaluate's stats[1 + d]); log k_d is added to the output
    bias of s_d.  Returns (new theta, k)."""
    _, stats = evaluate(theta, X, Y, round_bf16)
    k = np.sqrt(np.maximum(stats[1:7], 1e-12))
    out = np.array(theta, np.float64, copy=True)
    unflatten(out)[7][6:12] += np.log(k)
    return out, k


def loss(theta, X, Y, round_bf16=False):
    O, acts = forward(theta, X, round_bf16)
    return loss_and_grad_out(O, Y, velocity(acts))[0]


def loss_and_grad(theta, X, Y, round_bf16=True):
    O, acts = forward(theta, X, round_bf16)
    L, G = loss_and_grad_out(O, Y, velocity(acts))
    return L, backward(theta, acts, G, round_bf16), O


# ----------------------------------------------------------------------------- Adam
class Adam:
    """Kingma & Ba 2015, Algorithm 1: m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
    theta <- theta - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)."""

    def __init__(self, n, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.beta1, self.beta2, self.eps = beta1, beta2, eps

    def step(self, theta, g, lr):
        self.t += 1
        self.m = self.beta1 * self.m + (1.0 - self.beta1) * g
        self.v = self.beta2 * self.v + (1.0 - self.beta2) * g * g
        mh = self.m / (1.0 - self.beta1 ** self.t)
        vh = self.v / (1.0 - self.beta2 ** self.t)
        return theta - lr * mh / (np.sqrt(vh) + self.eps)


# ----------------------------------------------------------------------------- proposal
def proposal(o, v, pose_prev, kappa=2.0, r_min=(2e-3, 2e-3, 2e-3, 4e-3, 4e-3, 4e-3),
             r_max=(0.2, 0.2, 0.2, 0.4, 0.4, 0.4)):
    """Initial swarm state of one frame from one network output o (>= 12 values)
    and its previous-offset input v (6 values): c_0 = s*_{t-1} (+) (mu * units),
    mu = v + o[0:6], and r_0 = clip(kappa * e^{clamp(s)} * units, r_min, r_max)
    per axis (quaternion-vector axes first, then translation)."""
    o = np.asarray(o, np.float64)
    delta = (np.asarray(v, np.float64) + o[0:6]) * OFFSET_UNITS
    c0 = compose_offset(np.asarray(pose_prev, np.float64), delta)
    r0 = np.clip(kappa * np.exp(np.clip(o[6:12], -S_CLAMP, S_CLAMP)) * OFFSET_UNITS, r_min, r_max)
    return c0, r0
