"""FP64 CPU oracle of the surrogate network (test infrastructure only).

The surrogate maps a standardised truncated trivariate t problem to its
probability and moments.  For X ~ t_3(0, R, m) with R a correlation matrix and
truncation point c (event X > c, componentwise):
    inputs  (7):  c_1, c_2, c_3, R_12, R_13, R_23, log m
    outputs (10): log P(X > c), E[X | X > c] (3),
                  E[X X^T | X > c] upper triangle (11, 12, 13, 22, 23, 33)
Network: 7 -> 128 -> 128 -> 128 -> 10, GELU (tanh form) after each hidden
layer; inputs are affinely normalised by fixed constants.  The network's
targets are the outputs in covariance form (`net_targets`: the second moments
minus the products of the first), standardised per output by a mean and a
standard deviation (`norm`).
Loss: mean over rows and outputs of LOSS_W[k] (prediction - normalised
target)^2, log P weighted above the moments because the log-likelihood
depends on it directly.

Parameters are one flat vector [W1 (7x128, in x out), b1, W2 (128x128), b2,
W3, b3, W4 (128x10), b4] of 35338 values.

`label` computes the targets with the oracle's separation-of-variables
lattice rule (the plain evaluator), so the surrogate's error is judged by the
method it replaces.
"""
from __future__ import annotations

import math

import numpy as np

from . import cfust_oracle as O

DIMS = [7, 128, 128, 128, 10]
C_LO, C_HI = -8.0, 4.0   # C_LO <= c_t <= C_HI
RHO_MAX = 0.9        # |R_ht| <= RHO_MAX
PIVOT_MIN = 0.05     # every squared Cholesky pivot of R at least this
LOGM_LO, LOGM_HI = math.log(3.0), math.log(30.0)


def n_params() -> int:
    return sum(DIMS[k] * DIMS[k + 1] + DIMS[k + 1] for k in range(4))


def unpack(theta):
    """Flat parameter vector -> [(W1, b1), .., (W4, b4)] views."""
    out, off = [], 0
    for k in range(4):
        a, b = DIMS[k], DIMS[k + 1]
        W = theta[off:off + a * b].reshape(a, b)
        off += a * b
        bias = theta[off:off + b]
        off += b
        out.append((W, bias))
    return out


def normalise_inputs(x):
    """c and log m mapped affinely from their ranges onto [-1, 1], rho / RHO_MAX."""
    x = np.asarray(x, dtype=np.float64)
    u = np.empty_like(x)
    u[:, 0:3] = (2.0 * x[:, 0:3] - (C_LO + C_HI)) / (C_HI - C_LO)
    u[:, 3:6] = x[:, 3:6] / RHO_MAX
    u[:, 6] = (2.0 * x[:, 6] - (LOGM_LO + LOGM_HI)) / (LOGM_HI - LOGM_LO)
    return u


LOSS_W = np.array([4.0] + [1.0] * 9)

GELU_K = math.sqrt(2.0 / math.pi)
GELU_A = 0.044715


def gelu(z):
    """0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))."""
    return 0.5 * z * (1.0 + np.tanh(GELU_K * (z + GELU_A * z ** 3)))


def gelu_grad(z):
    t = np.tanh(GELU_K * (z + GELU_A * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * GELU_K * (1.0 + 3.0 * GELU_A * z * z)


def forward(theta, u):
    """Network output for normalised inputs u [B, 7]; also the cache for backward."""
    layers = unpack(theta)
    h = u
    cache = [(h, None)]
    for k, (W, b) in enumerate(layers):
        z = h @ W + b
        h = gelu(z) if k < 3 else z
        cache.append((h, z))
    return h, cache


def loss_and_grad(theta, u, t):
    """Weighted mean squared error against normalised targets t [B, 10] and its gradient."""
    out, cache = forward(theta, u)
    B = u.shape[0]
    diff = out - t
    loss = float(np.mean(LOSS_W * diff * diff))
    layers = unpack(theta)
    grads = []
    d = 2.0 * LOSS_W * diff / diff.size             # d loss / d out
    for k in range(3, -1, -1):
        h_in = cache[k][0]
        W, _ = layers[k]
        gW = h_in.T @ d
        gb = d.sum(axis=0)
        grads.append((gW, gb))
        if k > 0:
            dh = d @ W.T
            d = dh * gelu_grad(cache[k][1])
    grads.reverse()
    flat = np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])
    del B
    return loss, flat


def in_domain(x):
    """Inputs inside the training domain (the same test the E-step applies)."""
    x = np.asarray(x, dtype=np.float64)
    ok = np.all((x[:, 0:3] >= C_LO) & (x[:, 0:3] <= C_HI), axis=1)
    ok &= np.all(np.abs(x[:, 3:6]) <= RHO_MAX, axis=1)
    ok &= (x[:, 6] >= LOGM_LO) & (x[:, 6] <= LOGM_HI)
    r12, r13, r23 = x[:, 3], x[:, 4], x[:, 5]
    p2 = 1.0 - r12 * r12
    with np.errstate(invalid="ignore", divide="ignore"):
        l32 = (r23 - r13 * r12) / np.sqrt(np.maximum(p2, 1e-300))
        p3 = 1.0 - r13 * r13 - l32 * l32
    ok &= (p2 >= PIVOT_MIN) & (p3 >= PIVOT_MIN)
    return ok


UPPER = [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]


NEGLOG_MIN = 1e-12   # floor of -log P in the target log(-log P)


def net_targets(y, norm=None):
    """Outputs -> network targets: log(-log P) (relative precision for P near
    1, where most posterior weight sits), E[X] unchanged, second moments
    replaced by the truncated covariance E[X_a X_b] - E[X_a] E[X_b]; with
    norm = (mean[10], std[10]) also standardised."""
    y = np.asarray(y, dtype=np.float64)
    t = y.copy()
    t[:, 0] = np.log(np.maximum(-y[:, 0], NEGLOG_MIN))
    for k, (a, b) in enumerate(UPPER):
        t[:, 4 + k] = y[:, 4 + k] - y[:, 1 + a] * y[:, 1 + b]
    if norm is not None:
        norm = np.asarray(norm, dtype=np.float64)
        t = (t - norm[:10]) / norm[10:]
    return t


def from_net(t, norm=None):
    """Inverse of net_targets."""
    t = np.asarray(t, dtype=np.float64)
    if norm is not None:
        norm = np.asarray(norm, dtype=np.float64)
        t = t * norm[10:] + norm[:10]
    y = t.copy()
    y[:, 0] = -np.exp(t[:, 0])
    for k, (a, b) in enumerate(UPPER):
        y[:, 4 + k] = t[:, 4 + k] + t[:, 1 + a] * t[:, 1 + b]
    return y


def label(x, U, m_grid=None):
    """Targets of inputs x [B, 7] by the lattice rule U ([N, 4] baker points):
    log P(X > c), E[X | X > c], E[X X^T | X > c] (upper triangle).
    With m_grid, log m is first snapped to the nearest grid value (the GPU
    labeller uses chi tables on such a grid)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((x.shape[0], 10))
    for b in range(x.shape[0]):
        c = x[b, 0:3]
        R = np.array([[1.0, x[b, 3], x[b, 4]], [x[b, 3], 1.0, x[b, 5]], [x[b, 4], x[b, 5], 1.0]])
        L = np.linalg.cholesky(R)
        m = math.exp(x[b, 6])
        if m_grid is not None:
            m = float(m_grid[np.argmin(np.abs(np.log(m_grid) - x[b, 6]))])
        T, EV, EVV = O.sov_pass(c[None, :], L, m, U, True)
        EX = L @ EV[0]
        EXX = L @ EVV[0] @ L.T
        out[b, 0] = math.log(T[0])
        out[b, 1:4] = EX
        out[b, 4:10] = [EXX[0, 0], EXX[0, 1], EXX[0, 2], EXX[1, 1], EXX[1, 2], EXX[2, 2]]
    return out
