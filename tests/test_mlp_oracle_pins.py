"""Pins of the surrogate network's FP64 oracle: its gradient against central
finite differences, GELU's derivative, the domain test against numpy's
Cholesky, and the labeller's limits (orthant probabilities, untruncated moments)."""
import math

import numpy as np
import pytest

from oracle import cfust_oracle as O
from oracle import mlp_oracle as M
from paper_2005_06848_gb300 import synth


def _theta(seed=0):
    rng = np.random.default_rng(seed)
    parts = []
    for k in range(4):
        a, b = M.DIMS[k], M.DIMS[k + 1]
        parts += [rng.normal(0, 1 / math.sqrt(a), size=a * b), rng.normal(0, 0.1, size=b)]
    return np.concatenate(parts)


def test_parameter_count():
    assert M.n_params() == 35338 == _theta().size


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(1)
    th = _theta(1)
    u = rng.uniform(-1, 1, size=(6, 7))
    t = rng.normal(size=(6, 10))
    loss, g = M.loss_and_grad(th, u, t)
    idx = rng.choice(th.size, 60, replace=False)
    idx = np.concatenate([idx, [0, 895, 896 + 127, th.size - 1, th.size - 11]])
    h = 1e-6
    for k in idx:
        tp, tm = th.copy(), th.copy()
        tp[k] += h
        tm[k] -= h
        fd = (M.loss_and_grad(tp, u, t)[0] - M.loss_and_grad(tm, u, t)[0]) / (2 * h)
        assert abs(fd - g[k]) <= 1e-7 * max(1.0, abs(fd)) + 1e-9, k


def test_gelu_values_and_derivative():
    z = np.linspace(-6, 6, 101)
    assert M.gelu(np.array([0.0]))[0] == 0.0
    assert np.allclose(M.gelu(np.array([8.0])), 8.0, atol=1e-12)
    assert np.allclose(M.gelu(np.array([-8.0])), 0.0, atol=1e-12)
    fd = (M.gelu(z + 1e-6) - M.gelu(z - 1e-6)) / 2e-6
    assert np.allclose(M.gelu_grad(z), fd, atol=1e-8)


def test_domain_test_matches_cholesky_pivots():
    rng = np.random.default_rng(4)
    x = np.column_stack([rng.uniform(-9, 5, (4000, 3)), rng.uniform(-1, 1, (4000, 3)),
                         rng.uniform(math.log(2), math.log(40), 4000)])
    ok = M.in_domain(x)
    for b in range(0, 4000, 7):
        R = np.array([[1, x[b, 3], x[b, 4]], [x[b, 3], 1, x[b, 5]], [x[b, 4], x[b, 5], 1]])
        try:
            piv = np.diag(np.linalg.cholesky(R)) ** 2
            pd = bool(np.all(piv >= M.PIVOT_MIN))
        except np.linalg.LinAlgError:
            pd = False
        ref = (pd and np.all((x[b, :3] >= M.C_LO) & (x[b, :3] <= M.C_HI))
               and np.all(np.abs(x[b, 3:6]) <= M.RHO_MAX)
               and M.LOGM_LO <= x[b, 6] <= M.LOGM_HI)
        assert ok[b] == ref, b


def test_label_limits():
    lat = synth.make_lattice(4096, 4, 0)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    r12, r13, r23, m = 0.3, -0.2, 0.5, 7.0
    R = np.array([[1, r12, r13], [r12, 1, r23], [r13, r23, 1]])
    # orthant: c = 0
    y0 = M.label(np.array([[0, 0, 0, r12, r13, r23, math.log(m)]]), U)[0]
    ex = 0.125 + (math.asin(r12) + math.asin(r13) + math.asin(r23)) / (4 * math.pi)
    assert abs(math.exp(y0[0]) - ex) < 2e-5
    # no truncation in effect: c far below, P = 1, E[X] = 0, E[X X^T] = m/(m-2) R
    y1 = M.label(np.array([[-60, -60, -60, r12, r13, r23, math.log(m)]]), U)[0]
    assert abs(y1[0]) < 1e-12
    assert np.allclose(y1[1:4], 0.0, atol=2e-3)
    full = m / (m - 2) * R
    # (the lattice resolves E[1/s^2] to a few percent at this N: chi-scale singularity)
    assert np.allclose(y1[4:10], [full[0, 0], full[0, 1], full[0, 2], full[1, 1], full[1, 2], full[2, 2]],
                       atol=0.05)


def test_net_targets_are_covariances_and_invert():
    # the covariance form of an untruncated problem is m/(m-2) R with zero mean;
    # a point mass at v has zero covariance
    rng = np.random.default_rng(9)
    y = rng.normal(size=(5, 10))
    y[:, 0] = -np.exp(rng.normal(size=5) * 3)            # log P < 0
    norm = np.r_[rng.normal(size=10), rng.uniform(0.5, 2, 10)]
    assert np.allclose(M.from_net(M.net_targets(y, norm), norm), y, atol=1e-12)
    v = np.array([0.5, -1.0, 2.0])
    pm = np.r_[-0.25, v, [v[a] * v[b] for a, b in M.UPPER]][None, :]
    assert np.allclose(M.net_targets(pm)[0, 4:], 0.0, atol=1e-15)
    assert np.allclose(M.net_targets(pm)[0, 1:4], pm[0, 1:4])
    assert np.isclose(M.net_targets(pm)[0, 0], math.log(0.25))
