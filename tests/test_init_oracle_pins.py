"""Pins of the initial-value oracle (oracle/init_oracle.py) against things
other than itself: library quadrature and densities, scikit-learn's Lloyd
k-means, Monte Carlo draws of the CFUST law, and the invariants that define
each rule (moment matching, fixed points, the halving rule).
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import init_oracle as IO
from paper_2005_06848_gb300 import synth


@pytest.mark.parametrize("nu", [3.0, 5.0, 10.0, 30.0])
def test_abs_t_moments_against_quadrature(nu):
    m1, C = IO.abs_t_moments(nu, 3)
    q1 = 2.0 * integrate.quad(lambda x: x * stats.t.pdf(x, nu), 0, np.inf, epsabs=1e-13)[0]
    assert abs(m1 - q1) <= 1e-9
    # E U^2 is the t variance
    assert abs(C[0, 0] - (stats.t.var(nu) - q1 * q1)) <= 1e-9
    # E|U1||U2| from the bivariate t density (identity scale), four quadrants
    mt = stats.multivariate_t(loc=[0.0, 0.0], shape=np.eye(2), df=nu)
    q2, _ = integrate.dblquad(lambda y, x: x * y * mt.pdf([x, y]), 0, np.inf, 0, np.inf, epsabs=1e-11)
    assert abs(C[0, 1] - (4.0 * q2 - q1 * q1)) <= 1e-7
    assert np.allclose(C, C.T)


def test_cfust_moments_against_monte_carlo():
    """Mean and covariance of a CFUST law with a full (non-diagonal) Delta:
    the sample moments of 400k draws agree within 5 standard errors."""
    rng = np.random.default_rng(3)
    p, r, nu = 3, 2, 12.0
    P = synth.Params(pi=np.array([1.0]), mu=np.array([[0.5, -1.0, 2.0]]),
                     Sigma=np.array([[[1.0, 0.3, -0.2], [0.3, 1.5, 0.1], [-0.2, 0.1, 0.8]]]),
                     Delta=np.array([[[1.2, -0.4], [0.3, 0.9], [-0.7, 0.5]]]), nu=np.array([nu]))
    Y, _ = synth.sample_cfust(P, 400_000, rng)
    mean, cov = IO.cfust_moments(P.mu[0], P.Sigma[0], P.Delta[0], nu)
    n = Y.shape[0]
    se_mean = Y.std(axis=0) / math.sqrt(n)
    assert np.all(np.abs(Y.mean(axis=0) - mean) <= 5 * se_mean)
    Z = Y - Y.mean(axis=0)
    for a in range(p):
        for b in range(a + 1):
            prod = Z[:, a] * Z[:, b]
            se = prod.std() / math.sqrt(n)
            assert abs(prod.mean() - cov[a, b]) <= 5 * se, (a, b, prod.mean(), cov[a, b], se)


def _data(seed=0, n=3000):
    Y, labels, truth, init, _, meta = synth.workload("cfust_p4r4g3_n100000_N4096", n=n, seed=seed)
    return Y, labels, truth


def test_moment_init_matches_group_moments():
    """Psi^(0) reproduces each group's sample mean and covariance exactly, its
    weights are the group shares, its Delta follows the skewness signs."""
    Y, labels, truth = _data()
    g, r = truth.g, truth.r
    pi, mu, Sigma, Delta, nu, lam = IO.moment_init(Y, labels, g, r, nu0=8.0, lam=0.5)
    assert np.allclose(nu, 8.0)
    for i in range(g):
        Yi = Y[labels == i]
        assert pi[i] == Yi.shape[0] / Y.shape[0]
        mean, cov = IO.cfust_moments(mu[i], Sigma[i], Delta[i], nu[i])
        S = np.cov(Yi.T, bias=True)
        assert np.allclose(mean, Yi.mean(axis=0), rtol=0, atol=1e-12 * np.abs(Yi).max())
        assert np.allclose(cov, S, rtol=1e-12, atol=1e-12 * np.abs(S).max())
        skew = stats.skew(Yi, axis=0)
        sd = Yi.std(axis=0)
        k = min(Y.shape[1], r)
        assert np.allclose(np.diag(Delta[i][:k, :k]), lam[i] * np.where(skew[:k] < 0, -1, 1) * sd[:k], rtol=1e-12)
        off = Delta[i].copy()
        off[np.arange(k), np.arange(k)] = 0.0
        assert np.all(off == 0.0)
        assert np.all(np.linalg.eigvalsh(Sigma[i]) > 0)


def test_moment_init_halves_until_positive_definite():
    """With lam far too large the rule keeps the largest lam / 2^h whose Sigma
    is positive definite: the previous (double) value is not."""
    Y, labels, truth = _data(seed=1)
    g, r = truth.g, truth.r
    nu0 = 4.0
    _, _, _, _, _, lam = IO.moment_init(Y, labels, g, r, nu0=nu0, lam=6.0)
    m1, C = IO.abs_t_moments(nu0, r)
    for i in range(g):
        assert 0.0 < lam[i] < 6.0
        assert math.log2(6.0 / lam[i]) == round(math.log2(6.0 / lam[i]))
        Yi = Y[labels == i]
        S = np.cov(Yi.T, bias=True)
        sign = np.where(stats.skew(Yi, axis=0) < 0, -1.0, 1.0)
        sd = Yi.std(axis=0)

        def sigma_at(l):
            D = np.zeros((Y.shape[1], r))
            for k in range(min(Y.shape[1], r)):
                D[k, k] = l * sign[k] * sd[k]
            return (nu0 - 2) / nu0 * (S - D @ C @ D.T)
        assert np.linalg.eigvalsh(sigma_at(lam[i])).min() > 0
        assert np.linalg.eigvalsh(sigma_at(2 * lam[i])).min() <= 0


def test_moment_init_rejects_small_groups():
    Y, labels, truth = _data(n=500)
    lab = labels.copy()
    lab[:] = 0
    lab[:4] = 1           # 4 members < p + 1 = 5
    with pytest.raises(IO.DegenerateGroup):
        IO.moment_init(Y, lab, 2, truth.r)
    with pytest.raises(ValueError):
        IO.moment_init(Y, labels, truth.g, truth.r, nu0=2.0)


def _seeds(Y, g, seed):
    rng = np.random.default_rng(seed)
    return Y[rng.choice(Y.shape[0], size=g, replace=False)].copy()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_kmeans_matches_scikit_learn_lloyd(seed):
    sk = pytest.importorskip("sklearn.cluster")
    Y, _, truth = _data(seed=seed, n=4000)
    c0 = _seeds(Y, truth.g, seed)
    labels, C, it = IO.kmeans(Y, c0, 300)
    km = sk.KMeans(n_clusters=truth.g, init=c0, n_init=1, max_iter=300, tol=0.0, algorithm="lloyd").fit(Y)
    assert it < 300
    assert np.array_equal(labels, km.labels_)
    assert np.allclose(C, km.cluster_centers_, rtol=1e-12, atol=1e-12)


def test_kmeans_invariants():
    """Objective never increases; the result is a fixed point: every label is
    the nearest centre (brute force) and every centre is its group's mean."""
    Y, _, truth = _data(seed=4, n=2500)
    c0 = _seeds(Y, truth.g, 9)
    prev = math.inf
    for iters in range(1, 12):
        labels, C, it = IO.kmeans(Y, c0, iters)
        obj = IO.kmeans_objective(Y, labels, C)
        assert obj <= prev * (1 + 1e-15)
        prev = obj
    labels, C, it = IO.kmeans(Y, c0, 500)
    dist = ((Y[:, None, :] - C[None, :, :]) ** 2).sum(axis=2)
    assert np.array_equal(labels, np.argmin(dist, axis=1))
    for i in range(truth.g):
        assert np.allclose(C[i], Y[labels == i].mean(axis=0), rtol=1e-13, atol=1e-13)


def test_kmeans_separated_clusters_recover_the_groups():
    rng = np.random.default_rng(5)
    centres = np.array([[0.0, 0.0], [20.0, 0.0], [0.0, 20.0]])
    truth = np.repeat(np.arange(3), 200)
    Y = centres[truth] + rng.standard_normal((600, 2))
    labels, C, it = IO.kmeans(Y, Y[[0, 200, 400]], 50)
    assert np.array_equal(labels, truth)
    assert np.allclose(C, centres, atol=0.3)
