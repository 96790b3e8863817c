"""Plain FP64 CPU oracle for the initial values of Algorithm 1.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this module.  It shares
no code with the CUDA path.

Algorithm 1 (Section 3.1, parallel initialisation) starts from m initial
partitions of the data, obtained "for example" by k-means or at random, and
each thread computes Psi^(0) from its partition; the paper does not say how.
Readings of this library (each one is a plain, checkable rule):

* k-means: Lloyd's iterations from given centres.  One iteration assigns
  every observation to its nearest centre (squared Euclidean distance
  accumulated over the coordinates in order, ties to the lowest index), stops
  when no label changed since the previous assignment, and otherwise moves
  each centre to the mean of its members (a centre without members stays).
* Psi^(0) from a partition, by moments.  For group i (n_i >= p + 1 members):
  pi_i = n_i / n and nu_i = nu0 (> 2, given).  Delta_i is diagonal in its
  first min(p, r) columns: Delta_i[k, k] = lam sign(skew_k) sd_k, with sd_k
  and skew_k the group's sample standard deviation and skewness of
  coordinate k (sign +1 at zero skewness), other entries zero.  mu_i and
  Sigma_i then match the group's sample mean and covariance (divisor n_i)
  to those of the CFUST law (``cfust_moments``):
      mu_i    = ybar_i - m1 Delta_i 1_r,
      Sigma_i = (nu0 - 2)/nu0 (S_i - Delta_i C Delta_i^T),
  where m1 = E|U_k| and C = Cov(|U|) for U ~ t_r(0, I, nu0).  If Sigma_i is
  not positive definite, lam is halved (up to 20 times, then lam = 0).
"""
from __future__ import annotations

import math

import numpy as np

MAX_HALVINGS = 20


class DegenerateGroup(ValueError):
    """A group of the partition has fewer than p + 1 members, or its sample
    covariance is not positive definite."""


def kmeans(Y, centers0, max_iter):
    """Lloyd's k-means from ``centers0`` ([g, p]).

    Returns (labels [n] int32, centers [g, p], iterations), where iterations
    counts the assignment passes (the last one changed nothing unless
    max_iter ran out).
    """
    Y = np.asarray(Y, dtype=np.float64)
    C = np.array(centers0, dtype=np.float64, copy=True)
    n, p = Y.shape
    g = C.shape[0]
    labels = None
    it = 0
    for it in range(1, max_iter + 1):
        D = np.empty((n, g))
        for i in range(g):
            d = np.zeros(n)
            for k in range(p):
                t = Y[:, k] - C[i, k]
                d = d + t * t
            D[:, i] = d
        new = np.argmin(D, axis=1).astype(np.int32)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for i in range(g):
            members = labels == i
            if members.any():
                C[i] = Y[members].mean(axis=0)
    return labels, C, it


def kmeans_objective(Y, labels, centers):
    """Sum of squared distances of the observations to their centres."""
    diff = np.asarray(Y) - np.asarray(centers)[labels]
    return float(np.sum(diff * diff))


def abs_t_moments(nu, r):
    """m1 = E|U_k| and C = Cov(|U|) for U ~ t_r(0, I, nu), nu > 2.

    With U = Z / sqrt(W), Z ~ N_r(0, I), W ~ Gamma(nu/2, rate nu/2):
    E|Z_k| = sqrt(2/pi), E[W^-1/2] = sqrt(nu/2) Gamma((nu-1)/2) / Gamma(nu/2),
    E[1/W] = nu / (nu - 2); so m1 = sqrt(nu/pi) Gamma((nu-1)/2) / Gamma(nu/2),
    E U_k^2 = nu/(nu-2) and E|U_k||U_l| = (2/pi) nu/(nu-2) for k != l.
    """
    nu = float(nu)
    m1 = math.exp(0.5 * math.log(nu / math.pi) + math.lgamma(0.5 * (nu - 1.0)) - math.lgamma(0.5 * nu))
    s = nu / (nu - 2.0)
    C = np.full((r, r), (2.0 / math.pi) * s - m1 * m1)
    np.fill_diagonal(C, s - m1 * m1)
    return m1, C


def cfust_moments(mu, Sigma, Delta, nu):
    """Mean and covariance of one CFUST component (Eq. 2's law), nu > 2.

    Y = mu + Delta |U| + E with (U, E) ~ t_{r+p}(0, diag(I, Sigma), nu):
    E[Y] = mu + m1 Delta 1_r and Cov(Y) = nu/(nu-2) Sigma + Delta C Delta^T
    (|U| and E are uncorrelated: E is symmetric given the common W).
    """
    Delta = np.asarray(Delta, dtype=np.float64)
    m1, C = abs_t_moments(nu, Delta.shape[1])
    mean = np.asarray(mu, dtype=np.float64) + m1 * Delta.sum(axis=1)
    cov = nu / (nu - 2.0) * np.asarray(Sigma, dtype=np.float64) + Delta @ C @ Delta.T
    return mean, cov


def _is_pd(S):
    """Textbook Cholesky: positive definite iff every pivot is positive."""
    p = S.shape[0]
    L = np.zeros_like(S)
    for j in range(p):
        s = S[j, j] - np.dot(L[j, :j], L[j, :j])
        if not (s > 0.0) or not np.isfinite(s):
            return False
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, p):
            L[i, j] = (S[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    return True


def group_moments(Y, labels, g):
    """Per group: count, sample mean, covariance (divisor n_i), third central
    moments of the coordinates."""
    Y = np.asarray(Y, dtype=np.float64)
    out = []
    for i in range(g):
        Yi = Y[np.asarray(labels) == i]
        ni = Yi.shape[0]
        if ni == 0:
            out.append((0, None, None, None))
            continue
        ybar = Yi.mean(axis=0)
        Z = Yi - ybar
        out.append((ni, ybar, Z.T @ Z / ni, (Z ** 3).mean(axis=0)))
    return out


def moment_init(Y, labels, g, r, nu0=10.0, lam=0.5):
    """Psi^(0) from a partition by the moment rule above.

    Returns (pi [g], mu [g,p], Sigma [g,p,p], Delta [g,p,r], nu [g], lam_used [g]).
    Raises DegenerateGroup for a group with fewer than p + 1 members or a
    sample covariance that is not positive definite.
    """
    Y = np.asarray(Y, dtype=np.float64)
    n, p = Y.shape
    if not nu0 > 2.0:
        raise ValueError("nu0 must exceed 2 (finite covariance)")
    m1, C = abs_t_moments(nu0, r)
    pi = np.zeros(g)
    mu = np.zeros((g, p))
    Sigma = np.zeros((g, p, p))
    Delta = np.zeros((g, p, r))
    lam_used = np.zeros(g)
    for i, (ni, ybar, S, m3) in enumerate(group_moments(Y, labels, g)):
        if ni < p + 1 or not _is_pd(S):
            raise DegenerateGroup(f"group {i}: {ni} members")
        sd = np.sqrt(np.diag(S))
        sign = np.where(m3 < 0.0, -1.0, 1.0)
        li = float(lam)
        for h in range(MAX_HALVINGS + 2):
            if h == MAX_HALVINGS + 1:
                li = 0.0
            D = np.zeros((p, r))
            for k in range(min(p, r)):
                D[k, k] = li * sign[k] * sd[k]
            Sig = (nu0 - 2.0) / nu0 * (S - D @ C @ D.T)
            if _is_pd(Sig):
                break
            li *= 0.5
        pi[i] = ni / n
        mu[i] = ybar - m1 * D.sum(axis=1)
        Sigma[i] = Sig
        Delta[i] = D
        lam_used[i] = li
    return pi, mu, Sigma, Delta, np.full(g, float(nu0)), lam_used
