"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module holds input construction only: the data recipe of the CFUST
mixture (the latent structure of Section 2: a gamma weight W, a half-normal
skew vector U and a normal error), the parameter draws of the benchmark
workloads, the perturbed starting values, and the rank-1 lattice rule
(generator vector and random shift) that the E-step integrates over.  It holds
none of the E- or M-step arithmetic.

Parameter arrays follow the model's notation (Eq. 2): ``pi[g]``, ``mu[g,p]``,
``Sigma[g,p,p]``, ``Delta[g,p,r]`` and ``nu[g]``; the skew dimension, written
``q`` in the paper, is called ``r`` here.
"""
from __future__ import annotations

import dataclasses
import functools
import math

import numpy as np

__all__ = [
    "Params", "Lattice", "splitmix64_stream", "korobov_generator",
    "make_lattice", "sample_cfust", "perturb_params", "random_params",
    "workload", "WORKLOADS", "batched_workload", "random_partitions", "initial_centres",
]


@dataclasses.dataclass
class Params:
    """Mixture parameters Psi = (pi, mu, Sigma, Delta, nu) of Section 2 / Eq. 2."""
    pi: np.ndarray
    mu: np.ndarray
    Sigma: np.ndarray
    Delta: np.ndarray
    nu: np.ndarray

    @property
    def g(self) -> int:
        return int(self.pi.shape[0])

    @property
    def p(self) -> int:
        return int(self.mu.shape[1])

    @property
    def r(self) -> int:
        return int(self.Delta.shape[2])

    def copy(self) -> "Params":
        return Params(*(np.array(a, dtype=np.float64, copy=True) for a in
                        (self.pi, self.mu, self.Sigma, self.Delta, self.nu)))

    def as_arrays(self):
        return (self.pi, self.mu, self.Sigma, self.Delta, self.nu)


@dataclasses.dataclass
class Lattice:
    """Shifted rank-1 lattice rule: point k is frac(k*z/n + shift), k = 0..n-1.

    Coordinate 0 drives the chi-square mixing variable, coordinates 1..r the
    r normal variables of the separation-of-variables integrand.
    """
    n: int
    z: np.ndarray      # int64 [dim]
    shift: np.ndarray  # float64 [dim], each in [0, 1)

    @property
    def dim(self) -> int:
        return int(self.z.shape[0])


_MASK64 = (1 << 64) - 1


def splitmix64_stream(seed: int, count: int) -> list[int]:
    """``count`` successive outputs of Vigna's SplitMix64 generator from ``seed``."""
    out = []
    x = seed & _MASK64
    for _ in range(count):
        x = (x + 0x9E3779B97F4A7C15) & _MASK64
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out.append(z ^ (z >> 31))
    return out


# Results of the search below for sizes whose search takes tens of seconds
# (the 2^16-point reference rule); tests/test_synth_lattice.py re-runs the
# search for every entry.
KOROBOV_TABLE = {(65536, 4): 1443, (65536, 5): 15845}


@functools.lru_cache(maxsize=None)
def korobov_generator(n: int, dim: int) -> int:
    """Korobov parameter a (generator (1, a, a^2, ...) mod n) minimising P_2.

    P_2 is the worst-case error of the lattice rule for periodic integrands with
    square-integrable mixed first derivatives:
    P_2(z) = -1 + (1/n) sum_k prod_d (1 + 2 pi^2 B_2({k z_d / n})),
    B_2(x) = x^2 - x + 1/6.  Ties go to the smallest a.  Up to 4096 candidates
    coprime to n are tried (all of them for n <= 8192).
    """
    if dim < 1 or n < 2:
        raise ValueError("need n >= 2 and dim >= 1")
    if dim == 1:
        return 1
    if (n, dim) in KOROBOV_TABLE:
        return KOROBOV_TABLE[(n, dim)]
    return korobov_search(n, dim)


def korobov_search(n: int, dim: int) -> int:
    """The P_2 search of korobov_generator, without the table."""
    cands = np.array([a for a in range(2, n) if math.gcd(a, n) == 1], dtype=np.int64)
    if cands.size > 4096:
        # large n: search an evenly spread subset (the criterion costs O(n) per candidate)
        cands = cands[np.linspace(0, cands.size - 1, 4096).astype(np.int64)]
    k = np.arange(n, dtype=np.int64)
    best_a, best_val = None, np.inf
    for c0 in range(0, cands.size, 128):
        block = cands[c0:c0 + 128]
        prod = np.ones((block.size, n))
        zd = np.ones(block.size, dtype=np.int64)
        for _ in range(dim):
            x = ((zd[:, None] * k[None, :]) % n) / n
            prod *= 1.0 + 2.0 * math.pi ** 2 * (x * x - x + 1.0 / 6.0)
            zd = (zd * block) % n
        vals = prod.mean(axis=1) - 1.0
        i = int(np.argmin(vals))
        if best_a is None or vals[i] < best_val - 1e-15 * abs(best_val):
            best_val, best_a = float(vals[i]), int(block[i])
    return best_a


def make_lattice(n: int, dim: int, seed: int = 0) -> Lattice:
    """Korobov lattice of ``n`` points in ``dim`` dimensions with a SplitMix64 shift.

    shift_d = (splitmix64 output d >> 11) * 2^-53, a double in [0, 1).
    """
    a = korobov_generator(int(n), int(dim))
    z = np.array([pow(a, d, n) for d in range(dim)], dtype=np.int64)
    shift = np.array([(v >> 11) * 2.0 ** -53 for v in splitmix64_stream(seed, dim)],
                     dtype=np.float64)
    return Lattice(n=int(n), z=z, shift=shift)


def sample_cfust(params: Params, n: int, rng: np.random.Generator):
    """Draw n observations from the CFUST mixture.

    y = mu_i + W^{-1/2} (Delta_i |U0| + e) with U0 ~ N_r(0, I), e ~ N_p(0, Sigma_i),
    W ~ Gamma(nu_i/2, rate nu_i/2) and the label i ~ Categorical(pi): the latent
    gamma / truncated-normal representation named in Section 2.
    Returns (Y[n,p] float64 C-contiguous, labels[n] int64).
    """
    g, p, r = params.g, params.p, params.r
    labels = rng.choice(g, size=n, p=params.pi)
    Y = np.empty((n, p))
    for i in range(g):
        idx = np.nonzero(labels == i)[0]
        m = idx.size
        if m == 0:
            continue
        w = rng.gamma(shape=params.nu[i] / 2.0, scale=2.0 / params.nu[i], size=m)
        u0 = np.abs(rng.standard_normal((m, r)))
        Ls = np.linalg.cholesky(params.Sigma[i])
        e = rng.standard_normal((m, p)) @ Ls.T
        Y[idx] = params.mu[i] + (u0 @ params.Delta[i].T + e) / np.sqrt(w)[:, None]
    return np.ascontiguousarray(Y), labels


def _wishart_scaled(rng, p, df):
    x = rng.standard_normal((df, p))
    return (x.T @ x) / df


def random_params(rng, g, p, r, mu_var, wishart_extra, delta_half, nu_lo, nu_hi) -> Params:
    """Component parameters drawn as in the large synthetic workloads.

    mu_i ~ N(0, mu_var I); Sigma_i = Wishart(p + wishart_extra, I)/(p + wishart_extra);
    Delta_i entries U(-delta_half, delta_half); nu_i ~ U(nu_lo, nu_hi); pi equal.
    """
    mu = rng.normal(0.0, math.sqrt(mu_var), size=(g, p))
    Sigma = np.stack([_wishart_scaled(rng, p, p + wishart_extra) for _ in range(g)])
    Delta = rng.uniform(-delta_half, delta_half, size=(g, p, r))
    nu = rng.uniform(nu_lo, nu_hi, size=g)
    pi = np.full(g, 1.0 / g)
    return Params(pi, mu, Sigma, Delta, nu)


def perturb_params(truth: Params, rng: np.random.Generator, sd: float = 0.3) -> Params:
    """Starting values 'truth + N(0, sd)'.

    mu and Delta get N(0, sd^2) added entrywise; Sigma's Cholesky factor gets
    N(0, sd^2) on its lower triangle and is re-formed (kept positive definite by
    a diagonal floor); pi is perturbed, clipped at 0.05 and renormalised; nu is
    perturbed in log space.
    """
    g, p, r = truth.g, truth.p, truth.r
    mu = truth.mu + rng.normal(0.0, sd, size=(g, p))
    Delta = truth.Delta + rng.normal(0.0, sd, size=(g, p, r))
    Sigma = np.empty_like(truth.Sigma)
    for i in range(g):
        L = np.linalg.cholesky(truth.Sigma[i])
        L = L + np.tril(rng.normal(0.0, sd, size=(p, p)))
        dg = np.maximum(np.abs(np.diag(L)), 0.1)
        L[np.diag_indices(p)] = dg
        Sigma[i] = L @ L.T
    pi = np.clip(truth.pi + rng.normal(0.0, sd, size=g) * truth.pi, 0.05, None)
    pi = pi / pi.sum()
    nu = truth.nu * np.exp(rng.normal(0.0, sd, size=g))
    return Params(pi, mu, Sigma, Delta, nu)


def _workload_small_p2(seed=0):
    """p=2, r=2, g=2 fit with fixed truth; Delta entries U(-2, 2); nu = (4, 8)."""
    rng = np.random.default_rng(seed)
    pi = np.array([0.4, 0.6])
    mu = np.array([[0.0, 0.0], [4.0, 3.0]])
    Sigma = np.array([np.eye(2), [[1.0, 0.5], [0.5, 1.0]]])
    Delta = rng.uniform(-2.0, 2.0, size=(2, 2, 2))
    nu = np.array([4.0, 8.0])
    return Params(pi, mu, Sigma, Delta, nu), rng


WORKLOADS = {
    # name: (n, g, p, r, lattice points, EM iterations)
    "cfust_p2r2g2_n2000_N1024": dict(n=2000, g=2, p=2, r=2, lattice_n=1024, iters=20),
    "cfust_p4r4g3_n100000_N4096": dict(n=100000, g=3, p=4, r=4, lattice_n=4096, iters=50),
    "cfust_p3r3g4_n1000000_N2048": dict(n=1000000, g=4, p=3, r=3, lattice_n=2048, iters=30),
    "cfust_p8r4g6_n1000000_N8192": dict(n=1000000, g=6, p=8, r=4, lattice_n=8192, iters=30),
}


def workload(name: str, n: int | None = None, seed: int = 0):
    """Build (Y, labels, truth, init, lattice, meta) for a named synthetic workload.

    ``n`` overrides the row count (rows are a prefix of the same seeded draw
    only for the fixed-truth small workload; larger workloads redraw).
    """
    meta = dict(WORKLOADS[name])
    if n is not None:
        meta["n"] = int(n)
    g, p, r = meta["g"], meta["p"], meta["r"]
    if name.startswith("cfust_p2r2g2"):
        truth, rng = _workload_small_p2(seed)
    elif name.startswith("cfust_p4r4g3"):
        rng = np.random.default_rng(seed)
        truth = random_params(rng, g, p, r, 9.0, 2, 3.0, 3.0, 12.0)
    elif name.startswith("cfust_p3r3g4"):
        rng = np.random.default_rng(seed)
        truth = random_params(rng, g, p, r, 9.0, 2, 2.0, 3.0, 12.0)
    elif name.startswith("cfust_p8r4g6"):
        rng = np.random.default_rng(seed)
        truth = random_params(rng, g, p, r, 16.0, 4, 2.0, 3.0, 20.0)
    else:
        raise KeyError(name)
    Y, labels = sample_cfust(truth, meta["n"], rng)
    init = perturb_params(truth, rng)
    lattice = make_lattice(meta["lattice_n"], r + 1, seed)
    return Y, labels, truth, init, lattice, meta


def batched_workload(nfits: int = 256, seed0: int = 0, n_lo: int = 5000, n_hi: int = 200000,
                     p: int = 3, r: int = 3, g_lo: int = 2, g_hi: int = 5):
    """Many independent fits: fit f draws with seed seed0 + f its component
    count g ~ U{g_lo..g_hi}, its size n log-uniform in [n_lo, n_hi], its truth
    (mu ~ N(0, 9I), Sigma = Wishart(p+2, I)/(p+2), Delta ~ U(-2, 2),
    nu ~ U(3, 12), equal pi), its data, and a perturbed start (a random
    restart).  Returns (list of Y, list of truth, list of init)."""
    Ys, truths, inits = [], [], []
    for f in range(nfits):
        rng = np.random.default_rng(seed0 + f)
        g = int(rng.integers(g_lo, g_hi + 1))
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        truth = random_params(rng, g, p, r, 9.0, 2, 2.0, 3.0, 12.0)
        Y, _ = sample_cfust(truth, n, rng)
        Ys.append(Y)
        truths.append(truth)
        inits.append(perturb_params(truth, rng))
    return Ys, truths, inits


def random_partitions(n: int, g: int, m: int, seed: int = 0) -> np.ndarray:
    """m seeded random partitions of n observations into g groups (Algorithm 1's
    random initial partitions): int32 [m, n], labels uniform on 0..g-1."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(rng.integers(0, g, size=(m, n)).astype(np.int32))


def initial_centres(Y: np.ndarray, g: int, m: int, seed: int = 0) -> np.ndarray:
    """m seeded sets of k-means starting centres: g distinct observations each,
    float64 [m, g, p]."""
    rng = np.random.default_rng(seed)
    return np.stack([Y[rng.choice(Y.shape[0], size=g, replace=False)] for _ in range(m)]).astype(np.float64)
