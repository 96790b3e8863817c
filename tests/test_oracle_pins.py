"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form, an exact
identity, a library routine for a special case, or brute-force Monte Carlo.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _U(n, dim, seed=0):
    lat = synth.make_lattice(n, dim, seed)
    return O.lattice_points(n, lat.z, lat.shift)


def _params(mu, Sigma, Delta, nu, pi):
    return synth.Params(np.asarray(pi, float), np.asarray(mu, float), np.asarray(Sigma, float),
                        np.asarray(Delta, float), np.asarray(nu, float))


# --------------------------------------------------------------------------- lattice / chi scale

def test_lattice_points_in_open_unit_cube_and_baker_symmetric():
    U = _U(1024, 4, 7)
    assert U.shape == (1024, 4)
    assert np.all(U > 0) and np.all(U < 1)
    # coordinate 0 has generator 1: its un-transformed values are an equally spaced
    # grid, so after the baker's transform the values come in mirror pairs.
    v = np.sort(U[:, 0])
    assert np.allclose(v[0::2], v[1::2], atol=1e-15) or np.unique(v).size >= 512


def test_chi_scale_inverts_incomplete_gamma():
    """P(chi^2_m <= m s^2) must equal the lattice coordinate (definition of a quantile)."""
    u = np.array([1e-15, 1e-6, 0.01, 0.3, 0.5, 0.77, 0.999, 1 - 1e-12])
    for m in (2.5, 6.0, 13.7, 30.0):
        s = O.chi_scale(u, m)
        back = np.where(u < 0.5, special.gammainc(m / 2, m * s * s / 2),
                        1 - special.gammaincc(m / 2, m * s * s / 2))
        assert np.allclose(back, u, rtol=1e-12, atol=1e-15)


def test_chi_scale_mean_square_is_one():
    """E[chi^2_m / m] = 1, integrated over the lattice's first coordinate."""
    U = _U(1 << 14, 2, 0)
    for m in (4.0, 9.5):
        s = O.chi_scale(U[:, 0], m)
        assert abs(np.mean(s * s) - 1.0) < 1e-5


# --------------------------------------------------------------------------- r = 1 closed forms

def _t_trunc_closed(c, m):
    """Z ~ t_m given Z > c: P, E[Z], E[Z^2] (integration by parts of the t density)."""
    S0 = stats.t.sf(c, m)
    f = stats.t.pdf(c, m)
    E1 = f * (m + c * c) / ((m - 1) * S0)
    E2 = (c * f * (m + c * c) + m * S0) / ((m - 2) * S0)
    return S0, E1, E2


@pytest.mark.parametrize("m", [5.0, 6.3, 12.5])
def test_r1_matches_univariate_t_closed_forms(m):
    a = np.array([[-1.5], [-0.3], [0.0], [0.7], [1.6]])
    l = 0.8
    S0, E1, E2 = _t_trunc_closed(a[:, 0] / l, m)
    errs = []
    for N in (128, 1 << 14):
        T, EV, EVV = O.sov_pass(a, np.array([[l]]), m, _U(N, 2, 3), True)
        errs.append(np.max(np.abs(T - S0) / S0))
        if N == 1 << 14:
            assert np.allclose(T, S0, rtol=2e-5)
            assert np.allclose(EV[:, 0], E1, rtol=2e-3)
            assert np.allclose(EVV[:, 0, 0], E2, rtol=1e-2)
    assert errs[1] < errs[0]


def test_r1_tail_error_shrinks_with_lattice_size():
    """Tail limits converge more slowly (chi-scale singularity) but do converge."""
    a = np.array([[2.5], [5.0]])
    l, m = 0.8, 6.3
    S0, _, _ = _t_trunc_closed(a[:, 0] / l, m)
    e = [np.max(np.abs(O.sov_pass(a, np.array([[l]]), m, _U(N, 2, 0), False) - S0) / S0)
         for N in (1024, 1 << 16)]
    assert e[1] < 2e-3 and e[1] < e[0] / 10


# --------------------------------------------------------------------------- orthants, identity Lambda

def test_orthant_probabilities_r2_r3():
    """P(X > 0) for an elliptical law: 1/4 + asin(rho)/(2 pi) (r=2) and
    1/8 + sum asin(rho_ht)/(4 pi) (r=3), with rho the correlations of Lambda."""
    rng = np.random.default_rng(0)
    for r in (2, 3):
        A = rng.standard_normal((r, r))
        Lam = A @ A.T + 0.5 * np.eye(r)
        D = np.sqrt(np.diag(Lam))
        R = Lam / np.outer(D, D)
        if r == 2:
            ex = 0.25 + math.asin(R[0, 1]) / (2 * math.pi)
        else:
            ex = 0.125 + (math.asin(R[0, 1]) + math.asin(R[0, 2]) + math.asin(R[1, 2])) / (4 * math.pi)
        for m in (3.5, 11.0):
            T = O.sov_pass(np.zeros((1, r)), np.linalg.cholesky(Lam), m, _U(4096, r + 1, 2), False)
            assert abs(T[0] - ex) < 2e-5


def test_random_shifts_give_an_unbiased_rule_and_an_honest_error_estimate():
    """Randomised QMC: with independent uniform shifts the lattice estimate of
    an orthant probability (closed form: 1/4 + asin(rho)/(2 pi)) is unbiased
    and the spread over shifts bounds its error: over 120 shifts of a small
    64-point rule the mean lies within 4 standard errors of the exact value,
    while single shifts do miss it by more than their own standard error."""
    rng = np.random.default_rng(7)
    Lam = np.array([[1.0, 0.6], [0.6, 1.0]])
    ex = 0.25 + math.asin(0.6) / (2 * math.pi)
    z = synth.make_lattice(64, 3, 0).z
    L = np.linalg.cholesky(Lam)
    Ts = np.array([O.sov_pass(np.zeros((1, 2)), L, 6.0, O.lattice_points(64, z, rng.uniform(size=3)), False)[0]
                   for _ in range(120)])
    se = Ts.std(ddof=1) / math.sqrt(Ts.size)
    assert se > 0
    assert abs(Ts.mean() - ex) <= 4 * se, (Ts.mean(), ex, se)
    assert np.max(np.abs(Ts - ex)) > se


@pytest.mark.parametrize("r", [2, 3, 4])
def test_identity_lambda_zero_limit_half_t_moments(r):
    """Lambda = I, a = 0: every point has weight 2^-r, so T is exact; the moments
    are those of |t_m| components: E|V| = 2 sqrt(m) G((m+1)/2) / (sqrt(pi)(m-1) G(m/2)),
    E V^2 = m/(m-2), E V_t V_h = (2/pi) m/(m-2)."""
    m = 7.5
    T, EV, EVV = O.sov_pass(np.zeros((1, r)), np.eye(r), m, _U(1 << 14, r + 1, 1), True)
    assert T[0] == 2.0 ** -r
    ev = 2 * math.sqrt(m) * math.exp(special.gammaln((m + 1) / 2) - special.gammaln(m / 2)) / (
        math.sqrt(math.pi) * (m - 1))
    assert np.allclose(EV[0], ev, rtol=5e-4)
    assert np.allclose(np.diag(EVV[0]), m / (m - 2), rtol=1e-2)
    off = EVV[0][~np.eye(r, dtype=bool)]
    assert np.allclose(off, (2 / math.pi) * m / (m - 2), rtol=1e-2)


def test_general_limits_match_library_mvt_cdf_and_mc_moments():
    """T_3 at general limits vs scipy's multivariate t CDF; truncated moments vs MC."""
    Lam = np.array([[1.0, 0.3, -0.2], [0.3, 0.7, 0.1], [-0.2, 0.1, 1.3]])
    L = np.linalg.cholesky(Lam)
    m = 8.2
    x = np.array([0.4, -0.9, 1.1])
    T, EV, EVV = O.sov_pass(-x[None, :], L, m, _U(1 << 15, 4, 0), True)
    ref = stats.multivariate_t(loc=np.zeros(3), shape=Lam, df=m).cdf(x, maxpts=2_000_000,
                                                                     random_state=1)
    assert abs(T[0] - ref) < 3e-6
    rng = np.random.default_rng(5)
    M = 2_000_000
    V = rng.standard_normal((M, 3)) / np.sqrt(rng.chisquare(m, M) / m)[:, None]
    Vs = V[(V @ L.T > -x).all(axis=1)]
    se = Vs.std(axis=0) / math.sqrt(Vs.shape[0])
    assert np.all(np.abs(EV[0] - Vs.mean(axis=0)) < 5 * se + 1e-4)
    M2 = (Vs[:, :, None] * Vs[:, None, :])
    se2 = M2.std(axis=0) / math.sqrt(Vs.shape[0])
    assert np.all(np.abs(EVV[0] - M2.mean(axis=0)) < 5 * se2 + 1e-3)


def test_underflowing_point_keeps_zero_weight_and_finite_moments():
    """Where p_t underflows to 0 at some points they add nothing and the moments
    stay finite; where it underflows at every point T is exactly 0."""
    L = np.linalg.cholesky(np.array([[1.0, 0.99], [0.99, 1.0]]))
    U = _U(1024, 3, 0)
    s = O.chi_scale(U[:, 0], 5.0)
    T, EV, EVV = O.sov_pass(np.array([[-1.0, 8.0]]), L, 5.0, U, True)
    assert np.all(np.isfinite(EV)) and np.all(np.isfinite(EVV))
    assert T[0] > 0.0
    assert s.max() > 2.0    # 8 s / L_22 > 110 there: p_2 underflows to 0 at those points
    T0 = O.sov_pass(np.array([[-1.0, 60.0]]), L, 5.0, U, False)
    assert T0[0] == 0.0


# --------------------------------------------------------------------------- Delta = 0: t mixture

def test_delta_zero_reduces_to_t_density_and_exact_weights():
    rng = np.random.default_rng(3)
    p, r, nu = 3, 2, 5.5
    mu = np.array([0.5, -1.0, 2.0])
    A = rng.standard_normal((p, p))
    Sigma = A @ A.T + np.eye(p)
    Y = rng.standard_normal((40, p)) * 2 + mu
    U = _U(512, r + 1, 4)
    out = O.estep_component(Y, mu, Sigma, np.zeros((p, r)), nu, U)
    ref = stats.multivariate_t(loc=mu, shape=Sigma, df=nu).logpdf(Y)
    assert np.allclose(out["logf"], ref, rtol=1e-12, atol=1e-12)
    d = np.einsum("jp,pq,jq->j", Y - mu, np.linalg.inv(Sigma), Y - mu)
    assert np.allclose(out["e1"], (nu + p) / (nu + d), rtol=1e-13)
    e2_exact = special.digamma((nu + p) / 2) - np.log((nu + d) / 2)
    assert np.allclose(out["e2"], e2_exact, rtol=1e-12, atol=1e-12)
    # the lattice estimate of E[log W | y] agrees with the closed form to QMC error
    out1 = O.estep_component(Y, mu, Sigma, np.zeros((p, r)), nu, _U(1 << 14, r + 1, 4), e2_mode=1)
    assert np.allclose(out1["e2"], e2_exact, atol=5e-4)


# --------------------------------------------------------------------------- brute-force Monte Carlo

def _mc_posterior(y, mu, Sigma, Delta, nu, M, rng):
    """Sample (W, U) from the prior of Section 2's latent structure, weight by
    N_p(y; mu + Delta U, Sigma / W): self-normalised importance sampling."""
    p, r = Delta.shape
    W = rng.gamma(nu / 2, 2 / nu, size=M)
    Uu = np.abs(rng.standard_normal((M, r))) / np.sqrt(W)[:, None]
    Sinv = np.linalg.inv(Sigma)
    _, logdet = np.linalg.slogdet(Sigma)
    res = y[None, :] - mu[None, :] - Uu @ Delta.T
    quad = np.einsum("jp,pq,jq->j", res, Sinv, res)
    logw = 0.5 * p * np.log(W) - 0.5 * W * quad - 0.5 * p * math.log(2 * math.pi) - 0.5 * logdet
    wt = np.exp(logw)
    f = wt.mean()
    sw = wt.sum()

    def ratio(h):
        R = (wt[:, None] * h).sum(axis=0) / sw
        se = np.sqrt(((wt[:, None] * (h - R)) ** 2).sum(axis=0)) / sw
        return R, se
    e1 = ratio(W[:, None])
    e2 = ratio(np.log(W)[:, None])
    e3 = ratio(W[:, None] * Uu)
    e4 = ratio((W[:, None, None] * Uu[:, :, None] * Uu[:, None, :]).reshape(M, -1))
    fse = wt.std() / math.sqrt(M)
    return f, fse, e1, e2, e3, e4


@pytest.mark.parametrize("case", [0, 1])
def test_estep_matches_brute_force_monte_carlo(case):
    rng = np.random.default_rng(11 + case)
    p, r = 2, (2 if case == 0 else 1)
    mu = np.array([0.3, -0.4])
    Sigma = np.array([[1.0, 0.4], [0.4, 0.8]])
    Delta = np.array([[1.2, -0.5], [0.7, 1.5]])[:, :r]
    nu = 6.0
    Ys = np.array([[1.5, 1.0], [-0.5, 0.2], [2.5, 3.0]])
    U = _U(1 << 14, r + 1, 9)
    out = O.estep_component(Ys, mu, Sigma, Delta, nu, U, e2_mode=1)
    for j, y in enumerate(Ys):
        f, fse, e1, e2, e3, e4 = _mc_posterior(y, mu, Sigma, Delta, nu, 1_500_000, rng)
        assert abs(math.exp(out["logf"][j]) - f) < 5 * fse + 2e-4 * f
        assert abs(out["e1"][j] - e1[0][0]) < 5 * e1[1][0] + 1e-3
        assert abs(out["e2"][j] - e2[0][0]) < 5 * e2[1][0] + 2e-3
        assert np.all(np.abs(out["e3"][j] - e3[0]) < 5 * e3[1] + 2e-3)
        assert np.all(np.abs(out["e4"][j].ravel() - e4[0]) < 5 * e4[1] + 5e-3)


# --------------------------------------------------------------------------- normalisation

@pytest.mark.parametrize("r", [1, 2])
def test_density_integrates_to_one_p1(r):
    """int f(y) dy = 1 over y = mu + c tan(theta), Gauss-Legendre in theta."""
    mu, Sigma, nu = np.array([0.2]), np.array([[0.8]]), 4.5
    Delta = np.array([[1.3, -0.8][:r]])
    x, wq = np.polynomial.legendre.leggauss(600)
    th = 0.5 * math.pi * x * (1 - 1e-12)
    c = 2.0
    Y = (mu + c * np.tan(th))[:, None]
    jac = c / np.cos(th) ** 2 * 0.5 * math.pi
    out = O.estep_component(Y, mu, Sigma, Delta, nu, _U(1 << 14, r + 1, 2), density_only=True)
    total = np.sum(wq * jac * np.exp(out["logf"]))
    assert abs(total - 1.0) < 2e-5


def test_density_integrates_to_one_p2_r1():
    mu, nu = np.array([0.0, 0.5]), 6.0
    Sigma = np.array([[1.0, 0.3], [0.3, 0.6]])
    Delta = np.array([[1.1], [-0.7]])
    x, wq = np.polynomial.legendre.leggauss(140)
    th = 0.5 * math.pi * x * (1 - 1e-12)
    c = 2.0
    t1, t2 = np.meshgrid(th, th, indexing="ij")
    Y = np.stack([mu[0] + c * np.tan(t1).ravel(), mu[1] + c * np.tan(t2).ravel()], axis=1)
    jac = (c * 0.5 * math.pi) ** 2 / (np.cos(t1) ** 2 * np.cos(t2) ** 2)
    W = np.outer(wq, wq) * jac
    out = O.estep_component(Y, mu, Sigma, Delta, nu, _U(2048, 2, 2), density_only=True)
    total = np.sum(W.ravel() * np.exp(out["logf"]))
    assert abs(total - 1.0) < 2e-4


# --------------------------------------------------------------------------- tau, M-step, EM

def _small_problem(seed=0, n=300):
    Y, _, truth, init, lat, _ = synth.workload("cfust_p2r2g2_n2000_N1024", n=n, seed=seed)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    return Y, truth, init, U


def test_tau_rows_sum_to_one_and_loglik_is_sum_of_lse():
    Y, truth, init, U = _small_problem()
    E = O.estep(Y, init, U)
    assert np.allclose(E["tau"].sum(axis=0), 1.0, atol=1e-15)
    f = (init.pi[:, None] * np.exp(E["logf"])).sum(axis=0)
    assert math.isclose(E["loglik"], float(np.log(f).sum()), rel_tol=1e-13)


def test_mstep_updates_are_conditional_maximisers_of_q():
    """Finite-difference gradient of the expected complete-data log-likelihood,
    written per observation, vanishes at each conditional-maximisation step."""
    Y, truth, init, U = _small_problem(n=200)
    E = O.estep(Y, init, U)
    args = (Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"])
    sums = O.mstep_sums(*args)
    new = O.mstep_update(sums, init, Y.shape[0])
    assert math.isclose(new.pi.sum(), 1.0, rel_tol=1e-14)
    assert np.allclose(new.pi, E["tau"].sum(axis=1) / Y.shape[0])
    h = 1e-5
    for i in range(init.g):
        def bump(P, which, idx, dv):
            arr = getattr(P, which)
            arr[(i,) + idx] += dv
            if which == "Sigma":
                arr[(i,) + idx[::-1]] = arr[(i,) + idx]

        def grad(which, base, idx):
            P1, P2 = base.copy(), base.copy()
            bump(P1, which, idx, h)
            bump(P2, which, idx, -h)
            return (O.q_function(*args, P1, i) - O.q_function(*args, P2, i)) / (2 * h)

        def scale(which, base, idx):
            P = base.copy()
            bump(P, which, idx, 0.1)
            return abs(O.q_function(*args, P, i) - O.q_function(*args, base, i)) / 0.1
        # mu is maximised with Delta and Sigma at their old values
        b = init.copy(); b.mu[i] = new.mu[i]
        for k in range(init.p):
            assert abs(grad("mu", b, (k,))) < 1e-6 * (1 + scale("mu", b, (k,)))
        # Delta with the new mu
        b.Delta[i] = new.Delta[i]
        for k in range(init.p):
            for t in range(init.r):
                assert abs(grad("Delta", b, (k, t))) < 1e-6 * (1 + scale("Delta", b, (k, t)))
        # Sigma with the new mu and Delta
        b.Sigma[i] = new.Sigma[i]
        for k in range(init.p):
            for l in range(k + 1):
                assert abs(grad("Sigma", b, (k, l))) < 1e-6 * (1 + scale("Sigma", b, (k, l)))
        b.nu[i] = new.nu[i]
        assert abs(grad("nu", b, ())) < 1e-6 * (1 + scale("nu", b, ()))


def test_mstep_delta_zero_is_textbook_t_mixture_update():
    rng = np.random.default_rng(2)
    Y, _, _, init, lat, _ = synth.workload("cfust_p2r2g2_n2000_N1024", n=200)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    P = init.copy(); P.Delta[:] = 0.0
    E = O.estep(Y, P, U)
    new = O.mstep_update(O.mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]),
                         P, Y.shape[0], fix_delta=True)
    for i in range(P.g):
        w = E["tau"][i] * E["e1"][i]
        mu = (w[:, None] * Y).sum(0) / w.sum()
        dy = Y - mu
        Sig = (w[:, None, None] * dy[:, :, None] * dy[:, None, :]).sum(0) / E["tau"][i].sum()
        assert np.allclose(new.mu[i], mu, rtol=1e-12)
        assert np.allclose(new.Sigma[i], Sig, rtol=1e-11)
    del rng


def test_em_monotone_for_t_mixture():
    """With Delta held at 0 the E-step is exact, so EM never lowers l (Section 2)."""
    Y, truth, init, U = _small_problem(n=400)
    P = init.copy(); P.Delta[:] = 0.0
    _, trace = O.fit(Y, P, U, iters=8, fix_delta=True)
    assert np.all(np.diff(trace) >= -1e-12 * np.abs(trace[1:]))


def test_em_general_increases_likelihood():
    """For the full CFUST fit the lattice E-step makes EM approximate: l must
    rise overall and any step that lowers it must be tiny."""
    Y, truth, init, U = _small_problem(n=400)
    _, trace = O.fit(Y, init, U, iters=6)
    assert trace[-1] > trace[0]
    assert np.all(np.diff(trace) > -1e-6 * np.abs(trace[1:]))


# --------------------------------------------------------------------------- Algorithms 4 and 1

def test_aitken_exact_on_geometric_sequence():
    """Aitken's extrapolation is exact for l^k = L - c rho^k, so the test of
    Algorithm 4 fires at the first k with c rho^k < eps and not before."""
    Linf, c, rho, eps = -1234.5, 50.0, 0.6, 1e-3
    tr = [Linf - c * rho ** k for k in range(40)]
    stop, est = O.aitken_stop(tr[:5], eps)
    assert math.isclose(est, Linf, rel_tol=1e-12)
    assert not stop
    first = next(k for k in range(2, 40) if c * rho ** k < eps * 0.999)
    fired = next(k for k in range(2, 40) if O.aitken_stop(tr[:k + 1], eps)[0])
    assert fired == first


def test_select_start_largest_first_on_ties():
    assert O.select_start([-10.0, -3.0, -5.0, -3.0]) == 1


# --------------------------------------------------------------------------- skew-normal limit (nu = inf)

def _sn_case(rng, p, r):
    A = rng.standard_normal((p, p))
    Sigma = A @ A.T / p + 0.5 * np.eye(p)
    Delta = rng.uniform(-1.2, 1.2, (p, r))
    mu = rng.standard_normal(p)
    return mu, Sigma, Delta


def test_skew_normal_limit_r1_matches_the_closed_form():
    """nu = inf, r = 1: f(y) = 2 phi_p(y; mu, Omega) Phi(q / sqrt(Lambda)), the
    multivariate skew-normal density (Azzalini & Dalla Valle), exact on the
    lattice (with s = 1 every point has the same weight); U | y is N(q, Lambda)
    truncated to U > 0, whose moments scipy's truncnorm gives; W = 1."""
    rng = np.random.default_rng(11)
    p = 3
    mu, Sigma, Delta = _sn_case(rng, p, 1)
    Y = mu + rng.standard_normal((40, p)) * 1.5
    out = O.estep_component(Y, mu, Sigma, Delta, math.inf, _U(1 << 14, 2, 1))
    coarse = O.estep_component(Y, mu, Sigma, Delta, math.inf, _U(1024, 2, 1))
    Omega = Sigma + Delta @ Delta.T
    Oinv = np.linalg.inv(Omega)
    q = (Y - mu) @ Oinv @ Delta[:, 0]
    lam = 1.0 - Delta[:, 0] @ Oinv @ Delta[:, 0]
    ref = (math.log(2.0) + stats.multivariate_normal(mu, Omega).logpdf(Y)
           + stats.norm.logcdf(q / math.sqrt(lam)))
    assert np.allclose(out["logf"], ref, rtol=0, atol=1e-11)
    assert np.all(out["e1"] == 1.0) and np.all(out["e2"] == 0.0)
    sd = math.sqrt(lam)
    tn = stats.truncnorm(-q / sd, np.inf, loc=q, scale=sd)
    # the lattice moments converge (the draw -Phi^-1((1-u)p) is unbounded as
    # u -> 1, so slowly; the second moment more so): at 16384 points ten times
    # closer than at 1024, within 1e-5 (mean) and 5e-5 (second moment)
    for k, ex, tol in (("e3", tn.mean(), 1e-5), ("e4", tn.moment(2), 5e-5)):
        fine = np.abs(out[k].reshape(len(Y)) - ex).max()
        rough = np.abs(coarse[k].reshape(len(Y)) - ex).max()
        assert 10 * fine < rough and fine < tol * max(1.0, np.abs(ex).max()), (k, fine, rough)


def test_skew_normal_is_the_large_nu_limit():
    """nu = inf against nu = 1e8 (the law differs by O(1/sqrt(nu)) in the chi
    scale and O(1/nu) elsewhere): p = 3, r = 2, every output."""
    rng = np.random.default_rng(12)
    mu, Sigma, Delta = _sn_case(rng, 3, 2)
    Y = mu + rng.standard_normal((30, 3)) * 1.5
    U = _U(2048, 3, 4)
    a = O.estep_component(Y, mu, Sigma, Delta, math.inf, U)
    b = O.estep_component(Y, mu, Sigma, Delta, 1e8, U)
    assert np.allclose(a["logf"], b["logf"], rtol=0, atol=2e-3)
    for k in ("e1", "e3", "e4"):
        assert np.allclose(a[k], b[k], rtol=2e-3, atol=2e-3), k
    assert np.allclose(b["e2"], 0.0, atol=2e-3)


def test_skew_normal_density_integrates_to_one_p1():
    mu, Sigma, Delta = np.array([0.2]), np.array([[0.8]]), np.array([[1.3, -0.8]])
    x, wq = np.polynomial.legendre.leggauss(400)
    th = 0.5 * math.pi * x * (1 - 1e-12)
    c = 2.0
    Y = (mu + c * np.tan(th))[:, None]
    jac = c / np.cos(th) ** 2 * 0.5 * math.pi
    out = O.estep_component(Y, mu, Sigma, Delta, math.inf, _U(1 << 14, 3, 2), density_only=True)
    assert abs(np.sum(wq * jac * np.exp(out["logf"])) - 1.0) < 2e-5


def test_skew_normal_delta_zero_is_the_gaussian_mixture_update():
    """nu = inf and Delta = 0: the E-step is the Gaussian mixture's (e1 = 1) and
    the M-step the textbook weighted mean and covariance; nu stays inf."""
    Y, _, _, init, lat, _ = synth.workload("cfust_p2r2g2_n2000_N1024", n=200)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    P = init.copy()
    P.Delta[:] = 0.0
    P.nu[:] = math.inf
    E = O.estep(Y, P, U)
    for i in range(P.g):
        ref = stats.multivariate_normal(P.mu[i], P.Sigma[i]).logpdf(Y)
        assert np.allclose(E["logf"][i], ref + P.r * math.log(2.0) + P.r * math.log(0.5), atol=1e-12)
    new = O.mstep_update(O.mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]),
                         P, Y.shape[0], fix_delta=True)
    for i in range(P.g):
        t = E["tau"][i]
        mu = (t[:, None] * Y).sum(0) / t.sum()
        dy = Y - mu
        Sig = (t[:, None, None] * dy[:, :, None] * dy[:, None, :]).sum(0) / t.sum()
        assert np.allclose(new.mu[i], mu, rtol=1e-12)
        assert np.allclose(new.Sigma[i], Sig, rtol=1e-11)
        assert math.isinf(new.nu[i])


# --------------------------------------------------------------------------- variable prioritisation

def test_prioritised_order_rule():
    """Decreasing standardised limit a_t / sqrt(Lambda_tt); ties keep the lower index."""
    Lam = np.diag([1.0, 4.0, 1.0, 0.25])
    a = np.array([[0.5, 3.0, 2.0, -1.0],     # standardised 0.5, 1.5, 2.0, -2.0
                  [1.0, 2.0, 1.0, 0.5]])     # standardised 1.0, 1.0, 1.0, 1.0 (all tied)
    assert np.array_equal(O.prioritised_order(a, Lam), [[2, 1, 0, 3], [0, 1, 2, 3]])


def _prio_case(seed=21, n=60):
    rng = np.random.default_rng(seed)
    p, r = 3, 3
    A = rng.standard_normal((p, p))
    Sigma = A @ A.T / p + 0.3 * np.eye(p)
    Delta = rng.uniform(-1.5, 1.5, (p, r))
    mu = np.zeros(p)
    Y = rng.standard_normal((n, p)) * 2.5
    return Y, mu, Sigma, Delta, 6.5


def test_prioritised_rule_agrees_with_natural_order_at_high_n():
    """The reordering changes the integrand, not the integral: at 2^15 points
    both orders give the same T, e1..e4 (within their integration error), with
    non-identity permutations present, so a moment scattered back to the wrong
    coordinate fails."""
    Y, mu, Sigma, Delta, nu = _prio_case()
    U = _U(1 << 15, 4, 5)
    a = O.estep_component(Y, mu, Sigma, Delta, nu, U)
    b = O.estep_component(Y, mu, Sigma, Delta, nu, U, prioritise=True)
    d, q, Lam, _ = O.component_terms(Y, mu, Sigma, Delta, nu)
    perms = O.prioritised_order(-q, Lam)
    assert (perms != np.arange(3)).any(axis=1).mean() > 0.5
    # the natural order's own error grows in the tail (e4 off by ~1% at log f
    # = -13 here); a moment scattered to the wrong coordinate is off by O(1)
    ok = np.isfinite(a["logf"]) & (a["logf"] > -15)
    assert ok.sum() > 40
    assert np.allclose(a["logf"][ok], b["logf"][ok], rtol=0, atol=1e-3)
    for k in ("e1", "e3", "e4"):
        assert np.allclose(a[k][ok], b[k][ok], rtol=2e-2, atol=2e-2), k


def test_prioritised_rule_is_more_accurate_per_point():
    """Normal limit (nu = inf), r = 2, correlation 0.6, the restrictive limit
    second: P(X1 > a1, X2 > a2) = int_{a2}^inf phi(x) Phi((rho x - a1) /
    sqrt(1 - rho^2)) dx by quadrature.  At 1024 points the natural order
    misses tail probabilities by percents; the prioritised order takes the
    restrictive variable first (its probability exact, the conditional
    integrand nearly flat) and is exact to 1e-6 or better."""
    from scipy import integrate
    rho = 0.6
    Lam = np.array([[1.0, rho], [rho, 1.0]])
    sd = math.sqrt(1.0 - rho * rho)
    for a in (np.array([-1.0, 5.0]), np.array([0.5, 4.0]), np.array([1.0, 6.0])):
        ref = integrate.quad(lambda x: stats.norm.pdf(x) * stats.norm.cdf((rho * x - a[0]) / sd), a[1], np.inf,
                             epsabs=0, epsrel=1e-12)[0]
        errs = {}
        for prio in (False, True):
            perm = O.prioritised_order(a[None, :], Lam)[0] if prio else np.arange(2)
            assert list(perm) == ([1, 0] if prio else [0, 1])
            Lp = np.linalg.cholesky(Lam[np.ix_(perm, perm)])
            est = np.array([O.sov_pass(a[None, perm], Lp, math.inf, _U(1024, 3, s), False)[0] for s in range(4)])
            errs[prio] = float(np.max(np.abs(est - ref)) / ref)
        assert errs[True] < 1e-6 and errs[False] > 1e-2, (a, errs)


# --------------------------------------------------------------------------- pass B on pass A's points

@pytest.mark.parametrize("m", [5.0, 6.3, 12.5])
def test_shared_points_r1_match_univariate_t_closed_forms_at_dof_plus_two(m):
    """r = 1: pass B estimated on pass A's points (weight x/m_A) is the t law at
    dof m + 2 truncated at its own limit a_B = a_A sqrt((m+2)/m): scipy's t
    survival function and the closed-form truncated moments at dof m + 2."""
    aA = np.array([[-1.5], [-0.3], [0.0], [0.7], [1.6]])
    l = 0.8
    mB = m + 2.0
    cB = aA[:, 0] * math.sqrt(mB / m) / l
    S0, E1, E2 = _t_trunc_closed(cB, mB)
    U = _U(1 << 14, 2, 3)
    TA, _, TB, EV, EVV = O.sov_pass_shared(aA, np.array([[l]]), m, mB, U, O.chi_scale(U[:, 0], m))
    assert np.allclose(TA, stats.t.sf(aA[:, 0] / l, m), rtol=2e-5)
    assert np.allclose(TB, S0, rtol=2e-5)
    assert np.allclose(EV[:, 0], E1, rtol=2e-3)
    assert np.allclose(EVV[:, 0, 0], E2, rtol=1e-2)


def test_shared_points_agree_with_the_separate_pass_b_at_high_n():
    """r = 3, general Lambda: the two estimators of pass B (its own chi-square
    quantile at dof m + 2, or pass A's points with the density ratio x/m) are
    different rules for the same integrals, so at 65536 points they agree to
    the rules' error on pairs whose probability is not in the far tail."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((3, 3))
    Lam = A @ A.T / 3 + 0.6 * np.eye(3)
    dinv = 1 / np.sqrt(np.diag(Lam))
    Lam = Lam * dinv[:, None] * dinv[None, :]
    L = np.linalg.cholesky(Lam)
    m = 7.5
    aA = rng.uniform(-1.5, 0.8, (12, 3))
    aB = aA * math.sqrt((m + 2) / m)
    U = _U(1 << 16, 4, 2)
    TA, _, TB, EV, EVV = O.sov_pass_shared(aA, L, m, m + 2, U, O.chi_scale(U[:, 0], m))
    TB2, EV2, EVV2 = O.sov_pass(aB, L, m + 2, U, True)
    assert np.all(TB2 > 1e-2)
    assert np.allclose(TB, TB2, rtol=2e-4)
    assert np.allclose(EV, EV2, rtol=0, atol=2e-3)
    assert np.allclose(EVV, EVV2, rtol=0, atol=5e-3)
    # and pass A is the plain pass at dof m
    assert np.array_equal(TA, O.sov_pass(aA, L, m, U, False))


def test_shared_points_skew_normal_limit_is_the_separate_passes():
    """nu = inf: the chi scale is 1 and both passes take the limits -q, so the
    weight x/m is 1 and the shared estimate is the separate one bit for bit."""
    rng = np.random.default_rng(13)
    mu, Sigma, Delta = _sn_case(rng, 3, 2)
    Y = mu + rng.standard_normal((25, 3)) * 1.5
    U = _U(1024, 3, 4)
    a = O.estep_component(Y, mu, Sigma, Delta, math.inf, U)
    b = O.estep_component(Y, mu, Sigma, Delta, math.inf, U, shared=True)
    for k in ("logf", "e1", "e2", "e3", "e4"):
        assert np.array_equal(a[k], b[k]), k


def test_estep_shared_points_match_brute_force_monte_carlo():
    """The E-step with pass B on pass A's points against self-normalised
    importance sampling of Section 2's latent structure (as the natural rule)."""
    rng = np.random.default_rng(11)
    p, r = 2, 2
    mu = np.array([0.3, -0.4])
    Sigma = np.array([[1.0, 0.4], [0.4, 0.8]])
    Delta = np.array([[1.2, -0.5], [0.7, 1.5]])
    nu = 6.0
    Ys = np.array([[1.5, 1.0], [-0.5, 0.2], [2.5, 3.0]])
    U = _U(1 << 14, r + 1, 9)
    out = O.estep_component(Ys, mu, Sigma, Delta, nu, U, e2_mode=1, shared=True)
    for j, y in enumerate(Ys):
        f, fse, e1, e2, e3, e4 = _mc_posterior(y, mu, Sigma, Delta, nu, 1_500_000, rng)
        assert abs(math.exp(out["logf"][j]) - f) < 5 * fse + 2e-4 * f
        assert abs(out["e1"][j] - e1[0][0]) < 5 * e1[1][0] + 1e-3
        assert abs(out["e2"][j] - e2[0][0]) < 5 * e2[1][0] + 2e-3
        assert np.all(np.abs(out["e3"][j] - e3[0]) < 5 * e3[1] + 2e-3)
        assert np.all(np.abs(out["e4"][j].ravel() - e4[0]) < 5 * e4[1] + 5e-3)
