"""Plain FP64 CPU oracle for the CFUST-mixture EM hot path.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline / reference legs of ``bench.py`` may import this module.  The
product path (the CUDA library and its Python binding) never touches it, and
it shares no code with that path: the two meet only through the seeded inputs
of ``paper_2005_06848_gb300.synth``, which hold none of the arithmetic here.

What it computes, and where each step comes from:

* Mixture density, log-likelihood and posterior memberships: Eq. 1, Eq. 3 and
  Eq. 4 (Section 2).
* The CFUST component density: Eq. 2, with Omega = Sigma + Delta Delta^T,
  Lambda = I - Delta^T Omega^{-1} Delta and d(y) the Mahalanobis distance.
* The E-step conditional expectations e1 = E[W | y], e2 = E[log W | y],
  e3 = E[W U | y], e4 = E[W U U^T | y] of the latent gamma W and latent
  truncated normal U that Section 2 introduces.  The paper defers their
  formulas to its references; they are derived here from that latent
  structure (W ~ Gamma(nu/2, nu/2), U | W ~ N_r(0, I/W) truncated to the
  positive orthant, Y | U, W ~ N_p(mu + Delta U, Sigma/W)):
      W | y  is proportional to Gamma(w; (nu+p)/2, (nu+d)/2) Phi_r(sqrt(w) q; 0, Lambda),
      U | y, w ~ N_r(q, Lambda/w) truncated to R_+^r,  q = Delta^T Omega^{-1}(y - mu).
  This gives
      f(y) = 2^r t_p(y; mu, Omega, nu) T_A,
      e1 = (nu+p)/(nu+d) * T_B / T_A,
      e3 = e1 * E[X | X > 0],  e4 = e1 * E[X X^T | X > 0],
  where T_A = P(L V > a_A), V ~ t_r(0, I, nu+p), a_A = -q sqrt((nu+p)/(nu+d));
  T_B = P(L V > a_B), V ~ t_r(0, I, nu+p+2), a_B = -q sqrt((nu+p+2)/(nu+d));
  L = chol(Lambda) and X = q + sigma L V with sigma = sqrt((nu+d)/(nu+p+2)).
* The r-variate t probabilities and truncated moments: Genz's separation of
  variables over a shifted rank-1 (Korobov) lattice with the baker's
  transform; the t law is handled as a normal divided by an independent
  chi scale, coordinate 0 of the lattice drawing the chi-square quantile.
* Opt-in (``shared``): pass B estimated on pass A's lattice points.  The
  chi-square densities satisfy chi2_{m+2}(x) = chi2_m(x) x / m, so pass B's
  integrals are pass A's integrand weighted by x / (nu+p) at pass A's points
  (sov_pass_shared): the same T_B and truncated moments, half the normal
  evaluations of two separate passes.
* The M-step: the paper's Algorithm 3 updates each component from the
  E-step's partial sums (Section 3.2's "eight partial sums").  The eight sums
  and the conditional-maximisation updates are derived by maximising the
  expected complete-data log-likelihood in the order pi, mu, Delta, Sigma, nu.
* The stopping rule of Algorithm 4 (Aitken acceleration) and the multi-start
  selection of Algorithm 1.
* The skew-normal limit (the paper's Section 2 notes the CFUST family's
  limiting cases): a component with nu = +inf is the canonical fundamental
  skew normal law, W = 1: t_p becomes the normal density phi_p, the chi scale
  is 1, a_A = a_B = -q, e1 = 1, e2 = 0, and the nu update keeps nu = inf.

Readings of the paper (its typos and silences) are listed in the module-level
docstrings of the functions that use them.  Parity is pinned against closed
forms, exact identities and brute-force Monte Carlo in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize, special

LOG2 = math.log(2.0)
TINY64 = np.finfo(np.float64).tiny          # smallest positive normal double
U_MIN = 2.0 ** -53                          # clamp of the baker-transformed lattice

# ----------------------------------------------------------------------------
# Lattice rule (the integration points of the E-step's r-variate integrals)
# ----------------------------------------------------------------------------


def lattice_points(n_points: int, z, shift) -> np.ndarray:
    """Points of the shifted rank-1 lattice after the baker's transform.

    u_k = frac(((k z) mod N)/N + shift), then u <- 1 - |2u - 1|, clamped to
    [2^-53, 1 - 2^-53] so that neither quantile below sees 0 or 1.
    Returns [N, dim] float64.
    """
    z = np.asarray(z, dtype=np.int64)
    shift = np.asarray(shift, dtype=np.float64)
    k = np.arange(n_points, dtype=np.int64)[:, None]
    idx = (k * z[None, :]) % n_points
    u = idx / n_points + shift[None, :]
    u = u - np.floor(u)
    u = 1.0 - np.abs(2.0 * u - 1.0)
    return np.clip(u, U_MIN, 1.0 - U_MIN)


def chi_scale(u0: np.ndarray, m: float) -> np.ndarray:
    """s = sqrt(F^{-1}_{chi^2_m}(u0) / m): the scale that turns N(0,1) into t_m.

    The chi-square quantile is 2 * P^{-1}(m/2, u0) with P the regularised lower
    incomplete gamma function; the upper-tail inverse is used for u0 >= 1/2.
    """
    u0 = np.asarray(u0, dtype=np.float64)
    if math.isinf(m):
        return np.ones_like(u0)         # chi^2_m / m -> 1: the normal law
    a = 0.5 * m
    lo = special.gammaincinv(a, np.where(u0 < 0.5, u0, 0.25))
    hi = special.gammainccinv(a, np.where(u0 < 0.5, 0.75, 1.0 - u0))
    x = np.where(u0 < 0.5, lo, hi)
    return np.sqrt(2.0 * x / m)


def _sov_chain(a, L, U, s):
    """Point weights w [P, N] and conditional draws z [P, N, r] of the
    separation-of-variables chain (the loop of sov_pass, below)."""
    P, r = a.shape
    N = U.shape[0]
    zs = np.zeros((P, N, r))
    w = np.ones((P, N))
    for t in range(r):
        cond = np.einsum("h,pnh->pn", L[t, :t], zs[:, :, :t]) if t > 0 else 0.0
        lim = (a[:, t, None] * s[None, :] - cond) / L[t, t]
        pt = special.ndtr(-lim)
        w = w * pt
        arg = np.maximum((1.0 - U[None, :, t + 1]) * pt, TINY64)
        zs[:, :, t] = -special.ndtri(arg)
    return w, zs


def sov_pass(a: np.ndarray, L: np.ndarray, m: float, U: np.ndarray,
             moments: bool, logchi: bool = False, s: np.ndarray | None = None):
    """Genz separation-of-variables estimate of P(L V > a), V ~ t_r(0, I, m).

    For each lattice point (s from coordinate 0, uniforms u_1..u_r):
        lim_t = (a_t s - sum_{h<t} L_th z_h) / L_tt
        p_t   = Phi(-lim_t)
        z_t   = -Phi^{-1}((1 - u_t) p_t)      (a draw of Z_t given Z_t > lim_t)
    weight w = prod_t p_t and V = z / s.  Then P = mean(w), and the truncated
    moments are the weighted means E[V] = sum w V / sum w, E[V V^T] likewise.
    Reading: no variable reordering, so that both implementations see the same
    integrand; the quantile argument is floored at the smallest normal double
    so a point whose p_t underflows to 0 keeps a finite z and weight 0.

    a: [P, r] limits; L: [r, r] lower Cholesky factor; U: [N, r+1] points;
    ``s`` optionally the precomputed chi_scale(U[:, 0], m).
    Returns T [P]; with ``moments`` also EV [P, r], EVV [P, r, r]; with
    ``logchi`` also E[log chi^2_m] under the weights [P].
    """
    N = U.shape[0]
    if s is None:
        s = chi_scale(U[:, 0], m)                            # [N]
    w, zs = _sov_chain(a, L, U, s)
    T = w.sum(axis=1) / N
    out = [T]
    if moments:
        v = zs / s[None, :, None]
        W = w.sum(axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            EV = np.einsum("pn,pnr->pr", w, v) / W[:, None]
            EVV = np.einsum("pn,pnr,pns->prs", w, v, v) / W[:, None, None]
        out += [EV, EVV]
    if logchi:
        W = w.sum(axis=1)
        with np.errstate(invalid="ignore", divide="ignore"):
            out.append((w @ np.log(m * s * s)) / W)
    return tuple(out) if len(out) > 1 else T


def _chunks(n, size):
    for j0 in range(0, n, size):
        yield slice(j0, min(n, j0 + size))


# ----------------------------------------------------------------------------
# Component density (Eq. 2) and E-step quantities
# ----------------------------------------------------------------------------


def component_terms(Y, mu, Sigma, Delta, nu):
    """Per-observation pieces of Eq. 2 for one component.

    Omega = Sigma + Delta Delta^T, d = (y-mu)^T Omega^{-1} (y-mu),
    q = Delta^T Omega^{-1} (y-mu), Lambda = I - Delta^T Omega^{-1} Delta,
    log t_p(y; mu, Omega, nu).  Reading: the lowercase delta of Eq. 2 is Delta.
    """
    n, p = Y.shape
    r = Delta.shape[1]
    Omega = Sigma + Delta @ Delta.T
    Oinv = np.linalg.inv(Omega)
    sign, logdet = np.linalg.slogdet(Omega)
    if sign <= 0:
        raise np.linalg.LinAlgError("Omega not positive definite")
    Lam = np.eye(r) - Delta.T @ Oinv @ Delta
    Lam = 0.5 * (Lam + Lam.T)
    dy = Y - mu[None, :]
    d = np.einsum("jp,pq,jq->j", dy, Oinv, dy)
    q = dy @ Oinv @ Delta                                    # [n, r]
    if math.isinf(nu):
        # the limit of t_p: the normal density phi_p(y; mu, Omega)
        log_tp = -0.5 * p * math.log(2.0 * math.pi) - 0.5 * logdet - 0.5 * d
    else:
        log_tp = (special.gammaln(0.5 * (nu + p)) - special.gammaln(0.5 * nu)
                  - 0.5 * p * math.log(nu * math.pi) - 0.5 * logdet
                  - 0.5 * (nu + p) * np.log1p(d / nu))
    return d, q, Lam, log_tp


def prioritised_order(a, Lam):
    """Genz's variable prioritisation, in this library's reading: the r
    variables of a pair are integrated in decreasing order of their
    standardised limit a_t / sqrt(Lambda_tt), i.e. the smallest marginal
    probability P(X_t > a_t) first (the most restrictive limit outermost);
    ties keep the lower index.  a: [P, r].  Returns [P, r] permutations."""
    c = a / np.sqrt(np.diag(Lam))[None, :]
    return np.argsort(-c, axis=1, kind="stable")


def sov_pass_shared(aA, L, mA, mB, U, sA, logchi=False):
    """Pass A and pass B from one set of lattice points (``shared`` reading).

    Pass B's law differs from pass A's only in the chi variable: V = Z / s with
    s^2 = x / m and x ~ chi^2_{m_B} instead of chi^2_{m_A}, m_B = m_A + 2.  The
    chi-square densities satisfy chi2_{m+2}(x) = chi2_m(x) x / m, and pass B's
    scaled limit a_B sqrt(x / m_B) = -q sqrt(x / (nu + d)) is pass A's
    a_A sqrt(x / m_A) at the same x.  So pass B is pass A's integrand at pass
    A's points (x = m_A s_A^2 from lattice coordinate 0) with the extra weight
    x / m_A = s_A^2 and V = z / s_B, s_B = sqrt(x / m_B) = s_A sqrt(m_A / m_B):
        T_B = mean(w s_A^2),
        E[V] = sum w s_A^2 V / sum w s_A^2,  E[V V^T] likewise,
    the same integrals as sov_pass at dof m_B, estimated on pass A's draws.  In
    the skew-normal limit (m_A = m_B = inf, s_A = 1) the weight is 1 and V = z.
    Returns T_A, E[log chi^2_{m_A}] (with ``logchi``, else None), T_B, E[V], E[V V^T].
    """
    N = U.shape[0]
    w, zs = _sov_chain(aA, L, U, sA)
    TA = w.sum(axis=1) / N
    el = None
    if logchi:
        with np.errstate(invalid="ignore", divide="ignore"):
            el = (w @ np.log(mA * sA * sA)) / w.sum(axis=1)
    ratio = 1.0 if math.isinf(mA) else math.sqrt(mA / mB)
    wb = w * (sA * sA)[None, :]
    v = zs / (sA * ratio)[None, :, None]
    W = wb.sum(axis=1)
    TB = W / N
    with np.errstate(invalid="ignore", divide="ignore"):
        EV = np.einsum("pn,pnr->pr", wb, v) / W[:, None]
        EVV = np.einsum("pn,pnr,pns->prs", wb, v, v) / W[:, None, None]
    return TA, el, TB, EV, EVV


def _passes(aA, aB, L, Lam, mA, mB, U, sA, sB, logchi, density_only, prioritise, shared=False):
    """Pass A (T_A, optionally E[log chi^2]) and pass B (T_B, L E[V], L E[V V^T] L^T)
    of the pairs of one chunk, in natural or prioritised variable order; the
    moments come back in the natural order of X = L V.  With ``shared`` pass B
    is estimated on pass A's lattice points (sov_pass_shared)."""
    P, r = aA.shape
    perms = prioritised_order(aA, Lam) if (prioritise and r > 1) else np.tile(np.arange(r), (P, 1))
    TA = np.empty(P); EL = np.empty(P) if logchi else None
    TB = np.empty(P); LEV = np.empty((P, r)); LEVVL = np.empty((P, r, r))
    for perm in np.unique(perms, axis=0):
        idx = np.nonzero((perms == perm).all(axis=1))[0]
        Lp = L if np.array_equal(perm, np.arange(r)) else np.linalg.cholesky(Lam[np.ix_(perm, perm)])
        if shared and not density_only:
            ta, el, tb, EV, EVV = sov_pass_shared(aA[idx][:, perm], Lp, mA, mB, U, sA, logchi)
            TA[idx] = ta
            if logchi:
                EL[idx] = el
        else:
            if logchi:
                TA[idx], EL[idx] = sov_pass(aA[idx][:, perm], Lp, mA, U, moments=False, logchi=True, s=sA)
            else:
                TA[idx] = sov_pass(aA[idx][:, perm], Lp, mA, U, moments=False, s=sA)
            if density_only:
                continue
            tb, EV, EVV = sov_pass(aB[idx][:, perm], Lp, mB, U, moments=True, s=sB)
        TB[idx] = tb
        # X_perm = Lp V: scatter its moments back to the natural coordinates
        lev = EV @ Lp.T
        levvl = np.einsum("th,jhk,sk->jts", Lp, EVV, Lp)
        LEV[np.ix_(idx, perm)] = lev
        LEVVL[np.ix_(idx, perm, perm)] = levvl
    return TA, EL, TB, LEV, LEVVL


def estep_component(Y, mu, Sigma, Delta, nu, U, e2_mode=0, density_only=False,
                    chunk=None, prioritise=False, shared=False):
    """log f_i(y_j) and e1..e4 for every observation j of one component i.

    Returns dict with logf [n], and unless ``density_only``: e1 [n], e2 [n],
    e3 [n, r], e4 [n, r, r].  e2_mode 0 uses the usual CFUST-EM approximation
    e2 = e1 - log((nu+d)/2) - (nu+p)/(nu+d) + psi((nu+p)/2) (exact at Delta = 0);
    e2_mode 1 uses the lattice estimate E[log chi^2_{nu+p}] - log(nu+d) from
    the density pass.  Reading: where T_A or T_B underflows (is 0 or below the
    smallest normal double, where its subnormal value keeps too few bits for
    the pair's outputs to be determined), log f is -inf (T_A) and e1..e4 are
    set to 0, their weight tau being 0.  ``prioritise``
    integrates each pair's variables in the order of ``prioritised_order``
    (pass B's limits are a positive multiple of pass A's: the same order).
    ``shared`` estimates pass B on pass A's lattice points (sov_pass_shared).
    """
    n, p = Y.shape
    r = Delta.shape[1]
    d, q, Lam, log_tp = component_terms(Y, mu, Sigma, Delta, nu)
    L = np.linalg.cholesky(Lam)
    N = U.shape[0]
    if chunk is None:
        chunk = max(1, (1 << 21) // (N * max(r, 1)))
    logf = np.empty(n)
    out = dict(logf=logf)
    if not density_only:
        e1 = np.empty(n); e2 = np.empty(n); e3 = np.empty((n, r)); e4 = np.empty((n, r, r))
        out.update(e1=e1, e2=e2, e3=e3, e4=e4)
    mA = nu + p
    mB = nu + p + 2.0
    sA = chi_scale(U[:, 0], mA)
    sB = chi_scale(U[:, 0], mB)
    for sl in _chunks(n, chunk):
        dd = d[sl]; qq = q[sl]
        aA = -qq * _dof_ratio(mA, nu, dd)[:, None]
        aB = -qq * _dof_ratio(mB, nu, dd)[:, None]
        logchi = (e2_mode == 1 and not density_only)
        TA, elogchi, TB, LEV, LEVVL = _passes(aA, aB, L, Lam, mA, mB, U, sA, sB, logchi, density_only,
                                              prioritise, shared)
        with np.errstate(divide="ignore"):
            # a probability below the smallest normal double counts as
            # underflowed (reading: subnormal values carry too few bits to
            # take part in the rule), so log f = -inf there
            logf[sl] = r * LOG2 + log_tp[sl] + np.log(np.where(TA >= TINY64, TA, 0.0))
        if density_only:
            continue
        c1, c2, c3, c4 = expectations(dd, qq, nu, p, TA, TB, LEV, LEVVL, e2_mode,
                                      elogchi if e2_mode == 1 else None)
        e1[sl], e2[sl], e3[sl], e4[sl] = c1, c2, c3, c4
    return out


def _dof_ratio(m, nu, d):
    """sqrt(m / (nu + d)), and its limit 1 at nu = inf."""
    if math.isinf(nu):
        return np.ones_like(d)
    return np.sqrt(m / (nu + d))


def expectations(d, q, nu, p, TA, TB, LEV, LEVVL, e2_mode=0, elogchi=None):
    """e1..e4 of the pairs of one component from the two passes' results.

    d [P], q [P, r]: the pair's Mahalanobis distance and skew projection;
    TA, TB [P]: the pass-A and pass-B probabilities; LEV [P, r] = L E[V] and
    LEVVL [P, r, r] = L E[V V^T] L^T of pass B (X = L V truncated at X > a_B).
    e1 = (nu+p)/(nu+d) T_B/T_A, sigma = sqrt((nu+d)/(nu+p+2)),
    e3 = e1 (q + sigma L E[V]),
    e4 = e1 (q q^T + sigma (q (L E[V])^T + L E[V] q^T) + sigma^2 L E[V V^T] L^T),
    e2 as in estep_component.  Pairs with T_A or T_B underflowed (below the
    smallest normal double) get zeros.
    """
    mA = nu + p
    mB = nu + p + 2.0
    # underflow: T_A or T_B below the smallest normal double (see estep_component)
    ok = (TA >= TINY64) & (TB >= TINY64)
    with np.errstate(invalid="ignore", divide="ignore"):
        if math.isinf(nu):
            # W = 1: both passes integrate the same normal law
            c1 = TB / TA
            sig = np.ones_like(d)
        else:
            c1 = (mA / (nu + d)) * TB / TA
            sig = np.sqrt((nu + d) / mB)
        EX = q + sig[:, None] * LEV
        EXX = (q[:, :, None] * q[:, None, :]
               + sig[:, None, None] * (q[:, :, None] * LEV[:, None, :]
                                       + LEV[:, :, None] * q[:, None, :])
               + (sig * sig)[:, None, None] * LEVVL)
        if math.isinf(nu):
            c2 = np.zeros_like(d)        # E[log W | y] = log 1
        elif e2_mode == 1:
            c2 = elogchi - np.log(nu + d)
        else:
            c2 = (c1 - np.log(0.5 * (nu + d)) - mA / (nu + d)
                  + special.digamma(0.5 * mA))
    return (np.where(ok, c1, 0.0), np.where(ok, c2, 0.0),
            np.where(ok[:, None], c1[:, None] * EX, 0.0),
            np.where(ok[:, None, None], c1[:, None, None] * EXX, 0.0))


def posterior(logf: np.ndarray, pi: np.ndarray):
    """tau_ij = pi_i f_ij / sum_h pi_h f_hj (Eq. 4) and l = sum_j log f_j (Eq. 3).

    Reading: the sum over components in Algorithms 1 and 2, printed with upper
    limit n, runs over i = 1..g.  Uses a max-shifted log-sum-exp.
    Returns (tau [g, n], loglik, per-observation log f_j [n]).
    """
    a = np.log(pi)[:, None] + logf
    amax = a.max(axis=0)
    lse = amax + np.log(np.exp(a - amax[None, :]).sum(axis=0))
    tau = np.exp(a - lse[None, :])
    return tau, float(lse.sum()), lse


def estep(Y, params, lattice_U, e2_mode=0, prioritise=False, shared=False):
    """E-step of Section 2 for all (i, j): log f_ij, tau_ij, e1..e4 and l(Psi).

    ``params`` has arrays pi[g], mu[g,p], Sigma[g,p,p], Delta[g,p,r], nu[g].
    Returns dict(logf[g,n], tau[g,n], e1[g,n], e2[g,n], e3[g,n,r],
    e4[g,n,r,r], loglik).
    """
    g = params.pi.shape[0]
    comps = [estep_component(Y, params.mu[i], params.Sigma[i], params.Delta[i],
                             params.nu[i], lattice_U, e2_mode=e2_mode, prioritise=prioritise,
                             shared=shared)
             for i in range(g)]
    out = {k: np.stack([c[k] for c in comps]) for k in comps[0]}
    tau, ll, _ = posterior(out["logf"], params.pi)
    out["tau"] = tau
    out["loglik"] = ll
    return out


def loglik(Y, params, lattice_U, prioritise=False):
    """l(Psi) = sum_j log sum_i pi_i f_i(y_j) (Eq. 1, Eq. 3): density pass only."""
    g = params.pi.shape[0]
    logf = np.stack([estep_component(Y, params.mu[i], params.Sigma[i], params.Delta[i],
                                     params.nu[i], lattice_U, density_only=True,
                                     prioritise=prioritise)["logf"]
                     for i in range(g)])
    return posterior(logf, params.pi)[1]


# ----------------------------------------------------------------------------
# M-step (Algorithm 3) from the partial sums of Algorithm 2
# ----------------------------------------------------------------------------


def mstep_sums(Y, tau, e1, e2, e3, e4):
    """The eight per-component sums over observations (Section 3.2, Algorithm 2).

    S1 = sum tau, S2 = sum tau e1, S3 = sum tau e1 y, S4 = sum tau e3,
    S5 = sum tau y e3^T, S6 = sum tau e4, S7 = sum tau e1 y y^T,
    S8 = sum tau (e2 - e1).  Arrays as returned by ``estep``.
    """
    g = tau.shape[0]
    sums = []
    for i in range(g):
        t = tau[i]
        te1 = t * e1[i]
        sums.append(dict(
            S1=t.sum(),
            S2=te1.sum(),
            S3=te1 @ Y,
            S4=t @ e3[i],
            S5=Y.T @ (t[:, None] * e3[i]),
            S6=np.einsum("j,jts->ts", t, e4[i]),
            S7=Y.T @ (te1[:, None] * Y),
            S8=(t * (e2[i] - e1[i])).sum(),
        ))
    return sums


def nu_equation(nu, s8_over_s1):
    """Stationarity condition for nu: log(nu/2) - psi(nu/2) + 1 + S8/S1."""
    return math.log(0.5 * nu) - special.digamma(0.5 * nu) + 1.0 + s8_over_s1


def solve_nu(s8_over_s1, nu_min=1.0, nu_max=200.0):
    """Root of ``nu_equation`` in [nu_min, nu_max]; the bound where no sign change.

    The left side decreases in nu, so a positive value at nu_max means the
    root lies beyond it and a negative value at nu_min means below it.
    """
    f_lo = nu_equation(nu_min, s8_over_s1)
    f_hi = nu_equation(nu_max, s8_over_s1)
    if f_hi >= 0.0:
        return nu_max
    if f_lo <= 0.0:
        return nu_min
    return optimize.brentq(nu_equation, nu_min, nu_max, args=(s8_over_s1,),
                           xtol=1e-14, rtol=4 * np.finfo(float).eps, maxiter=500)


def mstep_update(sums, params, n, nu_min=1.0, nu_max=200.0, fix_delta=False):
    """Conditional-maximisation updates of Algorithm 3, one component at a time.

    1. pi_i = S1 / n
    2. mu_i = (S3 - Delta_old S4) / S2
    3. Delta_i = (S5 - mu_i S4^T) S6^{-1}
    4. Sigma_i = [S7 - S3 mu^T - mu S3^T + S2 mu mu^T - C Delta^T - Delta C^T
                  + Delta S6 Delta^T] / S1,   C = S5 - mu S4^T
    5. nu_i solves log(nu/2) - psi(nu/2) + 1 + S8/S1 = 0
    ``fix_delta`` keeps Delta (used to reduce the model to a t mixture).
    """
    new = params.copy()
    for i, S in enumerate(sums):
        new.pi[i] = S["S1"] / n
        mu = (S["S3"] - params.Delta[i] @ S["S4"]) / S["S2"]
        C = S["S5"] - np.outer(mu, S["S4"])
        Delta = params.Delta[i] if fix_delta else np.linalg.solve(S["S6"].T, C.T).T
        Sig = (S["S7"] - np.outer(S["S3"], mu) - np.outer(mu, S["S3"])
               + S["S2"] * np.outer(mu, mu) - C @ Delta.T - Delta @ C.T
               + Delta @ S["S6"] @ Delta.T) / S["S1"]
        new.mu[i] = mu
        new.Delta[i] = Delta
        new.Sigma[i] = 0.5 * (Sig + Sig.T)
        # nu = inf (the skew-normal limit) is a model choice, not updated
        new.nu[i] = math.inf if math.isinf(params.nu[i]) else solve_nu(S["S8"] / S["S1"], nu_min, nu_max)
    return new


def q_function(Y, tau, e1, e2, e3, e4, params, i):
    """Expected complete-data log-likelihood terms of component i that depend
    on (mu, Delta, Sigma, nu), with the E-step quantities held fixed.

    sum_j tau_ij [ -1/2 log|Sigma| - 1/2 tr(Sigma^{-1} E[W (y-mu-Delta U)(.)^T])
                   + (nu/2) log(nu/2) - log Gamma(nu/2) + (nu/2 - 1) e2 - (nu/2) e1 ]
    Written per observation (no sums S1..S8), as an independent check of the
    M-step updates.
    """
    mu, Sig, Dl, nu = params.mu[i], params.Sigma[i], params.Delta[i], params.nu[i]
    Sinv = np.linalg.inv(Sig)
    _, logdet = np.linalg.slogdet(Sig)
    dy = Y - mu[None, :]
    t = tau[i]
    quad = (e1[i] * np.einsum("jp,pq,jq->j", dy, Sinv, dy)
            - 2.0 * np.einsum("jp,pq,qr,jr->j", dy, Sinv, Dl, e3[i])
            + np.einsum("pq,qr,jrs,ps->j", Sinv, Dl, e4[i], Dl))
    qn = (0.5 * nu * math.log(0.5 * nu) - special.gammaln(0.5 * nu)
          + (0.5 * nu - 1.0) * e2[i] - 0.5 * nu * e1[i])
    return float(np.sum(t * (-0.5 * logdet - 0.5 * quad + qn)))


def fit(Y, params0, lattice_U, iters, e2_mode=0, nu_min=1.0, nu_max=200.0,
        fix_delta=False, shared=False):
    """EM (Section 2 outline; Algorithms 2 and 3) for a fixed number of iterations.

    The E-step at Psi^(k) also yields l(Psi^(k)) (Algorithm 2 computes the
    log-likelihood from the same densities), so the trace holds
    l(Psi^(0)) .. l(Psi^(iters)), the last from one density-only pass.
    Returns (params, trace[iters + 1]).
    """
    n = Y.shape[0]
    params = params0.copy()
    trace = []
    for _ in range(iters):
        E = estep(Y, params, lattice_U, e2_mode, shared=shared)
        trace.append(E["loglik"])
        sums = mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"])
        params = mstep_update(sums, params, n, nu_min, nu_max, fix_delta)
    trace.append(loglik(Y, params, lattice_U))
    return params, np.array(trace)


# ----------------------------------------------------------------------------
# Algorithm 4 (stopping) and Algorithm 1 (start selection)
# ----------------------------------------------------------------------------


def aitken_stop(trace, eps):
    """Aitken-accelerated stopping test of Algorithm 4 on l^(k-2), l^(k-1), l^(k).

    Reading: the printed asymptote has a typo (l^(k) - l^(k) over 1 + a); the
    standard Aitken form is used: a = (l^k - l^(k-1)) / (l^(k-1) - l^(k-2)),
    l_inf = l^(k-1) + (l^k - l^(k-1)) / (1 - a); stop when |l_inf - l^k| < eps.
    Returns (stop, l_inf).  Needs at least three values.
    """
    if len(trace) < 3:
        return False, float("nan")
    l2, l1, l0 = trace[-3], trace[-2], trace[-1]
    den = l1 - l2
    if den == 0.0:
        return True, l0
    a = (l0 - l1) / den
    if a == 1.0:
        return False, float("inf")
    linf = l1 + (l0 - l1) / (1.0 - a)
    return abs(linf - l0) < eps, linf


def select_start(loglik0):
    """Index of the start with the LARGEST l^(0) (Algorithm 1).

    Reading: the paper prints 'smallest'; maximum likelihood needs the largest.
    Ties go to the lowest index.
    """
    vals = np.asarray(loglik0, dtype=np.float64)
    return int(np.argmax(vals))
