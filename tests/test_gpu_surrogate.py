"""The learned surrogate of the r = 3 lattice integrals, through the C ABI:
its GPU labeller against the FP64 lattice rule, its BF16 tensor-core forward
pass and gradient against the FP64 network oracle, training on the GPU, the
network judged by the lattice rule, and the surrogate E-step against the
plain lattice E-step."""
import math

import numpy as np
import pytest
from scipy import special

from oracle import cfust_oracle as O
from oracle import mlp_oracle as MO
from paper_2005_06848_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _domain_sample(rng, B):
    out = []
    while len(out) < B:
        x = np.r_[rng.uniform(MO.C_LO, MO.C_HI, 3), rng.uniform(-MO.RHO_MAX, MO.RHO_MAX, 3),
                  rng.uniform(MO.LOGM_LO, MO.LOGM_HI)]
        if MO.in_domain(x[None])[0]:
            out.append(x)
    return np.array(out)


@pytest.fixture(scope="module")
def lat8192():
    return synth.make_lattice(8192, 4, seed=11)


def test_labeller_matches_the_fp64_lattice_rule(lat8192):
    torch = _torch()
    rng = np.random.default_rng(5)
    x = _domain_sample(rng, 40).astype(np.float32).astype(np.float64)
    # plus the box corners in c, where the weights are smallest
    x[:4, :3] = [[MO.C_HI] * 3, [MO.C_LO] * 3, [MO.C_HI, MO.C_LO, MO.C_HI], [0.0, 0.0, 0.0]]
    s = binding.Surrogate(lat8192, seed=1)
    yg = s.cfust_surrogate_label(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    U = O.lattice_points(lat8192.n, lat8192.z, lat8192.shift)
    yo = MO.label(x, U)
    ok = np.isfinite(yo[:, 0])
    assert np.all(np.isfinite(yg[ok]))
    # single-precision sweep with chi tables interpolated in log m
    assert np.max(np.abs(yg[ok, 0] - yo[ok, 0])) < 5e-4
    assert np.max(np.abs(yg[ok, 1:] - yo[ok, 1:]) / (1 + np.abs(yo[ok, 1:]))) < 5e-4


def _bf16(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def test_forward_matches_the_fp64_network_within_bf16_bounds(lat8192):
    torch = _torch()
    rng = np.random.default_rng(6)
    s = binding.Surrogate(lat8192, seed=2)
    th, _ = s.cfust_surrogate_get_params()
    norm = np.r_[rng.normal(size=10), rng.uniform(0.5, 3, 10)].astype(np.float32)
    s.cfust_surrogate_set_params(th, norm)
    x = _domain_sample(rng, 700).astype(np.float32)
    pg = s.cfust_surrogate_predict(torch.tensor(x, dtype=torch.float32, device="cuda")).cpu().numpy()
    # the network oracle at BF16-rounded weights: what remains is the BF16
    # rounding of inputs and activations (relative 2^-9 per value)
    tb = th.astype(np.float64).copy()
    for (W, _b) in MO.unpack(tb):
        W[...] = _bf16(W)
    out, _ = MO.forward(tb, MO.normalise_inputs(x))
    on = MO.net_targets(pg, norm)  # back to the network's normalised outputs
    err = np.abs(on - out)
    assert err.max() < 1e-2 and np.sqrt((err ** 2).mean()) < 2e-3, (err.max(), np.sqrt((err ** 2).mean()))


def test_gradient_matches_the_fp64_network_oracle(lat8192):
    torch = _torch()
    rng = np.random.default_rng(7)
    s = binding.Surrogate(lat8192, seed=3)
    th, _ = s.cfust_surrogate_get_params()
    norm = np.r_[rng.normal(size=10), rng.uniform(0.5, 3, 10)].astype(np.float32)
    s.cfust_surrogate_set_params(th, norm)
    x = _domain_sample(rng, 3000).astype(np.float32)   # several row tiles and a ragged tail
    y = rng.normal(size=(3000, 10)).astype(np.float32)
    loss, g = s.cfust_surrogate_gradient(torch.tensor(x, device="cuda"), torch.tensor(y, device="cuda"))
    lo, go = MO.loss_and_grad(th.astype(np.float64), MO.normalise_inputs(x), MO.net_targets(y, norm))
    assert abs(loss - lo) < 2e-3 * lo
    assert np.linalg.norm(g - go) < 2e-2 * np.linalg.norm(go)
    # every layer's weight and bias block on its own
    off = 0
    for k in range(4):
        a, b = MO.DIMS[k], MO.DIMS[k + 1]
        for size in (a * b, b):
            blk = slice(off, off + size)
            assert np.linalg.norm(g[blk] - go[blk]) < 3e-2 * np.linalg.norm(go[blk]) + 1e-7, (k, size)
            off += size


def test_training_on_the_gpu_reduces_the_loss(lat8192):
    torch = _torch()
    s = binding.Surrogate(lat8192, seed=4)
    trace = s.cfust_surrogate_train(1 << 19, 4, batch=4096, lr=3e-3, seed=5)
    assert np.all(np.isfinite(trace)) and trace[-1] < 0.2 * trace[0], trace
    # judged by the lattice rule on held-out problems, in the network's units
    rng = np.random.default_rng(8)
    x = torch.tensor(_domain_sample(rng, 2048), dtype=torch.float32, device="cuda")
    y = s.cfust_surrogate_label(x).cpu().numpy()
    p = s.cfust_surrogate_predict(x).cpu().numpy()
    _, norm = s.cfust_surrogate_get_params()
    ok = np.all(np.isfinite(y), axis=1)
    e = MO.net_targets(p[ok], norm) - MO.net_targets(y[ok], norm)
    # predicting the training mean scores about 1 in these units
    assert np.sqrt(np.mean(e ** 2)) < 0.3


def _standardised(Y, params, i):
    """Per pair of component i: d, q, log t_p, D^{1/2}, the network inputs of
    passes A and B, and whether the pair is the network's (box rule)."""
    pi, mu, Sigma, Delta, nu = params.as_arrays()
    p = Y.shape[1]
    d, q, Lam, log_tp = O.component_terms(Y, mu[i], Sigma[i], Delta[i], nu[i])
    sD = np.sqrt(np.diag(Lam))
    R = Lam / np.outer(sD, sD)
    mA, mB = nu[i] + p, nu[i] + p + 2
    cA = -q * np.sqrt(mA / (nu[i] + d))[:, None] / sD
    cB = -q * np.sqrt(mB / (nu[i] + d))[:, None] / sD
    rr = np.tile([R[0, 1], R[0, 2], R[1, 2]], (len(d), 1))
    xA = np.column_stack([np.clip(cA, MO.C_LO, MO.C_HI), rr, np.full(len(d), math.log(mA))])
    xB = np.column_stack([np.clip(cB, MO.C_LO, MO.C_HI), rr, np.full(len(d), math.log(mB))])
    lo = -np.inf if mA >= 8 else MO.C_LO
    comp_ok = bool(MO.in_domain(np.r_[np.zeros(3), rr[0], math.log(mA)][None])[0] and mB <= 30)
    inside = comp_ok & np.all((cB >= lo) & (cB <= MO.C_HI), axis=1)
    # pairs within rounding of an edge may fall either way in single precision
    edge = np.any(np.isclose(cB, MO.C_HI, atol=1e-4) | np.isclose(cB, MO.C_LO, atol=1e-4), axis=1)
    return d, q, log_tp, sD, xA, xB, inside, edge


def _psd_repair(v, floor=1e-6, rho=0.999):
    """The E-step's repair of a predicted covariance (upper order 00 01 02 11
    12 22), in double: diagonal floored, first-row correlations clamped to
    |rho|, the last LDL^T factor shrunk so every pivot keeps 1 - rho^2 of its
    variance, diagonal kept."""
    v = np.asarray(v, dtype=np.float64)
    d0, d1, d2 = (np.maximum(v[:, k], floor) for k in (0, 3, 5))
    m01, m02 = rho * np.sqrt(d0 * d1), rho * np.sqrt(d0 * d2)
    c01 = np.clip(v[:, 1], -m01, m01)
    c02 = np.clip(v[:, 2], -m02, m02)
    l10, l20 = c01 / d0, c02 / d0
    p1 = d1 - l10 * c01
    lmax = np.sqrt(np.maximum(rho * rho * d2 - l20 * c02, 0.0) / p1)
    l21 = np.clip((v[:, 4] - l20 * c01) / p1, -lmax, lmax)
    return np.column_stack([d0, c01, c02, d1, l20 * c01 + l21 * p1, d2])


# Largest error of the BF16 tensor-core network in its normalised output units
# against the FP64 network at the same BF16 inputs and weights: the bar of
# test_forward_matches_the_fp64_network_within_bf16_bounds (BF16 rounding of
# the activations, 2^-9 relative per value, through three hidden layers).
NET_DELTA = 1e-2


def _pair_values(oA, oB, norm, d, q, nu, p, sD):
    """From the two normalised network output rows of pairs: log T_A, log T_B,
    and pass B's conditional moments in the form the E-step scales by e1,
    c3 = e3 / e1 and c4 = e4 / e1 (lower triangle, 6), by the oracle's
    formulas in FP64 (pass B's covariance made positive semi-definite as the
    E-step does)."""
    tA = MO.from_net(oA, norm)
    tB = MO.from_net(oB, norm)
    cov = _psd_repair(MO.net_targets(tB)[:, 4:])
    EX = tB[:, 1:4]
    S = np.zeros((len(d), 3, 3))
    for k, (a, b) in enumerate(MO.UPPER):
        S[:, a, b] = S[:, b, a] = cov[:, k] + EX[:, a] * EX[:, b]
    LEV = sD * EX
    LEVVL = S * np.outer(sD, sD)[None]
    # probabilities chosen so that the oracle's e1 is exactly 1: its e3, e4 are then c3, c4
    TB = np.ones_like(d) if math.isinf(nu) else (nu + d) / (nu + p)
    _, _, c3, c4 = O.expectations(d, q, nu, p, np.ones_like(d), TB, LEV, LEVVL)
    low = np.stack([c4[:, t, h] for t in range(3) for h in range(t + 1)], axis=1)
    return tA[:, 0], tB[:, 0], c3, low


def test_surrogate_estep_is_the_expectations_of_the_network_outputs(lat8192):
    """Every pair the network serves, element by element: the surrogate
    E-step's log f and e1..e4 against the oracle's E-step formulas (FP64)
    applied to the FP64 network oracle at BF16-rounded weights, evaluated on
    exactly the BF16 inputs the kernel gave the tensor cores
    (cfust_surrogate_inputs, the same device function).

    The outputs are compared in the form in which the network's error enters
    linearly: log f, log e1 (= log((nu+p)/(nu+d)) + log T_B - log T_A),
    e2 - e1 (no network term), e3 / e1 and e4 / e1 (pass B's conditional
    moments); e1..e4 follow from these exactly.  Each network output is within
    NET_DELTA of the FP64 network's in its normalised units, so
    log T = -exp(o_0 s_0 + m_0) is within |log T| (exp(s_0 NET_DELTA) - 1)
    exactly, and c3, c4 within their first-order sensitivity to pass B's nine
    moment outputs times NET_DELTA (central differences) plus the quadratic
    term of E[X] E[X]^T; single-precision slack on top (2e-4 + 2e-6 |value|
    for logarithms, 5e-5 (1 + |value|) for the moments).  The inputs
    themselves match the FP64 standardisation within BF16 rounding.  Pairs
    outside the domain: bit-identical to the lattice E-step."""
    torch = _torch()
    s = binding.Surrogate(lat8192, seed=6)
    s.cfust_surrogate_train(1 << 18, 2, batch=4096, lr=3e-3, seed=2)
    theta, norm = s.cfust_surrogate_get_params()
    tb = theta.astype(np.float64).copy()
    for (W, _b) in MO.unpack(tb):
        W[...] = _bf16(W)
    norm = norm.astype(np.float64)
    s0 = norm[10]
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=3000, seed=0)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    lat = synth.make_lattice(1024, 4, seed=0)
    p = Y.shape[1]
    checked = 0
    for P in (truth, init):
        plain = binding.Context(lat, precision=binding.CFUST_FP32)
        sur = binding.Context(lat, precision=binding.CFUST_FP32)
        sur.cfust_set_surrogate(s)
        Ep = plain.cfust_estep(Yd, P)
        Es = sur.cfust_estep(Yd, P)
        fb = sur.cfust_last_fallback()
        X, kind = sur.cfust_surrogate_inputs(Yd, P)
        X = X.cpu().numpy().astype(np.float64)
        kind = kind.cpu().numpy()
        assert fb == int(np.sum(kind != 2))
        for i in range(P.g):
            nu = float(P.nu[i])
            mA = nu + p
            d, q, log_tp, sD, xA, xB, inside, edge = _standardised(Y, P, i)
            m = kind[i] == 2
            # the kernel's inputs are the FP64 standardisation up to BF16 rounding
            for x64, xk in ((xA, X[i, :, 0]), (xB, X[i, :, 1])):
                u64 = MO.normalise_inputs(x64[m])
                assert np.all(np.abs(xk[m] - u64) <= 2.0 ** -8 * np.abs(u64) + 1e-5), i
            oA, _ = MO.forward(tb, X[i, m, 0])
            oB, _ = MO.forward(tb, X[i, m, 1])
            args = (norm, d[m], q[m], nu, p, sD)
            lTA, lTB, c3, c4 = _pair_values(oA, oB, *args)
            # first-order sensitivity of c3, c4 to pass B's moment outputs
            s3 = np.zeros_like(c3)
            s4 = np.zeros_like(c4)
            h = 1e-4
            for k in range(1, 10):
                dB = np.zeros_like(oB)
                dB[:, k] = h
                _, _, c3p, c4p = _pair_values(oA, oB + dB, *args)
                _, _, c3m, c4m = _pair_values(oA, oB - dB, *args)
                s3 += np.abs(c3p - c3m) / (2 * h) * NET_DELTA
                s4 += np.abs(c4p - c4m) / (2 * h) * NET_DELTA
            # second-order term of E[X] E[X]^T: |dEX_t dEX_h| sigma^2 D_t D_h
            sig2 = (nu + d[m]) / (nu + p + 2.0)
            quad = np.outer(sig2, [sD[t] * sD[hh] * norm[11 + t] * norm[11 + hh] * NET_DELTA ** 2
                                   for t in range(3) for hh in range(t + 1)])
            growth = math.expm1(s0 * NET_DELTA)
            g_logf = Es["logf"][i].cpu().numpy()[m].astype(np.float64)
            g_e1 = Es["e1"][i].cpu().numpy()[m].astype(np.float64)
            g_e2 = Es["e2"][i].cpu().numpy()[m].astype(np.float64)
            g_e3 = Es["e3"][i].cpu().numpy().T[m].astype(np.float64)
            g_e4 = Es["e4"][i].cpu().numpy().T[m].astype(np.float64)
            nz = g_e1 > 0
            logf_ref = 3 * math.log(2) + log_tp[m] + lTA
            le1_ref = math.log(mA) - np.log(nu + d[m]) + lTB - lTA
            e2m_ref = -(np.log(0.5 * (nu + d[m])) + mA / (nu + d[m]) - special.digamma(0.5 * mA))
            checks = [
                ("log f", g_logf, logf_ref, np.abs(lTA) * growth + 2e-4 + 2e-6 * np.abs(logf_ref)),
                ("log e1", np.log(np.where(nz, g_e1, 1.0)), np.where(nz, le1_ref, 0.0),
                 np.where(nz, (np.abs(lTA) + np.abs(lTB)) * growth + 2e-4 + 2e-6 * np.abs(le1_ref), 0.0)),
                ("e2 - e1", g_e2 - g_e1, e2m_ref, 5e-5 * (1 + np.abs(e2m_ref))),
                ("e3 / e1", g_e3[nz] / g_e1[nz, None], c3[nz], 1.1 * s3[nz] + 5e-5 * (1 + np.abs(c3[nz]))),
                ("e4 / e1", g_e4[nz] / g_e1[nz, None], c4[nz],
                 1.1 * (s4[nz] + quad[nz]) + 5e-5 * (1 + np.abs(c4[nz]))),
            ]
            for name, got, ref, bound in checks:
                err = np.abs(got - ref)
                if err.size:
                    w = np.unravel_index(np.argmax(err / np.maximum(bound, 1e-300)), err.shape)
                    assert np.all(err <= bound), (i, name, w, err[w], bound[w], got[w], ref[w])
            # e1 underflows to 0 in float only where log e1 is far below the float range
            assert np.all(le1_ref[~nz] < -80.0), (i, le1_ref[~nz].max() if (~nz).any() else None)
            checked += int(m.sum())
            # the rest went to the lattice rule: the same numbers as without a surrogate
            out = ~m
            for k in ("logf", "e1", "e2", "e3", "e4"):
                a = Es[k][i].cpu().numpy()
                b = Ep[k][i].cpu().numpy()
                assert np.array_equal(a[..., out], b[..., out]), (i, k)
        # tau from the same log f: rows sum to one
        assert np.allclose(Es["tau"].sum(0).cpu().numpy(), 1.0, atol=1e-5)
    assert checked > 5000, checked


def _timed_loglik(torch, ctx, Yd, P, reps=5):
    ctx.cfust_loglik(Yd, P)
    st = torch.cuda.current_stream()
    best, ll = float("inf"), None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        ll = ctx.cfust_loglik(Yd, P)
        e1.record(st)
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return ll, best


@pytest.fixture(scope="module")
def trained(lat8192):
    """The network as the bench trains it: 20 M lattice-labelled problems, 100 epochs."""
    _torch()
    s = binding.Surrogate(lat8192, seed=3)
    s.cfust_surrogate_train(20_000_000, 100, batch=16384, lr=3e-3, seed=7)
    return s


def test_surrogate_gain_at_equal_loglik_accuracy(trained):
    """The trained network against the method without it: on the p=3, r=3,
    g=4, n=10^6 mixture, the log-likelihood error of the surrogate E-step (judge:
    the plain lattice rule at 2^16 points) is matched by the cheapest plain
    lattice that is at least as accurate (RMS over three lattice shifts), and at
    that accuracy the surrogate E-step takes less device time."""
    torch = _torch()
    s = trained
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", seed=0)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    ladder = [32, 64, 128, 256, 512, 1024, 2048]
    report = []
    for P in (init, truth):
        judge = binding.Context(synth.make_lattice(1 << 16, 4, seed=0), precision=binding.CFUST_FP32)
        l_judge = judge.cfust_loglik(Yd, P)
        sur = binding.Context(synth.make_lattice(128, 4, seed=0), precision=binding.CFUST_FP32)
        sur.cfust_set_surrogate(s)
        l_sur, t_sur = _timed_loglik(torch, sur, Yd, P)
        e_sur = abs(l_sur - l_judge)
        rms, t_plain = {}, {}
        for N in ladder:
            errs = []
            for sd in range(3):
                c = binding.Context(synth.make_lattice(N, 4, seed=sd), precision=binding.CFUST_FP32)
                l, t = _timed_loglik(torch, c, Yd, P, reps=3 if sd == 0 else 1)
                errs.append(l - l_judge)
                if sd == 0:
                    t_plain[N] = t
            rms[N] = float(np.sqrt(np.mean(np.square(errs))))
        ok_n = [N for N in ladder if rms[N] <= e_sur]
        n_eq = min(ok_n) if ok_n else max(ladder)
        report.append((e_sur, n_eq, t_sur, t_plain[n_eq], rms))
        assert math.isfinite(l_sur)
        assert t_sur < t_plain[n_eq], report
    print("surrogate gain report", report)


def test_triage_margin_bounds_the_loglik_change(trained):
    """A triage margin of 12 nats instead of 30: every listed pair the lattice
    sweep then skips has tau_ij < exp(-12) by a proven upper bound of its
    density, so l moves by at most (listed pairs) x exp(-12)."""
    torch = _torch()
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=200_000, seed=0)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    lat = synth.make_lattice(128, 4, seed=0)
    ls, listed = {}, {}
    for T in (30.0, 12.0):
        with binding.Context(lat, precision=binding.CFUST_FP32, triage_nats=T) as c:
            c.cfust_set_surrogate(trained)
            ls[T] = c.cfust_loglik(Yd, init)
            listed[T] = c.cfust_last_fallback()
    assert listed[30.0] == listed[12.0] > 0
    assert abs(ls[12.0] - ls[30.0]) <= listed[12.0] * math.exp(-12.0), (ls, listed)


def test_surrogate_edge_cases(lat8192):
    """Attachment rules: FP64 contexts and r != 3 are refused when the E-step
    runs; a mixture whose dof leave the network's domain (nu + p + 2 > 30)
    sends every pair to the lattice rule and reproduces the plain E-step
    bit for bit; detaching restores the plain path."""
    torch = _torch()
    s = binding.Surrogate(lat8192, seed=9)
    Y, _, truth, _, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=700, seed=1)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    lat = synth.make_lattice(256, 4, seed=0)
    c64 = binding.Context(lat, precision=binding.CFUST_FP64)
    c64.cfust_set_surrogate(s)
    with pytest.raises(binding.CfustError) as ei:
        c64.cfust_loglik(Yd, truth)
    assert ei.value.status == -1
    # r = 2 mixture on a 3-dimensional lattice context
    Y2, _, t2, _, lat2, _ = synth.workload("cfust_p2r2g2_n2000_N1024", n=300, seed=0)
    c2 = binding.Context(lat2, precision=binding.CFUST_FP32)
    c2.cfust_set_surrogate(s)
    with pytest.raises(binding.CfustError):
        c2.cfust_loglik(torch.tensor(Y2, dtype=torch.float64, device="cuda"), t2)
    # dof outside the domain: all pairs to the lattice rule
    pi, mu, Sigma, Delta, nu = truth.as_arrays()
    high = synth.Params(pi, mu, Sigma, Delta, np.full_like(nu, 40.0))
    plain = binding.Context(lat, precision=binding.CFUST_FP32)
    sur = binding.Context(lat, precision=binding.CFUST_FP32)
    sur.cfust_set_surrogate(s)
    Ep, Es = plain.cfust_estep(Yd, high), sur.cfust_estep(Yd, high)
    assert sur.cfust_last_fallback() == high.g * len(Y)
    for k in ("logf", "tau", "e1", "e2", "e3", "e4"):
        assert torch.equal(Ep[k], Es[k]), k
    assert Ep["loglik"] == Es["loglik"]
    # detach: the plain path again
    sur.cfust_set_surrogate(None)
    assert sur.cfust_loglik(Yd, truth) == plain.cfust_loglik(Yd, truth)
    assert sur.cfust_last_fallback() == 0


def test_problems_and_finetune(lat8192):
    """cfust_surrogate_problems returns the network inputs of exactly the pairs
    the surrogate E-step keeps (two rows each, inside the domain box), and
    fine-tuning on them lowers the network's error on those problems."""
    torch = _torch()
    s = binding.Surrogate(lat8192, seed=12)
    s.cfust_surrogate_train(1 << 19, 3, batch=4096, lr=3e-3, seed=4)
    Y, _, truth, _, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=6000, seed=2)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    ctx = binding.Context(synth.make_lattice(256, 4, seed=0), precision=binding.CFUST_FP32)
    x = ctx.cfust_surrogate_problems(Yd, truth)
    ctx.cfust_set_surrogate(s)
    ctx.cfust_estep(Yd, truth)
    kept = truth.g * len(Y) - ctx.cfust_last_fallback()
    assert x.shape[0] == 2 * kept
    xn = x.cpu().numpy().astype(np.float64)
    assert np.all(xn[:, :3] >= MO.C_LO - 1e-6) and np.all(xn[:, :3] <= MO.C_HI + 1e-6)
    assert np.all(np.abs(xn[:, 3:6]) <= MO.RHO_MAX + 1e-6)
    assert np.all((xn[:, 6] >= MO.LOGM_LO - 1e-5) & (xn[:, 6] <= MO.LOGM_HI + 1e-5))
    # every other row: a stride of 3 keeps a third of the pairs
    x3 = ctx.cfust_surrogate_problems(Yd, truth, stride=3)
    assert abs(x3.shape[0] - x.shape[0] / 3) <= 0.05 * x.shape[0] / 3 + 4

    def err():
        y = s.cfust_surrogate_label(x).cpu().numpy()
        p = s.cfust_surrogate_predict(x).cpu().numpy()
        _, norm = s.cfust_surrogate_get_params()
        ok = np.all(np.isfinite(y), axis=1)
        return float(np.sqrt(np.mean((MO.net_targets(p[ok], norm) - MO.net_targets(y[ok], norm)) ** 2)))
    before = err()
    trace = s.cfust_surrogate_finetune(x, 4, batch=1024, lr=1e-3, seed=5)
    assert np.all(np.isfinite(trace))
    assert err() < 0.8 * before


def test_em_with_the_surrogate_improves_the_likelihood(trained):
    """Ten EM iterations with the network in the E-step (graph-captured fit)
    from the perturbed start: the log-likelihood of the result, judged by the
    plain lattice rule at 2^16 points, rises well above the start's, and ends
    within 0.5% of a plain 1024-point fit's after the same ten iterations."""
    torch = _torch()
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=200000, seed=3)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    judge = binding.Context(synth.make_lattice(1 << 16, 4, seed=0), precision=binding.CFUST_FP32)
    sur = binding.Context(synth.make_lattice(128, 4, seed=0), precision=binding.CFUST_FP32, max_iter=10)
    sur.cfust_set_surrogate(trained)
    Ps, trace_s, _ = sur.cfust_fit(Yd, init)
    plain = binding.Context(synth.make_lattice(1024, 4, seed=0), precision=binding.CFUST_FP32, max_iter=10)
    Pp, trace_p, _ = plain.cfust_fit(Yd, init)
    l0 = judge.cfust_loglik(Yd, init)
    ls, lp = judge.cfust_loglik(Yd, Ps), judge.cfust_loglik(Yd, Pp)
    assert np.all(np.isfinite(trace_s))
    assert ls - l0 > 0.5 * (lp - l0), (l0, ls, lp)
    assert abs(ls - lp) < 5e-3 * abs(lp), (ls, lp)


def test_prioritised_fallback_pairs_equal_the_prioritised_lattice_estep(lat8192):
    """With variable prioritisation and a surrogate attached, the pairs the
    network leaves to the lattice rule are integrated in the prioritised
    order: bit-identical to the plain prioritised E-step's."""
    torch = _torch()
    s = binding.Surrogate(lat8192, seed=6)
    s.cfust_surrogate_train(1 << 16, 1, batch=4096, lr=3e-3, seed=2)
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=2000, seed=0)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    lat = synth.make_lattice(512, 4, seed=0)
    with binding.Context(lat, precision=binding.CFUST_FP32, prioritise=True) as plain, \
            binding.Context(lat, precision=binding.CFUST_FP32, prioritise=True) as sur:
        sur.cfust_set_surrogate(s)
        Ep = plain.cfust_estep(Yd, init)
        Es = sur.cfust_estep(Yd, init)
        _, kind = sur.cfust_surrogate_inputs(Yd, init)
    out = kind.cpu().numpy() != 2
    assert out.sum() > 100
    for k in ("logf", "e1", "e2", "e3", "e4"):
        a = Es[k].cpu().numpy()
        b = Ep[k].cpu().numpy()
        for i in range(init.g):
            assert np.array_equal(a[i][..., out[i]], b[i][..., out[i]]), (i, k)
