"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Same seeded inputs and the same lattice on both sides.  Tolerances:
FP64 mode: log f_ij and l(Psi) to 1e-10 relative (|a - b| <= 1e-10 max(1, |b|)),
tau and e1..e4 to 1e-9; FP32 mode: log f_ij to 1e-4 absolute, tau to 1e-5,
l(Psi) to 1e-6 relative, parameters after 50 EM iterations to 1e-3 relative.
"""
import json
import os

import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import binding, synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

HERE = os.path.dirname(os.path.abspath(__file__))


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _problem(workload, n, N, seed=0):
    Y, labels, truth, init, _, meta = synth.workload(workload, n=n, seed=seed)
    lat = synth.make_lattice(N, meta["r"] + 1, seed)
    return Y, truth, init, lat


def _gpu_estep(Y, params, lat, precision, e2_mode=0, prioritise=False):
    torch = _torch()
    with binding.Context(lat, precision=precision, e2_mode=e2_mode, prioritise=prioritise) as ctx:
        Yd = torch.from_numpy(Y).cuda()
        out = ctx.cfust_estep(Yd, params)
        res = {k: (v.double().cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
        res["rescued"] = ctx.cfust_last_rescued()
    return res


def _oracle_estep(Y, params, lat, e2_mode=0, prioritise=False):
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    return O.estep(Y, params, U, e2_mode, prioritise=prioritise)


def _cmp(name, got, ref, rtol, atol=0.0):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    both_inf = np.isinf(got) & np.isinf(ref) & (np.sign(got) == np.sign(ref))
    err = np.where(both_inf, 0.0, np.abs(got - ref))
    tol = atol + rtol * np.maximum(1.0, np.abs(np.where(both_inf, 0.0, ref)))
    worst = float(np.max(err / tol)) if err.size else 0.0
    assert np.all(err <= tol), f"{name}: worst error / tolerance = {worst:.3g}, max abs err {err.max():.3g}"
    return float(err.max()) if err.size else 0.0


def _compare_estep(G, R, r, fp64):
    g, n = R["logf"].shape
    e4_ref = np.stack([R["e4"][:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1)
    e3_ref = np.transpose(R["e3"], (0, 2, 1))
    if fp64:
        _cmp("logf", G["logf"], R["logf"], 1e-10)
        _cmp("tau", G["tau"], R["tau"], 0, 1e-11)
        for k in ("e1", "e2"):
            _cmp(k, G[k], R[k], 1e-9)
        _cmp("e3", G["e3"], e3_ref, 1e-9)
        _cmp("e4", G["e4"], e4_ref, 1e-9)
        assert abs(G["loglik"] - R["loglik"]) <= 1e-10 * abs(R["loglik"])
    else:
        _cmp("logf", G["logf"], R["logf"], 0, 1e-4)
        _cmp("tau", G["tau"], R["tau"], 0, 1e-5)
        for k in ("e1", "e2"):
            _cmp(k, G[k], R[k], 2e-4)
        _cmp("e3", G["e3"], e3_ref, 2e-4)
        _cmp("e4", G["e4"], e4_ref, 2e-4)
        assert abs(G["loglik"] - R["loglik"]) <= 1e-6 * abs(R["loglik"])


CASES = [
    # (workload, n, lattice points)
    ("cfust_p2r2g2_n2000_N1024", 200, 1024),
    ("cfust_p4r4g3_n100000_N4096", 333, 1024),
    ("cfust_p3r3g4_n1000000_N2048", 150, 2048),
    ("cfust_p8r4g6_n1000000_N8192", 70, 1024),
]


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", CASES, ids=[c[0].split("_n")[0] for c in CASES])
def test_estep_matches_oracle(case, precision):
    wl, n, N = case
    Y, truth, init, lat = _problem(wl, n, N)
    R = _oracle_estep(Y, init, lat)
    G = _gpu_estep(Y, init, lat, precision)
    _compare_estep(G, R, init.r, precision == binding.CFUST_FP64)
    assert np.allclose(G["tau"].sum(axis=0), 1.0, atol=1e-12 if precision == 0 else 1e-5)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_estep_lattice_e2_mode(precision):
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 90, 1024)
    R = _oracle_estep(Y, init, lat, e2_mode=1)
    G = _gpu_estep(Y, init, lat, precision, e2_mode=1)
    _compare_estep(G, R, init.r, precision == binding.CFUST_FP64)


def _edge_params(rng, g, p, r, spread=3.0):
    P = synth.random_params(rng, g, p, r, spread ** 2, 2, 1.5, 3.0, 12.0)
    return P


@pytest.mark.parametrize("g,p,r,n,N", [
    (1, 1, 1, 1, 32),        # a single pair, the smallest lattice
    (1, 1, 1, 37, 64),       # fewer observations than one CTA tile, ragged
    (2, 16, 6, 40, 256),     # the largest p and r the library takes
    (3, 5, 2, 129, 96),      # lattice size not a power of two
    (5, 3, 3, 64, 128),      # exactly one tile
])
def test_estep_edge_shapes_fp64(g, p, r, n, N):
    rng = np.random.default_rng(100 + g * 7 + p)
    P = _edge_params(rng, g, p, r)
    Y, _ = synth.sample_cfust(P, n, rng)
    lat = synth.make_lattice(N, r + 1, 5)
    R = _oracle_estep(Y, P, lat)
    G = _gpu_estep(Y, P, lat, binding.CFUST_FP64)
    _compare_estep(G, R, r, True)


def test_estep_full_size_sampled_fp32():
    """The p=4, r=4, g=3, n=100000, N=4096 workload in the bench's launch
    configuration; the oracle recomputes 48 sampled observations (all three
    components each) and every E-step output is held to the single-precision
    bars: log f, tau, e1, e2, e3 and e4."""
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", None, 4096)
    G = _gpu_estep(Y, init, lat, binding.CFUST_FP32)
    idx = np.sort(np.random.default_rng(7).choice(Y.shape[0], 48, replace=False))
    R = _oracle_estep(Y[idx], init, lat)
    sub = {k: (v[:, idx] if k in ("logf", "tau", "e1", "e2") else v[..., idx]) for k, v in G.items()
           if k not in ("loglik", "rescued")}
    r = init.r
    _cmp("logf", sub["logf"], R["logf"], 0, 1e-4)
    _cmp("tau", sub["tau"], R["tau"], 0, 1e-5)
    for k in ("e1", "e2"):
        _cmp(k, sub[k], R[k], 2e-4)
    _cmp("e3", sub["e3"], np.transpose(R["e3"], (0, 2, 1)), 2e-4)
    _cmp("e4", sub["e4"], np.stack([R["e4"][:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1), 2e-4)
    assert np.allclose(G["tau"].sum(axis=0), 1.0, atol=1e-5)
    assert np.all(np.isfinite(G["logf"]))


def test_estep_full_size_sampled_fp32_largest_workload():
    """The largest workload (p=8, r=4, g=6, n=10^6, 8192-point lattice) in
    single precision through the same launch path as the bench; the oracle
    recomputes 16 sampled observations (all six components each) and every
    E-step output is held to the single-precision bars."""
    Y, truth, init, lat = _problem("cfust_p8r4g6_n1000000_N8192", None, 8192)
    G = _gpu_estep(Y, init, lat, binding.CFUST_FP32)
    assert np.allclose(G["tau"].sum(axis=0), 1.0, atol=1e-5)
    assert np.all(np.isfinite(G["logf"]) | (G["logf"] == -np.inf))
    idx = np.sort(np.random.default_rng(11).choice(Y.shape[0], 16, replace=False))
    R = _oracle_estep(Y[idx], init, lat)
    sub = {k: (v[:, idx] if k in ("logf", "tau", "e1", "e2") else v[..., idx]) for k, v in G.items()
           if k not in ("loglik", "rescued")}
    r = init.r
    _cmp("logf", sub["logf"], R["logf"], 0, 1e-4)
    _cmp("tau", sub["tau"], R["tau"], 0, 1e-5)
    for k in ("e1", "e2"):
        _cmp(k, sub[k], R[k], 2e-4)
    _cmp("e3", sub["e3"], np.transpose(R["e3"], (0, 2, 1)), 2e-4)
    _cmp("e4", sub["e4"], np.stack([R["e4"][:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1), 2e-4)


def test_estep_fp64_far_tail_pairs_with_subnormal_pass_sums():
    """5003 rows of the p=4, r=4, g=3 workload on a 512-point lattice: some
    pairs' pass-B lattice sums are subnormal doubles (1e-313 .. 2e-308, where
    1 / S_B overflows) and 400 have S_A > 0 with S_B = 0.  Every E-step output
    against the oracle at the FP64 bars, all finite, and the M-step on them."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 5003, 512)
    R = _oracle_estep(Y, init, lat)
    G = _gpu_estep(Y, init, lat, binding.CFUST_FP64)
    _compare_estep(G, R, init.r, True)
    for k in ("e1", "e2", "e3", "e4"):
        assert np.all(np.isfinite(G[k])), k
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        E = ctx.cfust_estep(Yd, init)
        ctx.cfust_mstep(Yd, E, init)


def test_loglik_matches_oracle_fp64():
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 257, 1024)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref = O.loglik(Y, init, U)
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        got = ctx.cfust_loglik(torch.from_numpy(Y).cuda(), init)
    assert abs(got - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_skew_normal_limit_matches_oracle(precision):
    """A mixture with one component in the skew-normal limit (nu = inf) beside
    skew t components: every E-step output against the oracle (the limit's
    e1 = 1 and e2 = 0 exactly), and the M-step keeps nu = inf."""
    import math
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 150, 1024)
    P = init.copy()
    P.nu[1] = math.inf
    R = _oracle_estep(Y, P, lat)
    G = _gpu_estep(Y, P, lat, precision)
    _compare_estep(G, R, P.r, precision == binding.CFUST_FP64)
    live = R["tau"][1] > 0
    assert np.all(G["e1"][1][live] == 1.0) and np.all(G["e2"][1][live] == 0.0)
    if precision == binding.CFUST_FP64:
        ref = O.mstep_update(O.mstep_sums(Y, R["tau"], R["e1"], R["e2"], R["e3"], R["e4"]), P, Y.shape[0])
        r = P.r
        dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        E = dict(tau=dev(R["tau"]), e1=dev(R["e1"]), e2=dev(R["e2"]),
                 e3=dev(np.transpose(R["e3"], (0, 2, 1))),
                 e4=dev(np.stack([R["e4"][:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1)))
        with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
            got = ctx.cfust_mstep(dev(Y), E, P)
        assert math.isinf(got.nu[1]) and math.isinf(ref.nu[1])
        for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
            _cmp(name, a, b, 1e-10)


def test_loglik_shifts_match_oracle_and_restore_the_rule():
    """l(Psi) under three shifted copies of the lattice (randomised QMC error
    estimate) against the oracle at each shifted rule; the context's own
    rule is back afterwards (bitwise), also after a rejected shift."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 130, 256)
    shifts = np.stack([synth.make_lattice(lat.n, 4, s).shift for s in (3, 4, 5)])
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        before = ctx.cfust_loglik(Yd, init)
        got = ctx.cfust_loglik_shifts(Yd, init, shifts)
        assert ctx.cfust_loglik(Yd, init) == before
        bad = shifts.copy()
        bad[1, 2] = 1.0
        with pytest.raises(binding.CfustError):
            ctx.cfust_loglik_shifts(Yd, init, bad)
        assert ctx.cfust_loglik(Yd, init) == before
    for m in range(shifts.shape[0]):
        ref = O.loglik(Y, init, O.lattice_points(lat.n, lat.z, shifts[m]))
        assert abs(got[m] - ref) <= 1e-10 * abs(ref), (m, got[m], ref)
    assert np.std(got) > 0


def test_mstep_matches_oracle_fp64():
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 300, 1024)
    R = _oracle_estep(Y, init, lat)
    ref = O.mstep_update(O.mstep_sums(Y, R["tau"], R["e1"], R["e2"], R["e3"], R["e4"]), init, Y.shape[0])
    r = init.r
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    E = dict(tau=dev(R["tau"]), e1=dev(R["e1"]), e2=dev(R["e2"]),
             e3=dev(np.transpose(R["e3"], (0, 2, 1))),
             e4=dev(np.stack([R["e4"][:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1)))
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        got = ctx.cfust_mstep(dev(Y), E, init)
    for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
        _cmp(name, a, b, 1e-10)


@pytest.mark.parametrize("workload", ["cfust_p4r4g3_n100000_N4096", "cfust_p3r3g4_n1000000_N2048",
                                      "cfust_p2r2g2_n2000_N1024"])
def test_mstep_matches_oracle_fp32(workload):
    """Single-precision-mode M-step (CFUST_FP32) against the oracle's FP64
    M-step on the same single-precision tau and e1..e4.  The three mixtures
    have 141, 120 and 34 sum entries: one, two and four threads share an
    entry's column sums in the kernel.

    The kernel forms every product tau e y exactly (two-product, y split
    into two floats) and sums them in double-float within a 64-observation
    tile, in double across tiles: the double-precision sums of the same
    inputs up to ~1e-13 of the sum of |terms|.  Sigma's update cancels the
    mean part of S7 (|mu|^2 / sigma^2 of order 10) and nu's equation uses
    1 + S8/S1 (of order 1/nu), so 1e-9 relative keeps a margin of ~100 on
    both.  2000 rows: 32 tiles over many blocks, a ragged last tile
    (2000 = 31 x 64 + 16).
    """
    torch = _torch()
    Y, truth, init, lat = _problem(workload, 2000, 1024)
    R = _oracle_estep(Y, init, lat)
    r = init.r
    f32 = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    tau, e1, e2, e3, e4 = (f32(R[k]) for k in ("tau", "e1", "e2", "e3", "e4"))
    ref = O.mstep_update(O.mstep_sums(Y, tau.astype(np.float64), e1.astype(np.float64), e2.astype(np.float64),
                                      e3.astype(np.float64), e4.astype(np.float64)), init, Y.shape[0])
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    E = dict(tau=dev(tau), e1=dev(e1), e2=dev(e2), e3=dev(np.transpose(e3, (0, 2, 1))),
             e4=dev(np.stack([e4[:, :, t, h] for t in range(r) for h in range(t + 1)], axis=1)))
    with binding.Context(lat, precision=binding.CFUST_FP32) as ctx:
        got = ctx.cfust_mstep(dev(Y), E, init)
    for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
        _cmp(name, a, b, 1e-9)


def _fit_gpu(Y, params, lat, precision, iters, use_graph=True):
    torch = _torch()
    with binding.Context(lat, precision=precision, max_iter=iters, use_graph=use_graph) as ctx:
        return ctx.cfust_fit(torch.from_numpy(Y).cuda(), params)


def test_fit_fp64_matches_oracle_and_graph_replay_is_bitwise_equal():
    Y, truth, init, lat = _problem("cfust_p2r2g2_n2000_N1024", 300, 1024)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref, ref_trace = O.fit(Y, init, U, 5)
    got, trace, done = _fit_gpu(Y, init, lat, binding.CFUST_FP64, 5)
    assert done == 5
    _cmp("trace", trace, ref_trace, 1e-10)
    for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
        _cmp(name, a, b, 1e-8)
    got2, trace2, _ = _fit_gpu(Y, init, lat, binding.CFUST_FP64, 5, use_graph=False)
    assert np.array_equal(trace, trace2)
    for a, b in zip(got.as_arrays(), got2.as_arrays()):
        assert np.array_equal(a, b)


def _load_golden(name):
    with open(os.path.join(HERE, "golden", name)) as f:
        return json.load(f)


def parameter_errors(got, ref):
    """Relative error of every fitted parameter entry, each against the scale
    of the quantity it measures (no common floor):
      pi_i, nu_i                 |a - b| / |b|
      mu_i[a]                    |a - b| / max(|b|, sqrt(Sigma_i[a][a]))   (a location: its own
                                 size, or the component's spread along a when it sits near 0)
      Sigma_i[a][b]              |a - b| / sqrt(Sigma_i[a][a] Sigma_i[b][b]) (>= |b| by
                                 Cauchy-Schwarz; equal to |b| on the diagonal)
      Delta_i[a][t]              |a - b| / max(|b|, sqrt(Omega_i[a][a])), Omega = Sigma + Delta Delta^T
                                 (a skewness loading in units of y_a)
    Returns {name: max error}."""
    pi, mu, Sig, Dl, nu = (np.asarray(x, dtype=np.float64) for x in ref)
    pa, ma, Sa, Da, na = (np.asarray(x, dtype=np.float64) for x in got)
    sd = np.sqrt(np.einsum("iaa->ia", Sig))
    om = np.sqrt(np.einsum("iaa->ia", Sig) + np.sum(Dl * Dl, axis=2))
    out = {"pi": np.max(np.abs(pa - pi) / np.abs(pi)),
           "nu": np.max(np.abs(na - nu) / np.abs(nu)),
           "mu": np.max(np.abs(ma - mu) / np.maximum(np.abs(mu), sd)),
           "Sigma": np.max(np.abs(Sa - Sig) / np.sqrt(sd[:, :, None] ** 2 * sd[:, None, :] ** 2)),
           "Delta": np.max(np.abs(Da - Dl) / np.maximum(np.abs(Dl), om[:, :, None]))}
    return {k: float(v) for k, v in out.items()}


@pytest.mark.parametrize("golden", ["fit_cfust_p4r4g3_n5000_N4096_it50.json",
                                    "fit_cfust_p4r4g3_n1500_N1024_it50.json",
                                    "fit_cfust_p2r2g2_n2000_N1024_it20.json"])
def test_fit_fp32_parameters_match_oracle_golden(golden):
    """Single-precision E-step fits against the FP64 oracle's fits (stored by
    tests/golden/make_fit_golden.py): the log-likelihood trace to 1e-6
    relative at every iteration and every parameter entry to 1e-3 relative
    after the last one (50 iterations on the p=4, r=4, g=3 workload; the 5000-row
    case uses the bench's 4096-point lattice), each entry against its own
    scale (parameter_errors)."""
    G = _load_golden(golden)
    Y, _, truth, init, _, meta = synth.workload(G["workload"], n=G["n"])
    assert np.allclose(Y[:4], G["y_head"], rtol=1e-10, atol=0) and \
        np.allclose(Y.sum(axis=0), G["y_colsum"], rtol=1e-10, atol=1e-9), "input generator drifted"
    lat = synth.make_lattice(G["lattice_n"], meta["r"] + 1, G["lattice_seed"])
    got, trace, done = _fit_gpu(Y, init, lat, binding.CFUST_FP32, G["iters"])
    assert done == G["iters"]
    ref_trace = np.array(G["trace"])
    assert np.all(np.abs(trace - ref_trace) <= 1e-6 * np.abs(ref_trace))
    ref = [np.array(G["params"][k]) for k in ("pi", "mu", "Sigma", "Delta", "nu")]
    errs = parameter_errors(got.as_arrays(), ref)
    print(golden, "FP32 parameter errors", errs)
    for name, e in errs.items():
        assert e <= 1e-3, f"{name}: relative error {e:.3g}"
    # the same fit in FP64 mode reproduces the oracle far more tightly
    got64, trace64, _ = _fit_gpu(Y, init, lat, binding.CFUST_FP64, G["iters"])
    assert np.all(np.abs(trace64 - ref_trace) <= 1e-9 * np.abs(ref_trace))
    errs64 = parameter_errors(got64.as_arrays(), ref)
    print(golden, "FP64 parameter errors", errs64)
    for name, e in errs64.items():
        assert e <= 1e-8, f"FP64 {name}: relative error {e:.3g}"


def test_repeat_runs_are_bitwise_identical_fp32():
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 5000, 2048)
    a = _gpu_estep(Y, init, lat, binding.CFUST_FP32)
    b = _gpu_estep(Y, init, lat, binding.CFUST_FP32)
    for k in ("logf", "tau", "e1", "e2", "e3", "e4"):
        assert np.array_equal(a[k], b[k]), k
    assert a["loglik"] == b["loglik"]


def test_invalid_parameters_are_rejected():
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p2r2g2_n2000_N1024", 50, 1024)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        bad = init.copy(); bad.Sigma[0] = np.array([[1.0, 2.0], [2.0, 1.0]])
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_loglik(Yd, bad)
        assert ei.value.status == -2
        bad = init.copy(); bad.pi[0] += 0.1
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_loglik(Yd, bad)
        assert ei.value.status == -1
        bad = init.copy(); bad.nu[1] = -1.0
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_loglik(Yd, bad)
        assert ei.value.status == -1
        # the context stays usable after errors
        assert np.isfinite(ctx.cfust_loglik(Yd, init))


def test_degenerate_component_is_reported():
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p2r2g2_n2000_N1024", 200, 1024)
    P = init.copy()
    P.mu[1] = np.array([1e4, -1e4])     # no observation near component 2
    P.Delta[1] = 0.0
    P.nu[1] = 30.0
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2) as ctx:
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_fit(torch.from_numpy(Y).cuda(), P)
        assert ei.value.status == -4


PRIO_CASES = [
    ("cfust_p2r2g2_n2000_N1024", 200, 1024),
    ("cfust_p4r4g3_n100000_N4096", 200, 1024),
    ("cfust_p3r3g4_n1000000_N2048", 150, 1024),
]


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", PRIO_CASES, ids=[c[0].split("_n")[0] for c in PRIO_CASES])
def test_prioritised_estep_matches_oracle(case, precision):
    """Variable prioritisation: the same reordered integrand on both sides (the
    order decided in double from the same q and Lambda), every E-step output
    at the usual bars, with most pairs actually reordered."""
    wl, n, N = case
    Y, truth, init, lat = _problem(wl, n, N)
    R = _oracle_estep(Y, init, lat, prioritise=True)
    G = _gpu_estep(Y, init, lat, precision, prioritise=True)
    _compare_estep(G, R, init.r, precision == binding.CFUST_FP64)
    moved = 0
    for i in range(init.g):
        d, q, Lam, _ = O.component_terms(Y, init.mu[i], init.Sigma[i], init.Delta[i], init.nu[i])
        moved += int((O.prioritised_order(-q, Lam) != np.arange(init.r)).any(axis=1).sum())
    assert moved > 0.3 * init.g * Y.shape[0]


def test_prioritised_fit_fp64_matches_oracle():
    """Two EM iterations with prioritisation against the oracle's (FP64)."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p2r2g2_n2000_N1024", 300, 512)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    n = Y.shape[0]
    ref, ref_tr = init.copy(), []
    for _ in range(2):
        E = O.estep(Y, ref, U, prioritise=True)
        ref_tr.append(E["loglik"])
        ref = O.mstep_update(O.mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]), ref, n)
    ref_tr.append(O.loglik(Y, ref, U, prioritise=True))
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2, prioritise=True) as ctx:
        got, tr, done = ctx.cfust_fit(Yd, init)
    assert done == 2
    assert np.allclose(tr, ref_tr, rtol=1e-10, atol=0)
    for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
        _cmp(name, a, b, 1e-8)


@pytest.mark.parametrize("prioritise", [False, True])
def test_fp32_rescued_pairs_match_oracle(prioritise):
    """Pairs whose float lattice weights underflow go through the log-domain
    rescue sweep; they must meet the same FP32 tolerances as the rest (with
    prioritisation the rescue integrates in the same order).  Rows planted at
    mu_i - c Delta_i 1 put T_A of one component near exp(-145) and exp(-274)."""
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 200, 512)
    extra = [init.mu[i] - c * init.Delta[i].sum(axis=1) for i in range(init.g) for c in (2.0, 4.0, 8.0, 16.0)]
    Y = np.ascontiguousarray(np.vstack([Y, np.array(extra)]))
    R = _oracle_estep(Y, init, lat, prioritise=prioritise)
    G = _gpu_estep(Y, init, lat, binding.CFUST_FP32, prioritise=prioritise)
    # in natural order these rows underflow the float sweep; the prioritised
    # order integrates the restrictive variable first and may keep them in range
    print("rescued pairs", G["rescued"], "prioritise", prioritise)
    if not prioritise:
        assert G["rescued"] >= 2, G["rescued"]
    _compare_estep(G, R, init.r, False)
    tiny = R["logf"] < -60.0
    assert tiny.sum() >= 2
    _cmp("logf tail", G["logf"][tiny], R["logf"][tiny], 0, 1e-4)


def test_stepwise_fit_equals_fit_and_triage_keeps_loglik():
    """cfust_fit_begin/step/trace/end reproduce cfust_fit bit for bit, and with
    planted far outliers (whose float sums underflow and are triaged) the FP32
    log-likelihood trace still matches the oracle to 1e-6 relative."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 300, 512)
    extra = [init.mu[i] - c * init.Delta[i].sum(axis=1) for i in range(init.g) for c in (4.0, 8.0, 16.0)]
    Y = np.ascontiguousarray(np.vstack([Y, np.array(extra)]))
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=3) as ctx:
        p1, t1, d1 = ctx.cfust_fit(Yd, init)
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=3) as ctx:
        ctx.cfust_fit_begin(Yd, init)
        ctx.cfust_fit_step(2)
        mid = ctx.cfust_fit_trace()
        ctx.cfust_fit_step(1)
        p2, t2, d2 = ctx.cfust_fit_end()
    assert d1 == d2 == 3 and np.array_equal(t1, t2) and np.array_equal(mid, t1[:2])
    for a, b in zip(p1.as_arrays(), p2.as_arrays()):
        assert np.array_equal(a, b)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref = O.loglik(Y, init, U)
    assert abs(t1[0] - ref) <= 1e-6 * abs(ref)


def _two_underflowing_components():
    """A p=1, r=1, g=2 mixture with both components near the normal limit and
    skewed downwards, its own draws plus four rows at y = 17.5 .. 19: there
    both pairs' single-precision lattice sums underflow, component 0
    outweighs component 1 by 256 to 296 nats under the 512-point rule, and yet
    component 0's pending density bound trails component 1's by about 30.5
    nats (both bounds sit at log t + log 1e-37 + 1, and component 1 has the
    larger log t)."""
    P = synth.Params(pi=np.array([0.5, 0.5]), mu=np.array([[1.400927034064857], [-0.4946095065202325]]),
                     Sigma=np.array([[[0.5344986830086018 ** 2]], [[0.4538790293528015 ** 2]]]),
                     Delta=np.array([[[-1.299385364828229]], [[-2.706859290038734]]]), nu=np.array([200.0, 200.0]))
    Y, _ = synth.sample_cfust(P, 300, np.random.default_rng(7))
    Y = np.ascontiguousarray(np.vstack([Y, np.array([[17.5], [18.0], [18.5], [19.0]])]))
    return Y, P, synth.make_lattice(512, 2, 0)


@pytest.mark.parametrize("fused", [False, True])
def test_triage_compares_with_final_values_only(fused):
    """The triage of pairs left to the double-precision rescue drops a pair
    only against another component's FINAL log f: another pending pair's
    bound is an upper bound (here it would wrongly drop the component that
    carries the far rows).  The FP32 log-likelihood, with the triage on,
    against the oracle to 1e-6 relative (-1599.7): a wrong drop of component
    0 at a far row would move it by more than 250 nats."""
    torch = _torch()
    Y, P, lat = _two_underflowing_components()
    ref = O.loglik(Y, P, O.lattice_points(lat.n, lat.z, lat.shift))
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP32, fused=fused, max_iter=1) as ctx:
        got = ctx.cfust_loglik(Yd, P)
        rescued = ctx.cfust_last_rescued()
        _, trace, _ = ctx.cfust_fit(Yd, P)
    print("rescued pairs", rescued)
    assert rescued >= 8, rescued
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
    assert abs(trace[0] - ref) <= 1e-6 * abs(ref), (trace[0], ref)
