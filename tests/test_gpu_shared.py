"""Pass B on pass A's lattice points (cfust_opts.shared_points) against the
FP64 oracle run with the same rule (shared=True), through the C ABI.

Same bars as the two-pass rule: FP64 mode log f and l to 1e-10 relative, tau
and e1..e4 to 1e-9; FP32 mode log f 1e-4 absolute, tau 1e-5, e1..e4 2e-4,
l 1e-6 relative, fitted parameters 1e-3 of their scale.
"""
import math

import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import binding, synth

from test_gpu_parity import CASES, _cmp, _compare_estep, _problem, parameter_errors

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _gpu(Y, params, lat, precision, shared=True, e2_mode=0, prioritise=False):
    torch = _torch()
    with binding.Context(lat, precision=precision, e2_mode=e2_mode, shared_points=shared,
                         prioritise=prioritise) as ctx:
        out = ctx.cfust_estep(torch.from_numpy(Y).cuda(), params)
        res = {k: (v.double().cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
        res["rescued"] = ctx.cfust_last_rescued()
    return res


def _oracle(Y, params, lat, e2_mode=0, prioritise=False):
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    return O.estep(Y, params, U, e2_mode, prioritise=prioritise, shared=True)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", CASES, ids=[c[0].split("_n")[0] for c in CASES])
def test_shared_estep_matches_oracle(case, precision):
    wl, n, N = case
    Y, truth, init, lat = _problem(wl, n, N)
    _compare_estep(_gpu(Y, init, lat, precision), _oracle(Y, init, lat), init.r,
                   precision == binding.CFUST_FP64)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_shared_estep_lattice_e2_mode(precision):
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 90, 1024)
    _compare_estep(_gpu(Y, init, lat, precision, e2_mode=1), _oracle(Y, init, lat, e2_mode=1), init.r,
                   precision == binding.CFUST_FP64)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("g,p,r,n,N", [
    (1, 1, 1, 1, 32),        # one point per lane: every second point is past N
    (1, 1, 1, 37, 64),       # ragged observations
    (2, 16, 6, 40, 256),     # the largest p and r
    (3, 5, 2, 129, 96),      # the last pair of points half past N
    (5, 3, 3, 64, 128),
])
def test_shared_estep_edge_shapes(g, p, r, n, N, precision):
    rng = np.random.default_rng(100 + g * 7 + p)
    P = synth.random_params(rng, g, p, r, 9.0, 2, 1.5, 3.0, 12.0)
    Y, _ = synth.sample_cfust(P, n, rng)
    lat = synth.make_lattice(N, r + 1, 5)
    _compare_estep(_gpu(Y, P, lat, precision), _oracle(Y, P, lat), r, precision == binding.CFUST_FP64)


def test_shared_full_size_sampled_fp32():
    """The p=4, r=4, g=3, n=100000, N=4096 workload in the bench's launch
    configuration; 48 sampled observations (all components) recomputed by the
    oracle, every E-step output at the single-precision bars."""
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", None, 4096)
    G = _gpu(Y, init, lat, binding.CFUST_FP32)
    idx = np.sort(np.random.default_rng(7).choice(Y.shape[0], 48, replace=False))
    R = _oracle(Y[idx], init, lat)
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


def test_shared_fp32_rescued_pairs_match_oracle():
    """Rows planted far on the short side of each component's skewness underflow
    the float sweep; the log-domain rescue takes pass B from pass A's draws too."""
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 200, 512)
    extra = [init.mu[i] - c * init.Delta[i].sum(axis=1) for i in range(init.g) for c in (2.0, 4.0, 8.0, 16.0)]
    Y = np.ascontiguousarray(np.vstack([Y, np.array(extra)]))
    G = _gpu(Y, init, lat, binding.CFUST_FP32)
    assert G["rescued"] >= 2, G["rescued"]
    _compare_estep(G, _oracle(Y, init, lat), init.r, False)


def test_shared_leaves_the_density_unchanged_fp64():
    """log f and l come from pass A alone: in double precision the shared rule
    gives them bit for bit as the two-pass rule does."""
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 300, 1024)
    a = _gpu(Y, init, lat, binding.CFUST_FP64, shared=False)
    b = _gpu(Y, init, lat, binding.CFUST_FP64, shared=True)
    assert np.array_equal(a["logf"], b["logf"])
    assert a["loglik"] == b["loglik"]


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_shared_skew_normal_limit_matches_oracle(precision):
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 150, 1024)
    P = init.copy()
    P.nu[1] = math.inf
    G = _gpu(Y, P, lat, precision)
    R = _oracle(Y, P, lat)
    _compare_estep(G, R, P.r, precision == binding.CFUST_FP64)
    live = R["tau"][1] > 0
    assert np.all(G["e1"][1][live] == 1.0) and np.all(G["e2"][1][live] == 0.0)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_shared_fit_matches_oracle_fit(precision):
    """Ten EM iterations of the p=4, r=4, g=3 workload (1500 rows, 1024 points)
    with the shared rule on both sides: the trace and every fitted parameter."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 1500, 1024)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref, ref_tr = O.fit(Y, init, U, 10, shared=True)
    with binding.Context(lat, precision=precision, max_iter=10, shared_points=True) as ctx:
        got, tr, done = ctx.cfust_fit(torch.from_numpy(Y).cuda(), init)
    assert done == 10
    if precision == binding.CFUST_FP64:
        _cmp("trace", tr, ref_tr, 1e-10)
        for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
            _cmp(name, a, b, 1e-8)
    else:
        assert np.all(np.abs(tr - ref_tr) <= 1e-6 * np.abs(ref_tr))
        errs = parameter_errors(got.as_arrays(), ref.as_arrays())
        assert max(errs.values()) <= 1e-3, errs


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", CASES[1:], ids=[c[0].split("_n")[0] for c in CASES[1:]])
def test_shared_prioritised_estep_matches_oracle(case, precision):
    """Variable prioritisation with pass B on pass A's points: each pair's
    chain in its own order serves both passes, the moments scattered back."""
    wl, n, N = case
    Y, truth, init, lat = _problem(wl, n, N)
    _compare_estep(_gpu(Y, init, lat, precision, prioritise=True), _oracle(Y, init, lat, prioritise=True),
                   init.r, precision == binding.CFUST_FP64)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", [("cfust_p4r4g3_n100000_N4096", 1003, 1024, False),
                                  ("cfust_p3r3g4_n1000000_N2048", 777, 512, True),
                                  ("cfust_p8r4g6_n1000000_N8192", 301, 1024, False)],
                         ids=["p4r4g3", "p3r3g4-prio", "p8r4g6"])
def test_shared_fused_fit_agrees_with_unfused(case, precision):
    """The fused E-step + sums pass with the shared rule against the unfused
    shared fit: the same per-pair arithmetic, sums in another order."""
    torch = _torch()
    wl, n, N, prio = case
    Y, truth, init, lat = _problem(wl, n, N)
    out = []
    for fused in (False, True):
        with binding.Context(lat, precision=precision, max_iter=3, fused=fused, prioritise=prio,
                             shared_points=True) as ctx:
            got, trace, done = ctx.cfust_fit(torch.from_numpy(Y).cuda(), init)
        assert done == 3
        out.append((got, trace))
    (a, ta), (b, tb) = out
    assert abs(tb[0] - ta[0]) <= 1e-12 * abs(ta[0]), (ta[0], tb[0])
    assert np.all(np.abs(tb - ta) <= 1e-9 * np.abs(ta)), (ta, tb)
    errs = parameter_errors(b.as_arrays(), a.as_arrays())
    bar = 1e-9 if precision == binding.CFUST_FP64 else 1e-6
    for name, e in errs.items():
        assert e <= bar, f"{name}: fused vs unfused relative difference {e:.3g}"


@pytest.mark.parametrize("prioritise", [False, True])
def test_shared_batched_fits_match_oracle_fp64(prioritise):
    """Two fits in one persistent launch per iteration with the shared rule:
    the trace and the fitted parameters against the oracle's fits."""
    torch = _torch()
    Ys, truths, inits = synth.batched_workload(2, seed0=7, n_lo=800, n_hi=1500, g_hi=3)
    lat = synth.make_lattice(256, 4, 3)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2, shared_points=True,
                         prioritise=prioritise) as ctx:
        bp, btr, st = ctx.cfust_fit_batched([torch.from_numpy(Y).cuda() for Y in Ys], inits)
    assert all(v == 0 for v in st)
    for f in range(2):
        if prioritise:
            # the oracle's fit takes the natural order: run its E- and M-steps by hand
            P = inits[f].copy()
            tr = []
            for _ in range(2):
                E = O.estep(Ys[f], P, U, prioritise=True, shared=True)
                tr.append(E["loglik"])
                P = O.mstep_update(O.mstep_sums(Ys[f], E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]), P,
                                   Ys[f].shape[0])
            tr.append(O.loglik(Ys[f], P, U, prioritise=True))
            ref, ref_tr = P, np.array(tr)
        else:
            ref, ref_tr = O.fit(Ys[f], inits[f], U, 2, shared=True)
        assert np.allclose(btr[f], ref_tr, rtol=1e-10, atol=0)
        for a, b in zip(bp[f].as_arrays(), ref.as_arrays()):
            assert np.allclose(a, b, rtol=1e-8, atol=1e-10)


def test_shared_batched_equals_single_fits_fp32():
    """The batched sweep and the single-fit sweep take the same shared rule:
    the same fits agree to their summation order."""
    torch = _torch()
    Ys, truths, inits = synth.batched_workload(5, seed0=40, n_lo=60, n_hi=1500)
    lat = synth.make_lattice(256, 4, 0)
    Yd = [torch.from_numpy(Y).cuda() for Y in Ys]
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=3, shared_points=True) as ctx:
        bp, btr, st = ctx.cfust_fit_batched(Yd, inits)
    for f, (Y, P0) in enumerate(zip(Yd, inits)):
        with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=3, shared_points=True) as ctx:
            sp, str_, _ = ctx.cfust_fit(Y, P0)
        assert np.allclose(btr[f], str_, rtol=1e-12, atol=0), f
        for a, b in zip(bp[f].as_arrays(), sp.as_arrays()):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14), f


@pytest.mark.parametrize("prioritise", [False, True])
def test_shared_fallback_pairs_equal_the_shared_lattice_estep(prioritise):
    """With a surrogate attached and the shared rule, the pairs the network
    leaves to the lattice rule are bit-identical to the plain shared E-step's."""
    torch = _torch()
    s = binding.Surrogate(synth.make_lattice(8192, 4, seed=11), seed=6)
    s.cfust_surrogate_train(1 << 16, 1, batch=4096, lr=3e-3, seed=2)
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=2000, seed=0)
    Yd = torch.tensor(Y, dtype=torch.float64, device="cuda")
    lat = synth.make_lattice(512, 4, seed=0)
    with binding.Context(lat, precision=binding.CFUST_FP32, prioritise=prioritise, shared_points=True) as plain, \
            binding.Context(lat, precision=binding.CFUST_FP32, prioritise=prioritise, shared_points=True) as sur:
        sur.cfust_set_surrogate(s)
        Ep = plain.cfust_estep(Yd, init)
        Es = sur.cfust_estep(Yd, init)
        _, kind = sur.cfust_surrogate_inputs(Yd, init)
    s.close()
    out = kind.cpu().numpy() != 2
    assert out.sum() > 100
    for k in ("logf", "e1", "e2", "e3", "e4"):
        a = Es[k].cpu().numpy()
        b = Ep[k].cpu().numpy()
        for i in range(init.g):
            assert np.array_equal(a[i][..., out[i]], b[i][..., out[i]]), (i, k)


def test_shared_repeat_fits_are_bitwise_identical_fp32():
    """Fixed-order sums everywhere: the same shared-rule fit twice (the bench
    workload's first 20000 rows, 8 EM iterations, rescued pairs included)
    gives the same trace and parameters bit for bit, as does the E-step."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 20000, 4096)
    Yd = torch.from_numpy(Y).cuda()
    runs = []
    for _ in range(2):
        with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=8, shared_points=True) as ctx:
            runs.append(ctx.cfust_fit(Yd, init))
    (pa, ta, _), (pb, tb, _) = runs
    assert np.array_equal(ta, tb)
    for a, b in zip(pa.as_arrays(), pb.as_arrays()):
        assert np.array_equal(a, b)
    a = _gpu(Y, init, lat, binding.CFUST_FP32)
    b = _gpu(Y, init, lat, binding.CFUST_FP32)
    for k in ("logf", "tau", "e1", "e2", "e3", "e4"):
        assert np.array_equal(a[k], b[k]), k
