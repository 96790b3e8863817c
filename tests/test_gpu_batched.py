"""Batched fits (one persistent sweep launch per EM iteration over every fit)
against the same fits run one at a time, and against the FP64 oracle."""
import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import binding, synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _small_batch(nfits=5, seed0=40):
    return synth.batched_workload(nfits, seed0=seed0, n_lo=60, n_hi=1500)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_batched_equals_single_fits(precision):
    torch = _torch()
    Ys, truths, inits = _small_batch()
    lat = synth.make_lattice(256, 4, 0)
    Yd = [torch.from_numpy(Y).cuda() for Y in Ys]
    iters = 3
    with binding.Context(lat, precision=precision, max_iter=iters) as ctx:
        bp, btr, st = ctx.cfust_fit_batched(Yd, inits)
    assert all(s == 0 for s in st)
    for f, (Y, P0) in enumerate(zip(Yd, inits)):
        with binding.Context(lat, precision=precision, max_iter=iters) as ctx:
            sp, str_, _ = ctx.cfust_fit(Y, P0)
        assert np.allclose(btr[f], str_, rtol=1e-12, atol=0), f
        for a, b in zip(bp[f].as_arrays(), sp.as_arrays()):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14), f


def test_batched_fp64_matches_oracle_on_two_fits():
    torch = _torch()
    # two fits with every component well populated (S6 well conditioned)
    Ys, truths, inits = synth.batched_workload(2, seed0=7, n_lo=800, n_hi=1500, g_hi=3)
    lat = synth.make_lattice(256, 4, 3)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2) as ctx:
        bp, btr, st = ctx.cfust_fit_batched([torch.from_numpy(Y).cuda() for Y in Ys], inits)
    for f in range(2):
        ref, ref_tr = O.fit(Ys[f], inits[f], U, 2)
        assert np.allclose(btr[f], ref_tr, rtol=1e-10, atol=0)
        for a, b in zip(bp[f].as_arrays(), ref.as_arrays()):
            assert np.allclose(a, b, rtol=1e-8, atol=1e-10)


def test_batched_skew_normal_limit_matches_oracle():
    """Two fits, one with a component in the skew-normal limit (nu = inf):
    FP64 batched EM against the oracle's fit; nu = inf is kept."""
    import math
    torch = _torch()
    Ys, truths, inits = synth.batched_workload(2, seed0=7, n_lo=800, n_hi=1500, g_hi=3)
    inits[0].nu[0] = math.inf
    lat = synth.make_lattice(256, 4, 3)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2) as ctx:
        bp, btr, st = ctx.cfust_fit_batched([torch.from_numpy(Y).cuda() for Y in Ys], inits)
    assert all(s_ == 0 for s_ in st)
    assert math.isinf(bp[0].nu[0])
    for f in range(2):
        ref, ref_tr = O.fit(Ys[f], inits[f], U, 2)
        assert np.allclose(btr[f], ref_tr, rtol=1e-10, atol=0)
        for a, b in zip(bp[f].as_arrays(), ref.as_arrays()):
            assert np.allclose(a, b, rtol=1e-8, atol=1e-10)


def test_autotuned_shape_gives_the_same_fits():
    torch = _torch()
    Ys, truths, inits = _small_batch(4, seed0=90)
    lat = synth.make_lattice(512, 4, 0)
    Yd = [torch.from_numpy(Y).cuda() for Y in Ys]
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=2, autotune=True) as ctx:
        a, ta, _ = ctx.cfust_fit_batched(Yd, inits)
        ppw, cps = ctx.cfust_batched_shape()
        # a second call on the same batch reuses the tuned shape and the graph
        a2, ta2, _ = ctx.cfust_fit_batched(Yd, inits)
    assert ppw in (2, 4, 8, 16) and cps in (1, 2)
    assert np.array_equal(ta, ta2)
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=2, pairs_per_warp=1) as ctx:
        b, tb, _ = ctx.cfust_fit_batched(Yd, inits)
    assert np.allclose(ta, tb, rtol=1e-12)
    for pa, pb in zip(a, b):
        for x, y in zip(pa.as_arrays(), pb.as_arrays()):
            assert np.allclose(x, y, rtol=1e-12, atol=1e-14)


def test_one_degenerate_fit_is_reported_alone():
    torch = _torch()
    Ys, truths, inits = _small_batch(3, seed0=11)
    bad = inits[1].copy()
    bad.mu[0] = 1e4            # no observation near this component
    bad.Delta[0] = 0.0
    inits = [inits[0], bad, inits[2]]
    lat = synth.make_lattice(256, 4, 0)
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2) as ctx:
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_fit_batched([torch.from_numpy(Y).cuda() for Y in Ys], inits)
    assert ei.value.status == -4
    assert "fit 1" in str(ei.value)


def test_full_batch_of_256_fits_matches_sampled_single_fits():
    """The 256-fit workload (n log-uniform in [5000, 200000], g in 2..5, 2048-point
    lattice) in the bench's launch configuration for one EM iteration; three
    sampled fits are rerun alone and must agree."""
    torch = _torch()
    Ys, truths, inits = synth.batched_workload(256)
    lat = synth.make_lattice(2048, 4, 0)
    Yd = [torch.from_numpy(Y).cuda() for Y in Ys]
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=1, autotune=True) as ctx:
        bp, btr, st = ctx.cfust_fit_batched(Yd, inits)
    assert all(s == 0 for s in st)
    assert np.all(np.isfinite(btr))
    for f in (0, 97, 255):
        with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=1) as ctx:
            sp, str_, _ = ctx.cfust_fit(Yd[f], inits[f])
        assert np.allclose(btr[f], str_, rtol=1e-12, atol=0)
        for a, b in zip(bp[f].as_arrays(), sp.as_arrays()):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14)


def test_multistart_keeps_the_best_burned_in_start():
    """Algorithm 1 with burn-in: four starts run three EM iterations together
    (one batched fit); the one with the largest log-likelihood (the oracle's
    selection rule) is fitted further, and equals that start's own burn-in
    continued by a single fit."""
    torch = _torch()
    Y, _, truth, init, _, _ = synth.workload("cfust_p3r3g4_n1000000_N2048", n=4000, seed=5)
    rng = np.random.default_rng(3)
    starts = [init] + [synth.perturb_params(truth, rng, 0.8) for _ in range(3)]
    lat = synth.make_lattice(1024, 4, seed=0)
    Yd = torch.from_numpy(Y).cuda()
    ctx = binding.Context(lat, precision=binding.CFUST_FP32, max_iter=5)
    best, P, trace, done, _ = ctx.cfust_fit_multistart(Yd, starts, burn_in=3)
    burned, lls = [], []
    for st in starts:
        c1 = binding.Context(lat, precision=binding.CFUST_FP32, max_iter=3)
        Pb, tr, _ = c1.cfust_fit(Yd, st)
        burned.append(Pb)
        lls.append(tr[-1])
    assert best == O.select_start(lls)
    c2 = binding.Context(lat, precision=binding.CFUST_FP32, max_iter=5)
    Pref, tref, dref = c2.cfust_fit(Yd, burned[best])
    assert done == dref and np.allclose(trace, tref, rtol=1e-10, atol=0)
    for a, b in zip(P.as_arrays(), Pref.as_arrays()):
        assert np.allclose(a, b, rtol=1e-8, atol=1e-10)
    # burn_in = 0 selects on the starts' own log-likelihoods
    c3 = binding.Context(lat, precision=binding.CFUST_FP32, max_iter=2)
    best0, _, _, _, _ = c3.cfust_fit_multistart(Yd, starts, burn_in=0)
    assert best0 == O.select_start([c3.cfust_loglik(Yd, st) for st in starts])


def _oracle_fit_prioritised(Y, P, U, iters):
    """The oracle's EM with variable prioritisation in every E-step."""
    n = Y.shape[0]
    params, trace = P.copy(), []
    for _ in range(iters):
        E = O.estep(Y, params, U, prioritise=True)
        trace.append(E["loglik"])
        params = O.mstep_update(O.mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]), params, n)
    trace.append(O.loglik(Y, params, U, prioritise=True))
    return params, np.array(trace)


def test_batched_prioritised_matches_oracle_fp64():
    """Variable prioritisation in the persistent batched sweep: two fits, two
    EM iterations in double precision against the oracle's prioritised EM."""
    torch = _torch()
    Ys, truths, inits = synth.batched_workload(2, seed0=7, n_lo=800, n_hi=1500, g_hi=3)
    lat = synth.make_lattice(256, 4, 3)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=2, prioritise=True) as ctx:
        bp, btr, st = ctx.cfust_fit_batched([torch.from_numpy(Y).cuda() for Y in Ys], inits)
    assert all(s_ == 0 for s_ in st)
    for f in range(2):
        ref, ref_tr = _oracle_fit_prioritised(Ys[f], inits[f], U, 2)
        assert np.allclose(btr[f], ref_tr, rtol=1e-10, atol=0)
        for a, b in zip(bp[f].as_arrays(), ref.as_arrays()):
            assert np.allclose(a, b, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_batched_prioritised_equals_single_prioritised_fits(precision):
    """The prioritised batched sweep reproduces the same fits run one at a
    time with prioritisation (same per-pair arithmetic)."""
    torch = _torch()
    Ys, truths, inits = _small_batch()
    lat = synth.make_lattice(256, 4, 0)
    Yd = [torch.from_numpy(Y).cuda() for Y in Ys]
    iters = 3
    with binding.Context(lat, precision=precision, max_iter=iters, prioritise=True) as ctx:
        bp, btr, st = ctx.cfust_fit_batched(Yd, inits)
    assert all(s == 0 for s in st)
    for f, (Y, P0) in enumerate(zip(Yd, inits)):
        with binding.Context(lat, precision=precision, max_iter=iters, prioritise=True) as ctx:
            sp, str_, _ = ctx.cfust_fit(Y, P0)
        assert np.allclose(btr[f], str_, rtol=1e-12, atol=0), f
        for a, b in zip(bp[f].as_arrays(), sp.as_arrays()):
            assert np.allclose(a, b, rtol=1e-12, atol=1e-14), f
