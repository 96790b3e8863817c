"""The fused E-step + M-step-sums pass (cfust_opts.fused = 1).

One kernel per EM iteration takes each tile of observations through all g
components, keeps log f_ij and e1..e4 in shared memory, and adds tau-weighted
sums into per-block partials (Algorithm 2's partial sums, Section 3.2's eight
statistics), which Algorithm 3's M-step combines.  The lattice rule and the
arithmetic of every pair are those of the per-pair path, so:
  - against the FP64 oracle it meets the same bars as the unfused path
    (FP64: trace 1e-10, parameters 1e-8; FP32: trace 1e-6, parameters 1e-3
    after 50 iterations, each entry on its own scale);
  - against the unfused path it agrees to summation order: the first
    log-likelihood (same E-step, different block partition of the sum) to
    1e-12 relative, later iterations to 1e-9 (FP32: a parameter difference
    of 1e-13 can flip a float rounding in the next sweep), parameters to 1e-9
    (FP64) and 1e-6 (FP32) relative.
Tiles are ragged (n not a multiple of the tile) in every case below.
"""
import ctypes
import math

import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import binding, synth

from test_gpu_parity import _cmp, _load_golden, _problem, parameter_errors

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _fit(Y, params, lat, precision, iters, fused, **kw):
    torch = _torch()
    with binding.Context(lat, precision=precision, max_iter=iters, fused=fused, **kw) as ctx:
        got, trace, done = ctx.cfust_fit(torch.from_numpy(Y).cuda(), params)
        rescued = ctx.cfust_last_rescued()
    assert done == iters
    return got, trace, rescued


def test_fused_fit_fp64_matches_oracle():
    Y, truth, init, lat = _problem("cfust_p2r2g2_n2000_N1024", 301, 1024)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref, ref_trace = O.fit(Y, init, U, 5)
    got, trace, _ = _fit(Y, init, lat, binding.CFUST_FP64, 5, True)
    _cmp("trace", trace, ref_trace, 1e-10)
    for a, b, name in zip(got.as_arrays(), ref.as_arrays(), ("pi", "mu", "Sigma", "Delta", "nu")):
        _cmp(name, a, b, 1e-8)


FUSED_CASES = [
    # (workload, n, lattice points, prioritise, e2_mode)
    ("cfust_p4r4g3_n100000_N4096", 1003, 1024, False, 0),
    ("cfust_p3r3g4_n1000000_N2048", 777, 512, True, 0),
    ("cfust_p8r4g6_n1000000_N8192", 301, 1024, False, 0),
    ("cfust_p2r2g2_n2000_N1024", 499, 1024, False, 1),
]


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
@pytest.mark.parametrize("case", FUSED_CASES, ids=[f"{c[0].split('_n')[0]}-prio{int(c[3])}-e2m{c[4]}"
                                                   for c in FUSED_CASES])
def test_fused_fit_agrees_with_unfused(case, precision):
    wl, n, N, prio, e2m = case
    Y, truth, init, lat = _problem(wl, n, N)
    a, ta, _ = _fit(Y, init, lat, precision, 3, False, prioritise=prio, e2_mode=e2m)
    b, tb, _ = _fit(Y, init, lat, precision, 3, True, prioritise=prio, e2_mode=e2m)
    assert abs(tb[0] - ta[0]) <= 1e-12 * abs(ta[0]), (ta[0], tb[0])
    assert np.all(np.abs(tb - ta) <= 1e-9 * np.abs(ta)), (ta, tb)
    errs = parameter_errors(b.as_arrays(), a.as_arrays())
    bar = 1e-9 if precision == binding.CFUST_FP64 else 1e-6
    for name, e in errs.items():
        assert e <= bar, f"{name}: fused vs unfused relative difference {e:.3g}"


def test_fused_fits_are_bitwise_repeatable():
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 2001, 512)
    a, ta, _ = _fit(Y, init, lat, binding.CFUST_FP32, 2, True)
    b, tb, _ = _fit(Y, init, lat, binding.CFUST_FP32, 2, True)
    assert np.array_equal(ta, tb)
    for x, y in zip(a.as_arrays(), b.as_arrays()):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("golden", ["fit_cfust_p4r4g3_n5000_N4096_it50.json",
                                    "fit_cfust_p2r2g2_n2000_N1024_it20.json"])
def test_fused_fit_matches_oracle_golden(golden):
    """The stored FP64 oracle fits (tests/golden/make_fit_golden.py), fused:
    FP32 trace to 1e-6 relative at every iteration and parameters to 1e-3
    after the last; FP64 trace to 1e-9, parameters to 1e-8."""
    G = _load_golden(golden)
    Y, _, truth, init, _, meta = synth.workload(G["workload"], n=G["n"])
    assert np.allclose(Y[:4], G["y_head"], rtol=1e-10, atol=0), "input generator drifted"
    lat = synth.make_lattice(G["lattice_n"], meta["r"] + 1, G["lattice_seed"])
    ref_trace = np.array(G["trace"])
    ref = [np.array(G["params"][k]) for k in ("pi", "mu", "Sigma", "Delta", "nu")]
    got, trace, _ = _fit(Y, init, lat, binding.CFUST_FP32, G["iters"], True)
    assert np.all(np.abs(trace - ref_trace) <= 1e-6 * np.abs(ref_trace))
    errs = parameter_errors(got.as_arrays(), ref)
    print(golden, "fused FP32 parameter errors", errs)
    for name, e in errs.items():
        assert e <= 1e-3, f"{name}: relative error {e:.3g}"
    got64, trace64, _ = _fit(Y, init, lat, binding.CFUST_FP64, G["iters"], True)
    assert np.all(np.abs(trace64 - ref_trace) <= 1e-9 * np.abs(ref_trace))
    errs64 = parameter_errors(got64.as_arrays(), ref)
    print(golden, "fused FP64 parameter errors", errs64)
    for name, e in errs64.items():
        assert e <= 1e-8, f"FP64 {name}: relative error {e:.3g}"


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_fused_loglik_matches_oracle(precision):
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 257, 1024)
    ref = O.loglik(Y, init, O.lattice_points(lat.n, lat.z, lat.shift))
    with binding.Context(lat, precision=precision, fused=True) as ctx:
        got = ctx.cfust_loglik(torch.from_numpy(Y).cuda(), init)
    tol = 1e-10 if precision == binding.CFUST_FP64 else 1e-6
    assert abs(got - ref) <= tol * abs(ref), (got, ref)


@pytest.mark.parametrize("prioritise", [False, True])
def test_fused_rescue_and_triage_match_oracle(prioritise):
    """Planted far outliers (rows at mu_i - c Delta_i 1) underflow the float
    sweep of some pairs: the tile's CTA triages or recomputes them in the log
    domain.  The FP32 log-likelihood against the oracle to 1e-6 relative, the
    first fit iteration against the unfused path."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p4r4g3_n100000_N4096", 300, 512)
    extra = [init.mu[i] - c * init.Delta[i].sum(axis=1) for i in range(init.g) for c in (2.0, 4.0, 8.0, 16.0)]
    Y = np.ascontiguousarray(np.vstack([Y, np.array(extra)]))
    ref = O.loglik(Y, init, O.lattice_points(lat.n, lat.z, lat.shift), prioritise=prioritise)
    with binding.Context(lat, precision=binding.CFUST_FP32, fused=True, prioritise=prioritise) as ctx:
        got = ctx.cfust_loglik(torch.from_numpy(Y).cuda(), init)
        rescued = ctx.cfust_last_rescued()
    print("rescued pairs", rescued, "prioritise", prioritise)
    if not prioritise:
        assert rescued >= 2
    assert abs(got - ref) <= 1e-6 * abs(ref), (got, ref)
    a, ta, _ = _fit(Y, init, lat, binding.CFUST_FP32, 1, False, prioritise=prioritise)
    b, tb, _ = _fit(Y, init, lat, binding.CFUST_FP32, 1, True, prioritise=prioritise)
    assert abs(tb[0] - ref) <= 1e-6 * abs(ref)
    assert abs(tb[0] - ta[0]) <= 1e-12 * abs(ta[0])
    for name, e in parameter_errors(b.as_arrays(), a.as_arrays()).items():
        assert e <= 1e-9, f"{name}: {e:.3g}"


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_fused_skew_normal_limit(precision):
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 409, 1024)
    P = init.copy()
    P.nu[1] = math.inf
    a, ta, _ = _fit(Y, P, lat, precision, 2, False)
    b, tb, _ = _fit(Y, P, lat, precision, 2, True)
    assert math.isinf(b.nu[1])
    assert np.all(np.abs(tb - ta) <= 1e-9 * np.abs(ta))
    assert abs(tb[0] - ta[0]) <= 1e-12 * abs(ta[0])


def test_fused_fit_at_full_size_allocates_no_pair_buffers():
    """The p=8, r=4, g=6 workload at its full n = 10^6 (on a 1024-point
    lattice to keep the test short): the fused context's fit allocates no
    per-pair buffers (the unfused one holds 6e6 pairs x 68 bytes of E-step
    outputs and an 8-byte rescue slot per pair, about 456 MB), and one EM
    iteration agrees with the unfused path to summation order (at this n the
    order of the log-likelihood's 10^6 terms alone can move it by n eps)."""
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p8r4g6_n1000000_N8192", 1000000, 1024)
    Yd = torch.from_numpy(Y).cuda()
    torch.cuda.synchronize()
    out = {}
    for fused in (True, False):
        with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=1, fused=fused) as ctx:
            free0 = torch.cuda.mem_get_info()[0]
            ctx.cfust_fit_begin(Yd, init)
            torch.cuda.synchronize()
            drop = free0 - torch.cuda.mem_get_info()[0]
            ctx.cfust_fit_step(1)
            got, trace, done = ctx.cfust_fit_end()
        out[fused] = (drop, got, trace)
        print("fused" if fused else "unfused", "device memory taken by the fit", drop / 1e6, "MB")
    assert out[True][0] < 64e6, out[True][0]
    assert out[False][0] > 400e6, out[False][0]
    ta, tb = out[False][2], out[True][2]
    # the same 10^6 values l_j summed in another order (other block rows):
    # up to n eps = 1.1e-10 of the sum of |l_j| apart
    assert abs(tb[0] - ta[0]) <= 1.1e-10 * abs(ta[0])
    assert np.all(np.abs(tb - ta) <= 1e-9 * np.abs(ta))
    for name, e in parameter_errors(out[True][1].as_arrays(), out[False][1].as_arrays()).items():
        assert e <= 1e-9, f"{name}: {e:.3g}"


def test_fused_with_a_surrogate_is_refused():
    torch = _torch()
    Y, truth, init, lat = _problem("cfust_p3r3g4_n1000000_N2048", 100, 512)
    sur = binding.Surrogate(lat, seed=0)
    try:
        with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=1, fused=True) as ctx:
            ctx.cfust_set_surrogate(sur)
            with pytest.raises(binding.CfustError) as ei:
                ctx.cfust_fit(torch.from_numpy(Y).cuda(), init)
            assert ei.value.status == -1 and "fused" in str(ei.value)
    finally:
        sur.close()


def test_fused_option_is_validated():
    _torch()
    lat = synth.make_lattice(256, 4, 0)
    lib = binding.load()
    z = np.ascontiguousarray(lat.z, dtype=np.int64)
    sh = np.ascontiguousarray(lat.shift, dtype=np.float64)
    L = binding.cfust_lattice(int(lat.n), int(z.shape[0]), z.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                              sh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    o = binding.cfust_opts(binding.CFUST_FP32, L, 0, 0.0, 0.0, 1, 0.0, 1, 0, 0, 0, 0.0, 0, 0, 2)
    h = ctypes.c_void_p()
    assert lib.cfust_create(ctypes.byref(h), ctypes.byref(o), None) == -1
    assert b"fused" in lib.cfust_last_error(None)
