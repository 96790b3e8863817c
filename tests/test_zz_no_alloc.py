"""The allocation-free M-step entry point (cfust_mstep_noalloc) against the
regular one (cfust_mstep), through the C ABI.

The entry point exists for callers that cannot allocate device memory on the
call path (an external memory manager that forbids cudaMalloc after start-up,
or a fixed device footprint): its scratch is a static device array.  Calls in
a row must each agree with cfust_mstep within the M-step parity tolerance.
The calls alternate between a large problem (g=16, p=16, r=6, where the
array's size caps the number of reduction blocks below what cfust_mstep uses,
so the partial sums are added in another order) and a small one, so what a
larger call leaves in the shared array would show up in the smaller call
after it.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2005_06848_gb300 import binding, synth

pytestmark = pytest.mark.gpu

NAMES = ("pi", "mu", "Sigma", "Delta", "nu")
# the M-step parity bars (same inputs, only the order of the partial sums differs)
RTOL = {binding.CFUST_FP64: 1e-10, binding.CFUST_FP32: 1e-9}


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _small_case(torch, precision):
    Y, _, truth, init, _, meta = synth.workload("cfust_p4r4g3_n100000_N4096", n=3000)
    lat = synth.make_lattice(1024, meta["r"] + 1, 0)
    return Y, init, lat


def _large_case(torch, precision):
    g, p, r, n = 16, 16, 6, 4096
    rng = np.random.default_rng(1234)
    P = synth.random_params(rng, g, p, r, 9.0, 2, 1.0, 3.0, 12.0)
    Y, _ = synth.sample_cfust(P, n, rng)
    lat = synth.make_lattice(256, r + 1, 3)
    return np.ascontiguousarray(Y), P, lat


def _inputs(torch, case, precision):
    Y, P, lat = case(torch, precision)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=precision) as ctx:
        E = ctx.cfust_estep(Yd, P)
        ref = ctx.cfust_mstep(Yd, E, P)
    return Yd, E, P, ref


def _check(got, ref, rtol, what):
    for name, a, b in zip(NAMES, got.as_arrays(), ref.as_arrays()):
        err = np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))
        assert err <= rtol, f"{what}: {name} differs by {err:.3g}"


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_noalloc_mstep_matches_mstep_on_calls_in_a_row(precision):
    torch = _torch()
    small = _inputs(torch, _small_case, precision)
    large = _inputs(torch, _large_case, precision)
    # the large problem really runs with fewer reduction blocks than cfust_mstep
    g, p, r, n = 16, 16, 6, 4096
    K = 3 + p + r + p * r + r * (r + 1) // 2 + p * (p + 1) // 2
    pbytes = 8 * g * (2 + p + p * p + p * r)
    cap = ((1 << 20) - 256 - ((pbytes + 255) // 256) * 256) // (8 * g * K)
    assert cap < (n + 63) // 64
    for call, (label, (Yd, E, P, ref)) in enumerate([("small", small), ("large", large), ("small", small),
                                                     ("large", large)]):
        got = binding.cfust_mstep_noalloc(precision, Yd, E, P)
        _check(got, ref, RTOL[precision], f"call {call} ({label})")


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    torch = _torch()
    g, p, r = 64, 16, 6      # parameters + 8 blocks of partial sums exceed the 1 MiB array
    rng = np.random.default_rng(0)
    P = synth.random_params(rng, g, p, r, 1.0, 2, 1.0, 3.0, 10.0)
    n = 64
    Yd = torch.zeros((n, p), dtype=torch.float64, device="cuda")
    rp = r * (r + 1) // 2
    E = dict(tau=torch.zeros((g, n), dtype=torch.float64, device="cuda"),
             e1=torch.zeros((g, n), dtype=torch.float64, device="cuda"),
             e2=torch.zeros((g, n), dtype=torch.float64, device="cuda"),
             e3=torch.zeros((g, r, n), dtype=torch.float64, device="cuda"),
             e4=torch.zeros((g, rp, n), dtype=torch.float64, device="cuda"))
    K = 3 + p + r + p * r + rp + p * (p + 1) // 2
    assert 8 * 8 * g * K + 256 + 8 * g * (2 + p + p * p + p * r) > 1 << 20
    with pytest.raises(binding.CfustError) as ei:
        binding.cfust_mstep_noalloc(binding.CFUST_FP64, Yd, E, P)
    assert ei.value.status == -1
    assert "CFUST_NOALLOC_SCRATCH_BYTES" in str(ei.value)


def test_noalloc_rejects_mismatched_tensors():
    """Element type, shape or device that do not match the call are refused
    before any kernel runs (the binding checks; the library checks the device)."""
    torch = _torch()
    Y, init, lat = _small_case(torch, binding.CFUST_FP32)
    Yd = torch.from_numpy(Y[:256]).cuda()
    g, r, n = init.g, init.r, 256
    E32 = dict(tau=torch.zeros((g, n), device="cuda"), e1=torch.zeros((g, n), device="cuda"),
               e2=torch.zeros((g, n), device="cuda"), e3=torch.zeros((g, r, n), device="cuda"),
               e4=torch.zeros((g, r * (r + 1) // 2, n), device="cuda"))
    with pytest.raises(ValueError):
        binding.cfust_mstep_noalloc(binding.CFUST_FP64, Yd, E32, init)   # float tensors, double mode
    bad = dict(E32, e3=torch.zeros((g, r, n - 1), device="cuda"))
    with pytest.raises(ValueError):
        binding.cfust_mstep_noalloc(binding.CFUST_FP32, Yd, bad, init)
    # host memory handed straight to the C entry point: refused by the library
    import ctypes
    lib = binding.load()
    hp = binding._HostParams(init)
    Yh = np.ascontiguousarray(Y[:256])
    rc = lib.cfust_mstep_noalloc(binding.CFUST_FP32, Yh.ctypes.data_as(ctypes.c_void_p), n,
                                 binding._ptr(E32["tau"]), binding._ptr(E32["e1"]), binding._ptr(E32["e2"]),
                                 binding._ptr(E32["e3"]), binding._ptr(E32["e4"]), 0.0, 0.0,
                                 ctypes.byref(hp.c), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == -1
    assert b"current device" in lib.cfust_last_error(None)
