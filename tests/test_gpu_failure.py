"""Failure paths of the GPU kernels that need no GPU fault to exercise.

The lattice sweeps stage each component's chi tables with an asynchronous bulk
copy and wait for it on an mbarrier for a bounded number of polls.  A context
made with test_wait_polls = -1 gives that wait no polls at all, so every block
takes the give-up path: it lets its copy land, reports CFUST_ETIMEOUT and
returns.  Nothing faults or hangs; the same device keeps serving a normal
context afterwards, whose result is checked against the oracle.
"""
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


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_staging_wait_gives_up_with_etimeout_and_the_device_stays_usable(precision):
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p3r3g4_n1000000_N2048", n=600)
    lat = synth.make_lattice(256, meta["r"] + 1, 0)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=precision, max_iter=2, test_wait_polls=-1) as ctx:
        for call in (lambda: ctx.cfust_loglik(Yd, init), lambda: ctx.cfust_estep(Yd, init),
                     lambda: ctx.cfust_fit(Yd, init), lambda: ctx.cfust_fit_batched([Yd, Yd[:300]], [init, init])):
            with pytest.raises(binding.CfustError) as ei:
                call()
            assert ei.value.status == -5, str(ei.value)
            assert "bounded device wait" in str(ei.value)
    torch.cuda.synchronize()
    # a context with the default bound on the same device: correct results
    with binding.Context(lat, precision=precision) as ctx:
        got = ctx.cfust_loglik(Yd, init)
    ref = O.loglik(Y, init, O.lattice_points(lat.n, lat.z, lat.shift))
    tol = 1e-10 if precision == binding.CFUST_FP64 else 1e-6
    assert abs(got - ref) <= tol * abs(ref)


def test_wait_polls_option_is_validated():
    _torch()
    lat = synth.make_lattice(256, 4, 0)
    with pytest.raises(binding.CfustError) as ei:
        binding.Context(lat, precision=binding.CFUST_FP32, test_wait_polls=-2)
    assert ei.value.status == -1
    # a small positive bound is legal and still lets ordinary copies land
    Y, _, truth, init, _, meta = synth.workload("cfust_p3r3g4_n1000000_N2048", n=200)
    import torch
    with binding.Context(lat, precision=binding.CFUST_FP64, test_wait_polls=1 << 20) as ctx:
        got = ctx.cfust_loglik(torch.from_numpy(Y).cuda(), init)
    assert np.isfinite(got)


@pytest.mark.parametrize("precision", [binding.CFUST_FP64, binding.CFUST_FP32])
def test_fused_staging_wait_gives_up_with_etimeout(precision):
    """The fused E-step + sums kernel stages its components through the same
    bounded wait: with no polls allowed each CTA lets its copy land and
    returns, the call reports CFUST_ETIMEOUT, and a normal fused context on
    the same device then matches the oracle."""
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p3r3g4_n1000000_N2048", n=600)
    lat = synth.make_lattice(256, meta["r"] + 1, 0)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=precision, max_iter=2, test_wait_polls=-1, fused=True) as ctx:
        for call in (lambda: ctx.cfust_loglik(Yd, init), lambda: ctx.cfust_fit(Yd, init)):
            with pytest.raises(binding.CfustError) as ei:
                call()
            assert ei.value.status == -5, str(ei.value)
    torch.cuda.synchronize()
    with binding.Context(lat, precision=precision, fused=True) as ctx:
        got = ctx.cfust_loglik(Yd, init)
    ref = O.loglik(Y, init, O.lattice_points(lat.n, lat.z, lat.shift))
    tol = 1e-10 if precision == binding.CFUST_FP64 else 1e-6
    assert abs(got - ref) <= tol * abs(ref)
