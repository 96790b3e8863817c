"""The allocation-free M-step entry point (cfust_mstep_noalloc) against the
regular one (cfust_mstep), through the C ABI.

The entry point exists for callers that cannot allocate device memory on the
call path (an external memory manager that forbids cudaMalloc after start-up,
or a fixed device footprint): its scratch is a static device array.  Two calls
in a row must both agree with cfust_mstep within the M-step parity tolerance,
which also shows that what the first call leaves in the shared array does not
leak into the second.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2005_06848_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision,rtol", [(binding.CFUST_FP64, 1e-10), (binding.CFUST_FP32, 1e-10)])
def test_noalloc_mstep_matches_mstep_twice(precision, rtol):
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p4r4g3_n100000_N4096", n=3000)
    lat = synth.make_lattice(1024, meta["r"] + 1, 0)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=precision) as ctx:
        E = ctx.cfust_estep(Yd, init)
        ref = ctx.cfust_mstep(Yd, E, init)
    names = ("pi", "mu", "Sigma", "Delta", "nu")
    for call in range(2):
        got = binding.cfust_mstep_noalloc(precision, Yd, E, init)
        for name, a, b in zip(names, got.as_arrays(), ref.as_arrays()):
            err = np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))
            assert err <= rtol, f"call {call}: {name} differs by {err:.3g}"


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
