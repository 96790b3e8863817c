"""The library's single-precision normal tail and quantile (used by the FP32
lattice sweep) against scipy's double-precision functions and against CUDA's
own normcdff / normcdfinvf, through the C ABI."""
import numpy as np
import pytest
from scipy import special

from paper_2005_06848_gb300 import binding

pytestmark = pytest.mark.gpu

F32_TINY = float(np.finfo(np.float32).tiny)


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _eval(x, which):
    torch = _torch()
    xt = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    return binding.cfust_normal_f32(xt, which).cpu().numpy().astype(np.float64)


def test_upper_tail_accuracy():
    y = np.concatenate([np.linspace(-8, 8, 100001), np.linspace(8, 13, 5001)]).astype(np.float32)
    ref = special.ndtr(-y.astype(np.float64))
    own = _eval(y, 0)
    cuda = _eval(y, 2)
    rel = np.abs(own - ref) / ref
    assert rel.max() < 1e-6, rel.max()
    # agreement with CUDA's normcdff within both functions' error
    assert np.max(np.abs(own - cuda) / ref) < 2e-6


def test_quantile_accuracy():
    x = np.concatenate([np.logspace(np.log10(F32_TINY), -1, 100000), np.linspace(0.1, 0.9, 50001),
                        1 - np.logspace(-7, -1, 10000)]).astype(np.float32)
    ref = special.ndtri(x.astype(np.float64))
    own = _eval(x, 1)
    cuda = _eval(x, 3)
    big = np.abs(ref) > 1e-3
    assert np.max(np.abs(own[big] - ref[big]) / np.abs(ref[big])) < 1.5e-6
    assert np.max(np.abs(own[~big] - ref[~big])) < 1e-8
    assert np.max(np.abs(own[big] - cuda[big]) / np.abs(ref[big])) < 3e-6


def test_log_tail_and_log_quantile():
    y = np.concatenate([np.linspace(-5, 40, 20001), np.linspace(40, 2000, 2001)]).astype(np.float32)
    ref = special.log_ndtr(-y.astype(np.float64))
    own = _eval(y, 4)
    assert np.max(np.abs(own - ref) / np.maximum(np.abs(ref), 1.0)) < 1e-6
    la = -np.concatenate([np.logspace(-3, np.log10(700), 5000)]).astype(np.float32)
    ref_z = -special.ndtri(np.exp(la.astype(np.float64)))
    own_z = _eval(la, 5)
    # near z = 0 the float input la itself rounds at ~6e-8, so compare absolutely there
    assert np.max(np.abs(own_z - ref_z) / np.maximum(np.abs(ref_z), 0.5)) < 2e-6
    # beyond double range: z solves log Phi(-z) = la; check through the log tail
    la2 = -np.logspace(3, 5, 200).astype(np.float32)
    z2 = _eval(la2, 5)
    back = special.log_ndtr(-z2)
    assert np.max(np.abs(back - la2) / np.abs(la2)) < 1e-6
