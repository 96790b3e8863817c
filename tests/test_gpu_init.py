"""Initial values of Algorithm 1 on the GPU (k-means partitions, Psi^(0) of a
partition by moments, the multi-start fit from partitions) against the
oracle in oracle/init_oracle.py, through the C ABI.

Tolerances: labels are integers decided by double-precision distances that
both sides accumulate in the same order with the same roundings: bit-exact.
Centres and moment sums differ only in summation order: 1e-12 relative.
"""
import numpy as np
import pytest

from oracle import cfust_oracle as O
from oracle import init_oracle as IO
from paper_2005_06848_gb300 import binding, synth

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _data(n, seed=0, wl="cfust_p4r4g3_n100000_N4096"):
    Y, labels, truth, init, _, meta = synth.workload(wl, n=n, seed=seed)
    return Y, truth


def _close(name, got, ref, rtol=1e-12):
    got, ref = np.asarray(got), np.asarray(ref)
    scale = max(1.0, float(np.max(np.abs(ref))))
    err = float(np.max(np.abs(got - ref))) if ref.size else 0.0
    assert err <= rtol * scale, f"{name}: max abs error {err:.3g} (scale {scale:.3g})"


@pytest.mark.parametrize("n,seed", [(20000, 0), (257, 1), (1, 2)])
def test_kmeans_matches_oracle(n, seed):
    """Several tiles with a ragged one (20000 = 78 x 256 + 32), one tile plus
    one row, and a single observation."""
    torch = _torch()
    Y, truth = _data(max(n, 8), seed)
    Y = np.ascontiguousarray(Y[:n])
    g = min(truth.g, n)
    c0 = synth.initial_centres(Y, g, 1, seed)[0]
    ref_lab, ref_c, ref_it = IO.kmeans(Y, c0, 100)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(synth.make_lattice(64, truth.r + 1)) as ctx:
        lab, C, it = ctx.cfust_kmeans(Yd, c0, 100)
    assert it == ref_it
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    _close("centres", C, ref_c)


def test_kmeans_stops_at_max_iter():
    torch = _torch()
    Y, truth = _data(5000, 3)
    c0 = synth.initial_centres(Y, truth.g, 1, 3)[0]
    ref_lab, ref_c, ref_it = IO.kmeans(Y, c0, 2)
    with binding.Context(synth.make_lattice(64, truth.r + 1)) as ctx:
        lab, C, it = ctx.cfust_kmeans(torch.from_numpy(Y).cuda(), c0, 2)
    assert it == ref_it == 2
    assert np.array_equal(lab.cpu().numpy(), ref_lab)
    _close("centres", C, ref_c)


@pytest.mark.parametrize("lam,nu0", [(0.5, 10.0), (6.0, 4.0), (0.0, 30.0)])
def test_init_partition_matches_oracle(lam, nu0):
    """From a k-means partition and from a random one; lam = 6 forces the
    halving rule, lam = 0 gives Delta = 0."""
    torch = _torch()
    Y, truth = _data(30000, 4)
    g, r = truth.g, truth.r
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(synth.make_lattice(64, r + 1)) as ctx:
        lab_km, _, _ = ctx.cfust_kmeans(Yd, synth.initial_centres(Y, g, 1, 4)[0], 50)
        lab_rand = torch.from_numpy(synth.random_partitions(Y.shape[0], g, 1, 5)[0]).cuda()
        for lab in (lab_km, lab_rand):
            got = ctx.cfust_init_partition(Yd, lab, g, r, nu0=nu0, lam=lam)
            ref = IO.moment_init(Y, lab.cpu().numpy(), g, r, nu0=nu0, lam=lam)
            for name, a, b in zip(("pi", "mu", "Sigma", "Delta", "nu"), got.as_arrays(), ref[:5]):
                _close(name, a, b)


def test_init_partition_errors():
    torch = _torch()
    Y, truth = _data(600, 6)
    g, r, p = truth.g, truth.r, truth.p
    Yd = torch.from_numpy(Y).cuda()
    lab = np.zeros(Y.shape[0], dtype=np.int32)
    lab[:p] = 1                       # p members < p + 1
    with binding.Context(synth.make_lattice(64, r + 1)) as ctx:
        with pytest.raises(binding.CfustError) as e:
            ctx.cfust_init_partition(Yd, torch.from_numpy(lab).cuda(), 2, r)
        assert e.value.status == -4
        bad = lab.copy()
        bad[7] = g                    # outside 0..g-1
        with pytest.raises(binding.CfustError) as e:
            ctx.cfust_init_partition(Yd, torch.from_numpy(bad).cuda(), g, r)
        assert e.value.status == -1
        with pytest.raises(binding.CfustError) as e:
            ctx.cfust_init_partition(Yd, torch.from_numpy(lab).cuda(), 2, r, nu0=2.0)
        assert e.value.status == -1
        # the context stays usable after the errors
        good = torch.from_numpy(synth.random_partitions(Y.shape[0], g, 1, 0)[0]).cuda()
        ctx.cfust_init_partition(Yd, good, g, r)


def test_multistart_from_partitions():
    """Algorithm 1 end to end: partitions (two k-means, two random) -> Psi^(0)
    by moments -> burn-in -> best start -> fit.  Bitwise equal to
    cfust_init_partition followed by cfust_fit_multistart (whose choice is
    pinned against the oracle in test_gpu_batched); with no burn-in the
    choice is the oracle's own largest l^(0) at the oracle's Psi^(0)."""
    torch = _torch()
    Y, truth = _data(3000, 7)
    g, r = truth.g, truth.r
    lat = synth.make_lattice(1024, r + 1)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=binding.CFUST_FP32, max_iter=5) as ctx:
        labs = [ctx.cfust_kmeans(Yd, c, 50)[0].cpu().numpy() for c in synth.initial_centres(Y, g, 2, 8)]
        labs += list(synth.random_partitions(Y.shape[0], g, 2, 9))
        L = torch.from_numpy(np.stack(labs).astype(np.int32)).cuda()
        best, P, trace, done, starts = ctx.cfust_multistart_partitions(Yd, L, g, r, nu0=10.0, lam=0.5, burn_in=2)
        gpu_inits = [ctx.cfust_init_partition(Yd, L[f], g, r, nu0=10.0, lam=0.5) for f in range(len(labs))]
        best2, P2, trace2, done2, _ = ctx.cfust_fit_multistart(Yd, gpu_inits, burn_in=2)
    assert best == best2
    assert done == done2
    assert np.array_equal(trace, trace2)
    for a, b in zip(P.as_arrays(), P2.as_arrays()):
        assert np.array_equal(a, b)

    inits = []
    for lab in labs:
        pi, mu, Sigma, Delta, nu, _ = IO.moment_init(Y, lab, g, r, nu0=10.0, lam=0.5)
        inits.append(synth.Params(pi, mu, Sigma, Delta, nu))

    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ll0 = [O.loglik(Y, p0, U) for p0 in inits]
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=1) as ctx:
        best0, _, _, _, starts0 = ctx.cfust_multistart_partitions(Yd, L, g, r, nu0=10.0, lam=0.5, burn_in=0)
    # k-means from different centres can reach the same partition: equal
    # l^(0), and both sides then take the first of the tied starts
    top = max(ll0)
    ties = [f for f, v in enumerate(ll0) if v >= top - 1e-9 * abs(top)]
    assert best0 == ties[0] == O.select_start(ll0), (best0, ll0)
