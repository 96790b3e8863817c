"""The M-step split at its exchange point on the GPU (cfust_mstep_sums /
cfust_mstep_apply, Algorithm 2's partial sums and Algorithm 3's combine):
the sums of k row shards, added on the host, equal the unsharded sums to
double rounding; the update from the totals equals cfust_mstep's; and a fit
driven shard by shard (paper_2005_06848_gb300.sharded, one process standing
in for the workers) reproduces the unsharded fit and the oracle."""
import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import binding, sharded, synth

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

NAMES = ("pi", "mu", "Sigma", "Delta", "nu")


def _torch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("precision,rtol", [(binding.CFUST_FP64, 1e-10), (binding.CFUST_FP32, 1e-9)])
def test_shard_sums_add_up_and_apply_equals_mstep(precision, rtol):
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p4r4g3_n100000_N4096", n=5003)
    lat = synth.make_lattice(512, meta["r"] + 1, 0)
    Yd = torch.from_numpy(Y).cuda()
    with binding.Context(lat, precision=precision) as ctx:
        E = ctx.cfust_estep(Yd, init)
        full = ctx.cfust_mstep_sums(Yd, E, init)
        ref = ctx.cfust_mstep(Yd, E, init)
        tot = np.zeros_like(full)
        for k in range(3):
            j0, j1 = sharded.shard_rows(Y.shape[0], 3, k)
            Ek = ctx.cfust_estep(Yd[j0:j1].contiguous(), init)
            # the shard's E-step is the unsharded E-step's rows, bit for bit
            for key in ("tau", "e1", "e2", "e3", "e4"):
                assert torch.equal(Ek[key], E[key][..., j0:j1]), key
            tot += ctx.cfust_mstep_sums(Yd[j0:j1].contiguous(), Ek, init)
        got = ctx.cfust_mstep_apply(tot, Y.shape[0], init)
    scale = np.maximum(1.0, np.abs(full))
    assert np.max(np.abs(tot - full) / scale) <= 1e-12
    for name, a, b in zip(NAMES, got.as_arrays(), ref.as_arrays()):
        err = np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b)))
        assert err <= rtol, f"{name}: {err:.3g}"
    # the sums themselves against the oracle's (FP64 mode: same E-step inputs)
    if precision == binding.CFUST_FP64:
        from test_sharded import pack_sums
        Eh = {k: E[k].cpu().numpy() for k in ("tau", "e1", "e2")}
        e3 = np.transpose(E["e3"].cpu().numpy(), (0, 2, 1))
        e4 = binding.unpack_e4(E["e4"].cpu().numpy(), init.r)
        S = pack_sums(O.mstep_sums(Y, Eh["tau"], Eh["e1"], Eh["e2"], e3, e4), init.p, init.r)
        assert np.max(np.abs(S - full) / np.maximum(1.0, np.abs(S))) <= 1e-11


def test_split_fit_reproduces_the_fit():
    """Three workers' shards advanced together for three EM iterations (one
    process, the all-reduce a plain sum over the shards) against cfust_fit on
    all rows and the oracle's fit (FP64 mode)."""
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p2r2g2_n2000_N1024", n=900)
    lat = synth.make_lattice(1024, meta["r"] + 1, 0)
    Yd = torch.from_numpy(Y).cuda()
    n, k, iters = Y.shape[0], 3, 3
    shards = [Yd[slice(*sharded.shard_rows(n, k, w))].contiguous() for w in range(k)]
    with binding.Context(lat, precision=binding.CFUST_FP64, max_iter=iters) as ctx:
        P, trace = init, []
        for _ in range(iters):
            parts = [(ctx.cfust_estep(S, P), S) for S in shards]
            vecs = [np.concatenate([ctx.cfust_mstep_sums(S, E, P).ravel(), [E["loglik"]]]) for E, S in parts]
            tot = np.sum(vecs, axis=0)
            P = ctx.cfust_mstep_apply(tot[:-1].reshape(P.g, -1), n, P)
            trace.append(tot[-1])
        ref, ref_trace, done = ctx.cfust_fit(Yd, init)
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    orc, orc_trace = O.fit(Y, init, U, iters)
    assert np.allclose(trace, ref_trace[:iters], rtol=1e-12, atol=0)
    assert np.allclose(trace, orc_trace[:iters], rtol=1e-10, atol=0)
    for name, a, b, c in zip(NAMES, P.as_arrays(), ref.as_arrays(), orc.as_arrays()):
        assert np.max(np.abs(a - b) / np.maximum(1.0, np.abs(b))) <= 1e-10, name
        assert np.max(np.abs(a - c) / np.maximum(1.0, np.abs(c))) <= 1e-8, name


def test_apply_rejects_bad_sums():
    torch = _torch()
    Y, _, truth, init, _, meta = synth.workload("cfust_p2r2g2_n2000_N1024", n=100)
    lat = synth.make_lattice(256, meta["r"] + 1, 0)
    with binding.Context(lat, precision=binding.CFUST_FP64) as ctx:
        bad = np.zeros((init.g, binding.sums_width(init.p, init.r)))
        bad[0, 0] = np.nan
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_mstep_apply(bad, 100, init)
        assert ei.value.status == -3
        with pytest.raises(binding.CfustError) as ei:
            ctx.cfust_mstep_apply(np.ones((init.g, binding.sums_width(init.p, init.r))), 0, init)
        assert ei.value.status == -1
