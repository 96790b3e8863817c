"""The split fit's host logic on CPU (the observation-sharded EM of
Algorithms 2 and 3: per-worker partial sums, one all-reduce, the same update
on every worker), with the FP64 oracle standing in for each worker's kernels.

Two checks: sums over row shards add up to the unsharded sums (so the update
from the totals is the unsharded update), and two gloo ranks running
paper_2005_06848_gb300.sharded.fit reproduce the one-process fit's
log-likelihood trace and parameters.
"""
import os
import socket

import numpy as np
import pytest

from oracle import cfust_oracle as O
from paper_2005_06848_gb300 import sharded, synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def pack_sums(S, p, r):
    """Oracle sums (list of dicts) -> [g][K] in the library's order: S1, S2,
    S3[p], S4[r], S5[p][r], S6 packed lower, S7 packed lower, S8."""
    rows = []
    for s in S:
        v = [s["S1"], s["S2"], *s["S3"], *s["S4"], *np.asarray(s["S5"]).ravel()]
        v += [s["S6"][t, h] for t in range(r) for h in range(t + 1)]
        v += [s["S7"][a, b] for a in range(p) for b in range(a + 1)]
        v.append(s["S8"])
        rows.append(v)
    return np.array(rows, dtype=np.float64)


def unpack_sums(M, p, r):
    out = []
    for v in np.asarray(M, dtype=np.float64):
        k = 0
        s = {"S1": v[0], "S2": v[1]}
        k = 2
        s["S3"] = v[k:k + p].copy(); k += p
        s["S4"] = v[k:k + r].copy(); k += r
        s["S5"] = v[k:k + p * r].reshape(p, r).copy(); k += p * r
        S6 = np.zeros((r, r))
        for t in range(r):
            for h in range(t + 1):
                S6[t, h] = S6[h, t] = v[k]; k += 1
        S7 = np.zeros((p, p))
        for a in range(p):
            for b in range(a + 1):
                S7[a, b] = S7[b, a] = v[k]; k += 1
        s["S6"], s["S7"], s["S8"] = S6, S7, v[k]
        out.append(s)
    return out


class OracleWorker:
    """The three calls of a worker, computed by the oracle (test stand-in for
    a binding.Context on one GPU)."""

    def __init__(self, lat):
        self.U = O.lattice_points(lat.n, lat.z, lat.shift)

    def cfust_estep(self, Y, params):
        return O.estep(Y, params, self.U)

    def cfust_mstep_sums(self, Y, E, params):
        return pack_sums(O.mstep_sums(Y, E["tau"], E["e1"], E["e2"], E["e3"], E["e4"]), params.p, params.r)

    def cfust_mstep_apply(self, sums, n_total, params):
        return O.mstep_update(unpack_sums(sums, params.p, params.r), params, n_total)


def _problem():
    Y, _, truth, init, _, meta = synth.workload("cfust_p2r2g2_n2000_N1024", n=240)
    lat = synth.make_lattice(256, meta["r"] + 1, 0)
    return Y, init, lat


def test_shard_rows_cover_every_row_once():
    for n, ws in [(10, 3), (7, 7), (100000, 8), (5, 8)]:
        got = [sharded.shard_rows(n, ws, k) for k in range(ws)]
        assert got[0][0] == 0 and got[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(got, got[1:]))
        sizes = [b - a for a, b in got]
        assert max(sizes) - min(sizes) <= 1


def test_shard_sums_add_up_to_the_unsharded_sums_and_update():
    Y, init, lat = _problem()
    w = OracleWorker(lat)
    full = w.cfust_mstep_sums(Y, w.cfust_estep(Y, init), init)
    tot = np.zeros_like(full)
    for k in range(3):
        j0, j1 = sharded.shard_rows(Y.shape[0], 3, k)
        tot += w.cfust_mstep_sums(Y[j0:j1], w.cfust_estep(Y[j0:j1], init), init)
    assert np.allclose(tot, full, rtol=1e-12, atol=1e-12 * np.abs(full).max())
    # the packing is a faithful round trip, and the update from the totals is the unsharded one
    S = O.mstep_sums(Y, *(w.cfust_estep(Y, init)[k] for k in ("tau", "e1", "e2", "e3", "e4")))
    assert np.array_equal(pack_sums(unpack_sums(full, init.p, init.r), init.p, init.r), full)
    a = O.mstep_update(S, init, Y.shape[0]).as_arrays()
    b = w.cfust_mstep_apply(tot, Y.shape[0], init).as_arrays()
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-10, atol=1e-12)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, iters, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    Y, init, lat = _problem()
    j0, j1 = sharded.shard_rows(Y.shape[0], ws, rank)
    params, trace = sharded.fit(OracleWorker(lat), Y[j0:j1], init, Y.shape[0], iters, sharded.torch_allreduce())
    out[rank] = ([a.tolist() for a in params.as_arrays()], trace.tolist())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_the_single_process_fit():
    iters = 3
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(2, port, iters, out), nprocs=2, start_method="spawn", join=True)
    Y, init, lat = _problem()
    U = O.lattice_points(lat.n, lat.z, lat.shift)
    ref, ref_trace = O.fit(Y, init, U, iters)
    for rank in (0, 1):
        params, trace = out[rank]
        assert np.allclose(trace, ref_trace[:iters], rtol=1e-12, atol=0)
        for a, b in zip(params, ref.as_arrays()):
            assert np.allclose(np.array(a), b, rtol=1e-9, atol=1e-12)
    # both ranks hold bit-identical parameters: the same update on the same totals
    assert out[0][0] == out[1][0]
