"""One EM fit whose observations are split over several workers (processes,
one GPU each): the M-step's single exchange point.

Algorithm 2 of the paper gives every worker a block of observations and has
it return partial sums; Algorithm 3's master adds them and updates the
parameters (Sections 3.2 and 3.3).  Here every worker runs the E-step on its
own rows and the eight per-component sums over them (cfust_estep,
cfust_mstep_sums), the workers add one vector of g K + 1 doubles (the sums
and the rows' log-likelihood) with an all-reduce, and every worker applies
the same update to the totals (cfust_mstep_apply), so all hold the same
parameters without any per-pair data crossing between them.

Host logic only: the arithmetic runs in the library's kernels, the exchange
in whatever collective the caller passes (torch.distributed over NCCL on GPUs).
"""
from __future__ import annotations

import numpy as np


def shard_rows(n_total: int, world_size: int, rank: int) -> tuple[int, int]:
    """Contiguous row range [j0, j1) of `rank`: the first n_total % world_size
    ranks take one row more."""
    base, extra = divmod(int(n_total), int(world_size))
    j0 = rank * base + min(rank, extra)
    return j0, j0 + base + (1 if rank < extra else 0)


def em_iteration(worker, Y_local, params, n_total: int, allreduce):
    """One EM iteration of the split fit on this worker.

    worker: an object with cfust_estep(Y, params) -> dict(tau, e1..e4, loglik),
    cfust_mstep_sums(Y, E, params) -> [g][K] and
    cfust_mstep_apply(sums, n_total, params) -> params (a binding.Context).
    allreduce: sums a float64 numpy vector over all workers and returns it.
    Returns (updated params, l(params) over all rows): the E-step at the given
    parameters yields their log-likelihood, as in the single-worker fit.
    """
    E = worker.cfust_estep(Y_local, params)
    sums = np.asarray(worker.cfust_mstep_sums(Y_local, E, params), dtype=np.float64)
    vec = np.concatenate([sums.ravel(), [float(E["loglik"])]])
    tot = np.asarray(allreduce(vec), dtype=np.float64)
    new = worker.cfust_mstep_apply(tot[:-1].reshape(sums.shape), n_total, params)
    return new, float(tot[-1])


def fit(worker, Y_local, params, n_total: int, iters: int, allreduce):
    """`iters` EM iterations of the split fit; returns (params, trace) with
    trace = l(Psi^(0)) .. l(Psi^(iters-1)), the log-likelihood of the
    parameters each E-step started from."""
    trace = []
    for _ in range(int(iters)):
        params, ll = em_iteration(worker, Y_local, params, n_total, allreduce)
        trace.append(ll)
    return params, np.array(trace)


def torch_allreduce(device=None):
    """An allreduce over the default torch.distributed process group (the
    vector travels as a float64 tensor on `device`: a CUDA device for NCCL,
    the CPU for gloo)."""
    import torch
    import torch.distributed as dist

    def red(vec):
        t = torch.from_numpy(np.ascontiguousarray(vec, dtype=np.float64))
        if device is not None:
            t = t.to(device)
        dist.all_reduce(t)
        return t.cpu().numpy()
    return red
