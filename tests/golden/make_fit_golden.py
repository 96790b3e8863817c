"""Write tests/golden/fit_*.json: FP64 oracle EM fits used as expected values.

Calls only oracle/ and the seeded input module; run from the repository root:
    python tests/golden/make_fit_golden.py [--jobs K] [substring of a golden file name ...]
(no name writes every case).  With --jobs K each E-step's per-component
sweeps run on K spawned processes over blocks of rows (every row's result is
its own, so the blocks change nothing); the posterior, log-likelihood,
sums and update then run on all rows as in the oracle's own fit.  The
p=4, r=4, g=3 case at 5000 rows and the bench's 4096-point lattice takes
about 45 minutes on one core.
Each file records the workload, a fingerprint of the generated Y (its first
rows and column sums, so a test can tell if the input generator drifted beyond
last-bit differences between machines), the final parameters and the
log-likelihood trace l(Psi^(0)) .. l(Psi^(iters)).
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cfust_oracle as O  # noqa: E402
from paper_2005_06848_gb300 import synth  # noqa: E402

CASES = [
    # (workload, n, lattice points, iterations)
    # a 5000-row subsample of the p=4, r=4, g=3, n=100000 workload on the
    # bench's own 4096-point lattice, 50 iterations: the single-precision
    # parameter bar (1e-3 relative after 50 iterations) at the bench's rule
    ("cfust_p4r4g3_n100000_N4096", 5000, 4096, 50),
    ("cfust_p4r4g3_n100000_N4096", 1500, 1024, 50),
    ("cfust_p2r2g2_n2000_N1024", 2000, 1024, 20),
]


def _component_block(args):
    """One spawned worker: oracle E-step of component i over rows [j0, j1)."""
    Y, mu, Sigma, Delta, nu, U, j0, j1, density_only = args
    return O.estep_component(Y[j0:j1], mu, Sigma, Delta, nu, U, density_only=density_only)


def fit_parallel(Y, params0, U, iters, pool, jobs):
    """The oracle's fit (O.fit) with each E-step's sweeps spread over the pool."""
    n = Y.shape[0]
    edges = [n * k // jobs for k in range(jobs + 1)]

    def estep(P, density_only=False):
        logf, parts = [], []
        for i in range(P.g):
            blocks = pool.map(_component_block, [(Y, P.mu[i], P.Sigma[i], P.Delta[i], P.nu[i], U,
                                                  edges[k], edges[k + 1], density_only) for k in range(jobs)
                                                 if edges[k + 1] > edges[k]])
            parts.append({k: np.concatenate([b[k] for b in blocks]) for k in blocks[0]})
        logf = np.stack([c["logf"] for c in parts])
        tau, ll, _ = O.posterior(logf, P.pi)
        return parts, tau, ll

    params, trace = params0.copy(), []
    for _ in range(iters):
        parts, tau, ll = estep(params)
        trace.append(ll)
        e = {k: np.stack([c[k] for c in parts]) for k in ("e1", "e2", "e3", "e4")}
        sums = O.mstep_sums(Y, tau, e["e1"], e["e2"], e["e3"], e["e4"])
        params = O.mstep_update(sums, params, n)
    trace.append(estep(params, density_only=True)[2])
    return params, np.array(trace)


def golden_name(workload, n, N, iters):
    return f"fit_{workload.split('_n')[0]}_n{n}_N{N}_it{iters}.json"


def main(selected=(), jobs=1):
    pool = None
    if jobs > 1:
        import multiprocessing as mp
        pool = mp.get_context("spawn").Pool(jobs)
    for wl, n, N, iters in CASES:
        if selected and not any(k in golden_name(wl, n, N, iters) for k in selected):
            continue
        Y, _, truth, init, _, meta = synth.workload(wl, n=n)
        lat = synth.make_lattice(N, meta["r"] + 1, 0)
        U = O.lattice_points(lat.n, lat.z, lat.shift)
        t0 = time.time()
        if pool is None:
            params, trace = O.fit(Y, init, U, iters)
        else:
            params, trace = fit_parallel(Y, init, U, iters, pool, jobs)
        out = dict(workload=wl, n=n, lattice_n=N, lattice_seed=0, iters=iters,
                   y_head=Y[:4].tolist(), y_colsum=Y.sum(axis=0).tolist(),
                   params={k: v.tolist() for k, v in zip(("pi", "mu", "Sigma", "Delta", "nu"),
                                                        params.as_arrays())},
                   trace=trace.tolist(), oracle_seconds=round(time.time() - t0, 1))
        path = os.path.join(HERE, golden_name(wl, n, N, iters))
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(path, out["oracle_seconds"], "s")


if __name__ == "__main__":
    argv = sys.argv[1:]
    jobs = 1
    if argv[:1] == ["--jobs"]:
        jobs, argv = int(argv[1]), argv[2:]
    main(tuple(argv), jobs)
