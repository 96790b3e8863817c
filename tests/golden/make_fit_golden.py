"""Write tests/golden/fit_*.json: FP64 oracle EM fits used as expected values.

Calls only oracle/ and the seeded input module; run from the repository root:
    python tests/golden/make_fit_golden.py
Each file records the workload, a fingerprint of the generated Y (its first
rows and column sums, so a test can tell if the input generator drifted beyond
last-bit differences between machines), the final parameters and the
log-likelihood trace l(Psi^(0)) .. l(Psi^(iters)).
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import cfust_oracle as O  # noqa: E402
from paper_2005_06848_gb300 import synth  # noqa: E402

CASES = [
    # (workload, n, lattice points, iterations)
    ("cfust_p4r4g3_n100000_N4096", 1500, 1024, 50),
    ("cfust_p2r2g2_n2000_N1024", 2000, 1024, 20),
]


def golden_name(workload, n, N, iters):
    return f"fit_{workload.split('_n')[0]}_n{n}_N{N}_it{iters}.json"


def main():
    for wl, n, N, iters in CASES:
        Y, _, truth, init, _, meta = synth.workload(wl, n=n)
        lat = synth.make_lattice(N, meta["r"] + 1, 0)
        U = O.lattice_points(lat.n, lat.z, lat.shift)
        t0 = time.time()
        params, trace = O.fit(Y, init, U, iters)
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
    main()
