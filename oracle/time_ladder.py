"""Wall-clock times of the dense CPU oracle (Eq. 1 by a dense FP64
Cholesky) on the first n points of the medium workload -- TEST
INFRASTRUCTURE: a measurement of the baseline, not part of the product.

    python -m oracle.time_ladder [--n 16384 32768 65536]

Prints one JSON line: per n the seconds of one evaluation (the Matern
matrix by the oracle's C code, then numpy's Cholesky and the forward
substitution), the host's core count and the matrix size in GB.
"""
from __future__ import annotations

import argparse
import json
import os
import time

import oracle
from paper_2104_07146_gb300 import synth


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, nargs="+", default=[16384, 32768, 65536])
    a = ap.parse_args()
    locs_all = synth.locations_blobs(65536, 2, 0.3, 8, 0.03, seed=1001)   # the benchmark's inputs
    z_all = synth.normal(1002, 65536)
    theta = (0.05, 0.5, 1.0, 1e-3)
    rows = []
    for n in a.n:
        t0 = time.time()
        ll, ld, q = oracle.loglik_dense(locs_all[:n], z_all[:n], theta)
        rows.append({"n": n, "s": time.time() - t0, "matrix_gb": 8.0 * n * n / 1e9, "loglik": ll})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"cores": os.cpu_count(), "rows": rows}))


if __name__ == "__main__":
    main()
