"""Writes large_rff_fold0.txt: the FP64 oracle's hold-out errors of fold 0 of
the large random-Fourier workload (n = 131072, d = 8192, c = 32, k = 5, g = 6,
r = 3, q = 101, Chebyshev basis in log lambda) at a few grid indices.

Calls only the oracle and the seeded generator; the GPU path is never run.
The oracle's Gram step alone is ~3.5e12 multiply-adds in plain loops, so the
values are computed once here and stored rather than recomputed in a test.

    python tests/golden/make_large_rff_golden.py      # ~10-20 min on 8 cores
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1404_0466_gb300 import synth  # noqa: E402

IDX = [0, 25, 50, 75, 100]
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "large_rff_fold0.txt")


def main():
    cfg = synth.LARGE_RFF
    t0 = time.time()
    prob = synth.large_rff()
    X = prob.X
    # fingerprint of the generated inputs, so a test can confirm it regenerated the same data
    rows = np.array([0, 1, 4095, 65536, 131071])
    fp = [float(np.sum(X[r].astype(np.float64))) for r in rows]
    ysum = float(np.sum(prob.Y.astype(np.float64)))
    ref = oracle.cv(X, prob.Y, k=cfg["k"], g=cfg["g"], r=cfg["r"], q=cfg["q"], lo=cfg["lo"], hi=cfg["hi"],
                    basis=oracle.BASIS_CHEB_LOG, folds=[0], lam_idx=IDX)
    el = time.time() - t0
    with open(OUT, "w") as fh:
        fh.write("# FP64 oracle (oracle.cv, plain loops): hold-out mean squared errors of fold 0 of the\n")
        fh.write("# large random-Fourier workload, piCholesky with the Chebyshev basis in log lambda\n")
        fh.write("# (Algorithm 1; hold-out error read as the mean squared error over held-out rows and\n")
        fh.write("# outputs, Sec. 3.1).  n=131072 d=8192 c=32 k=5 g=6 r=3 q=101, lambda in\n")
        fh.write("# [1e-3, 1e1] * tr(X^T X)/d, seed 2.  Written by make_large_rff_golden.py\n")
        fh.write(f"# ({el:.0f} s); the GPU path is never run to make it.\n")
        fh.write(f"tau {float(ref.tau)!r}\n")
        fh.write("fingerprint_rows " + " ".join(str(int(r)) for r in rows) + "\n")
        fh.write("fingerprint_sums " + " ".join(repr(v) for v in fp) + "\n")
        fh.write(f"y_sum {ysum!r}\n")
        fh.write("# index lambda E_fold0\n")
        for t in IDX:
            fh.write(f"{t} {float(ref.lam[t])!r} {float(ref.E[0, t])!r}\n")
    print(open(OUT).read())


if __name__ == "__main__":
    main()
