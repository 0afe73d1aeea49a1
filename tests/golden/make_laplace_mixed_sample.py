"""Writes tests/golden/laplace_mixed_1024_oracle_sample.txt: sampled entries of the oracle's
FP64 solution of the 1024 x 1024 Laplace problem of the mixed-precision workload.

Problem: the Nystrom discretization of a(x) sigma + int K(x, y) sigma(y) dy = f on [0,1]^2
(Sec. 5, general formulation) with K = -(1/2 pi) log|x - y|, a = 1, a 1024 x 1024 cell-centre
grid, leaves of 16 x 16 points, f ~ U[-1, 1] from seed 2.  The oracle factors it at eps = 1e-10
(Algorithm 1 with the E of Algorithm 2) and applies the inverse (Algorithm 6); this script
calls only the oracle.  It stores, for 2048 rows drawn with default_rng(2) (without
replacement), the row index, the oracle's solution there and the true residual (f - A x) there,
computed entry by entry over all N columns.  One run takes about half an hour on 8 host cores
and some 20 GB of host memory.

    python tests/golden/make_laplace_mixed_sample.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1303_5466_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(HERE, "laplace_mixed_1024_oracle_sample.txt")
ROWS = 2048


def main():
    cfg = W.WORKLOADS["laplace_mixed"]
    n, leaf, seed = cfg["n"], cfg["leaf"], cfg["seed"]
    f = W.rhs_uniform(n, seed)
    t0 = time.time()
    F = O.Factorization(n, leaf, 1e-10)
    t1 = time.time()
    x = F.solve(f)
    rows = np.sort(np.random.default_rng(seed).choice(n * n, ROWS, replace=False))
    r = f[rows] - O.matvec_rows(n, x, rows)
    rel = float(np.linalg.norm(r) / np.linalg.norm(f[rows]))
    with open(OUT, "w") as fh:
        fh.write("# Oracle FP64 solution of the 1024 x 1024 Laplace problem (a = 1, leaves 16 x 16,\n")
        fh.write("# f ~ U[-1,1] seed 2) at eps 1e-10: Algorithm 1 (E of Algorithm 2) and the inverse\n")
        fh.write("# apply of Algorithm 6; written by tests/golden/make_laplace_mixed_sample.py from the\n")
        fh.write("# oracle only.  %d rows drawn by default_rng(2).choice(N, %d, replace=False), sorted.\n"
                 % (ROWS, ROWS))
        fh.write("# oracle factor %.0f s; relative residual |f - A x| / |f| over these rows: %.3e\n"
                 % (t1 - t0, rel))
        fh.write("# columns: row  x_oracle(row)  (f - A x_oracle)(row)\n")
        for i, g in enumerate(rows):
            fh.write("%d %.17g %.17g\n" % (g, x[g], r[i]))
    print(OUT, "residual over the sample %.3e, factor %.0f s" % (rel, t1 - t0))


if __name__ == "__main__":
    main()
