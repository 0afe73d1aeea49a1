"""Per-level algorithmic flop counts of the batched Laplace workload (512 x 512 grid, leaves
16 x 16, eps 1e-10, a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2)), from a full oracle factorization.

Writes oracle/laplace_batched_level_flops.json.  The benchmark's CPU baseline times the oracle
on the finest levels only and scales the time by those levels' share of these counts.
Per box: CPQR 4rmk - 2k^2(r+m) + 4k^3/3, T k^2(m-k), F^{-1} 2m^3, W and E^{-1}
2m(m-k)k + 2k(m-k)k, E 2k^3; the root adds 2 m0^3 (counted at level 0).
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import oracle as O  # noqa: E402
from paper_1303_5466_gb300 import workloads as W  # noqa: E402


def level_flops(F):
    out = {}
    for l in range(1, F.depth + 1):
        s = 0.0
        for j in range(2 ** l):
            m, k, r, _ = F.sizes(l, j)
            s += (4.0 * r * m * k - 2.0 * k * k * (r + m) + 4.0 * k ** 3 / 3 + k * k * (m - k) + 2.0 * m ** 3
                  + 2.0 * m * (m - k) * k + 2.0 * k * (m - k) * k + 2.0 * k ** 3)
        out[l] = s
    m0 = F.root_inv().shape[0]
    out[0] = 2.0 * m0 ** 3
    return out


def main():
    cfg = W.WORKLOADS["laplace_batched"]
    n = cfg["n"]
    F = O.Factorization(n, cfg["leaf"], cfg["eps"], a=W.coeff_a_batched(n))
    fl = level_flops(F)
    path = os.path.join(HERE, "laplace_batched_level_flops.json")
    with open(path, "w") as fh:
        json.dump({str(k): v for k, v in sorted(fl.items())}, fh, indent=1)
    print(path, sum(fl.values()))


if __name__ == "__main__":
    main()
