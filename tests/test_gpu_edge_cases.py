"""Edge cases of the factor + solve path against the oracle.

- the smallest trees: one point per leaf (n = 2 and 4), where no box compresses (k = m at
  every level: Eq. 2.1 keeps every column) and the root holds every point;
- full rank at a tolerance of zero on a non-trivial tree (eps = 0: no truncation, so the
  factorization is exact and the solve reproduces the dense LU solution);
- ragged right-hand-side counts (1, 7, 9, 13, 65: the inverse apply takes them in compile-time
  chunks of up to 8, so every chunk length and a count above 64 run), on the device;
- a grid given in a shuffled input order with several right-hand sides;
- a solve whose input is all zeros (x must be exactly zero).
"""
import numpy as np
import pytest

import _dense as D
from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu
SOL_TOL = 1e-9


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    return P


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


@pytest.mark.parametrize("n,leaf", [(2, 1), (4, 1), (4, 2)])
def test_smallest_trees(rs, oracle_mod, n, leaf):
    F = oracle_mod.Factorization(n, leaf, 1e-10)
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10)
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S.op, l, j) == F.sizes(l, j), (l, j)
            np.testing.assert_array_equal(rs.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j))
    f = W.rhs_uniform(n, 4)
    assert _rel(S.solve(f), F.solve(f)) <= SOL_TOL
    assert _rel(S.solve(f), np.linalg.solve(D.laplace(n), f)) <= 1e-12


def test_eps_zero_is_exact(rs):
    n, leaf = 32, 8
    S = rs.Solver(W.grid_points(n), leaf, eps=0.0)
    f = W.rhs_normal(n, 8, nrhs=2)
    x = S.solve(f)
    A = D.laplace(n)
    xd = np.linalg.solve(A, f)
    for c in range(2):
        assert _rel(x[:, c], xd[:, c]) <= 1e-12


@pytest.mark.parametrize("nrhs", [1, 7, 9, 13, 65])
def test_ragged_rhs_counts_on_device(rs, oracle_mod, nrhs):
    import torch
    n, leaf, eps = 32, 8, 1e-10
    F = oracle_mod.Factorization(n, leaf, eps)
    S = rs.Solver(W.grid_points(n), leaf, eps=eps)
    f = W.rhs_normal(n, 20 + nrhs, nrhs=nrhs)
    fd = torch.from_numpy(np.ascontiguousarray(f.T)).cuda()
    xd = torch.full_like(fd, np.nan)
    rs.rs_solve(S.op, fd, nrhs, xd, torch.cuda.current_stream())
    torch.cuda.synchronize()
    x = xd.cpu().numpy().T.reshape(n * n, nrhs)
    xo = F.solve(f).reshape(n * n, nrhs)
    for c in range(nrhs):
        assert _rel(x[:, c], xo[:, c]) <= SOL_TOL, c


def test_shuffled_order_multi_rhs(rs, oracle_mod):
    n, leaf, eps = 64, 16, 1e-10
    order = W.shuffled(n, 31)
    F = oracle_mod.Factorization(n, leaf, eps)
    S = rs.Solver(W.grid_points(n)[order], leaf, eps=eps)
    f = W.rhs_normal(n, 32, nrhs=3)
    xo = F.solve(f)
    x = S.solve(np.ascontiguousarray(f[order]))
    assert _rel(x, xo[order]) <= SOL_TOL


def test_zero_rhs_gives_zero(rs):
    S = rs.Solver(W.grid_points(32), 8, eps=1e-10)
    x = S.solve(np.zeros(32 * 32))
    assert np.all(x == 0.0)
