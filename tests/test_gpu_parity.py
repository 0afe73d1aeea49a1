"""CUDA path vs the CPU oracle, element by element, through the C ABI (FP64, eps = 1e-10).

Integer results (ranks, skeleton sets, index lists) must be identical; floating-point blocks
and solutions must agree within the tolerances below.  The solution tolerance is the 1e-9
relative l2 bound of the FP64 path.  Block tolerances follow from the conditioning:
  - T = R11^{-1} R12 with |R_kk| / |R_11| ~ eps, so rounding differences in R reach T
    amplified by up to 1/eps: tolerance 100 u / eps (u = 1e-16), 1e-4 at eps = 1e-10;
  - F^{-1} of a leaf involves no T (F ~ I + O(h^2 log h)): 1e-11;
  - E = (R F^{-1} L)^{-1} carries T's differences times |F^{-1}_rs| << 1, and F^{-1} above
    the leaves and the root inverse carry those of the children's E (cond(F) ~ 1):
    tolerance 1e-6 (observed up to ~2e-7 at eps = 1e-10).
"""
import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-9


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    P.lib()
    return P


def _both(rs, oracle_mod, n, leaf, eps, a=None, order=None):
    F = oracle_mod.Factorization(n, leaf, eps, a=a)
    pts = W.grid_points(n)
    if order is not None:
        pts = pts[order]
        a = None if a is None else a[order]
    S = rs.Solver(pts, leaf, a=a, eps=eps)
    return F, S


def _rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


CASES = [(16, 4, 1e-10), (32, 8, 1e-10), (64, 8, 1e-10), (32, 8, 1e-5), (64, 16, 1e-10), (8, 2, 0.0)]


@pytest.mark.parametrize("n,leaf,eps", CASES)
def test_ranks_skeletons_and_index_lists_match(rs, oracle_mod, n, leaf, eps):
    F, S = _both(rs, oracle_mod, n, leaf, eps)
    mism = []
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            m, k, r, nn = F.sizes(l, j)
            assert rs.rs_op_box_sizes(S.op, l, j) == (m, k, r, nn), (l, j)
            np.testing.assert_array_equal(rs.rs_op_box_indices(S.op, l, j, 0), F.active(l, j))
            np.testing.assert_array_equal(rs.rs_op_box_indices(S.op, l, j, 1), F.near(l, j))
            if not np.array_equal(rs.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j)):
                mism.append((l, j))
    assert not mism, "skeleton sets differ at %s" % mism


@pytest.mark.parametrize("n,leaf,eps", CASES[:4])
def test_factor_blocks_match(rs, oracle_mod, n, leaf, eps):
    F, S = _both(rs, oracle_mod, n, leaf, eps)
    ttol = max(1e-10, 1e-16 / max(eps, 1e-16)) * 10 * 10
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            T = rs.rs_op_box_matrix(S.op, l, j, 0)
            if T.size:
                assert _rel(T, F.T(l, j)) <= ttol, ("T", l, j)
            ftol = 1e-11 if l == F.depth else 1e-6
            assert _rel(rs.rs_op_box_matrix(S.op, l, j, 1), F.Finv(l, j)) <= ftol, ("Finv", l, j)
            assert _rel(rs.rs_op_box_matrix(S.op, l, j, 2), F.E(l, j)) <= 1e-6, ("E", l, j)
    assert _rel(rs.rs_op_root_matrix(S.op), F.root_inv()) <= 1e-6


@pytest.mark.parametrize("n,leaf,eps", CASES)
def test_solve_matches_oracle(rs, oracle_mod, n, leaf, eps):
    F, S = _both(rs, oracle_mod, n, leaf, eps)
    f = W.rhs_uniform(n, 0)
    x = S.solve(f)
    xo = F.solve(f)
    assert _rel(x, xo) <= SOL_TOL
    if eps > 0:
        res = _rel(oracle_mod.matvec(n, x), f)
        assert res <= max(10 * eps, 1e-13)


def test_config_small_laplace_multi_rhs_device(rs, oracle_mod):
    """64 x 64 grid, leaves 8 x 8, eps 1e-10 (the small Laplace workload), 4 RHS on device."""
    import torch
    n, leaf, eps = 64, 8, 1e-10
    F, S = _both(rs, oracle_mod, n, leaf, eps)
    f = W.rhs_normal(n, 1, nrhs=4)                       # (N, 4)
    ft = torch.from_numpy(np.ascontiguousarray(f.T)).cuda()   # (4, N) = N x 4 column-major
    xt = S.solve(ft)
    torch.cuda.synchronize()
    x = xt.cpu().numpy().T
    xo = F.solve(f)
    for c in range(4):
        assert _rel(x[:, c], xo[:, c]) <= SOL_TOL
    # the host path gives the same bits
    xh = S.solve(f)
    np.testing.assert_array_equal(xh, x)


def test_varying_a_and_shuffled_points(rs, oracle_mod):
    """a(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2), points given in a shuffled order."""
    n, leaf, eps = 32, 8, 1e-10
    a = W.coeff_a_batched(n)
    order = W.shuffled(n, 9)
    F, S = _both(rs, oracle_mod, n, leaf, eps, a=a, order=order)
    f = W.rhs_uniform(n, 3)
    xo = F.solve(f)
    x = S.solve(f[order])
    assert _rel(x, xo[order]) <= SOL_TOL


def test_solve_rejects_bad_arguments(rs):
    import torch
    n = 16
    S = rs.Solver(W.grid_points(n), 4)
    f = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    xh = np.zeros(n * n)
    with pytest.raises(rs.RsError) as e:
        rs.rs_solve(S.op, f, 1, xh)           # device f, host x
    assert e.value.code == rs.RS_E_INVALID
    with pytest.raises(rs.RsError):
        rs.rs_solve(S.op, f, 0, f)
