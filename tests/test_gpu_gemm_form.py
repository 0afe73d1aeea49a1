"""The products forming E in Algorithm 1 (W = Phi_{:,r} T^T + Phi_{:,s}, E^{-1} = T W_r + W_s) of
FP64 operators, in the two forms of opts.gemm_form: FP64 FMA tiles (0) and exact products of
7-bit digit slices on the bf16 tensor cores (1, the default).  The digit form rounds each entry
once and leaves out only the parts below 2^-56 of the row and column maxima, so both forms agree
to rounding: identical ranks and skeletons, E blocks of every level within 1e-10 of each other
(E is the inverse of the product, which amplifies rounding differences by its condition
number), solutions within 1e-12 of each other and within the 1e-9 FP64 bound of the oracle.
The grids span several 64 x 32 tiles of C, ragged edges in M, N and K, K beyond one exact
128-digit chunk, the lower-triangle launch of the symmetric sweep, and Gauss-Jordan (which
takes every tile)."""
import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    P.lib()
    return P


def _opts(rs, form, spd=1):
    o = rs.rs_opts_default()
    o.gemm_form = form
    o.spd_inverse = spd
    return o


def _rel(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300))


@pytest.mark.parametrize("n,leaf,spd", [(64, 8, 1), (128, 16, 1), (64, 16, 0)])
def test_digit_products_match_fp64_tiles(rs, oracle_mod, n, leaf, spd):
    a = W.coeff_a_batched(n)
    S0 = rs.Solver(W.grid_points(n), leaf, a=a, eps=1e-10, opts=_opts(rs, 0, spd))
    S1 = rs.Solver(W.grid_points(n), leaf, a=a, eps=1e-10, opts=_opts(rs, 1, spd))
    d = S0.stats()["depth"]
    worst = 0.0
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S1.op, l, j) == rs.rs_op_box_sizes(S0.op, l, j), (l, j)
            np.testing.assert_array_equal(rs.rs_op_box_indices(S1.op, l, j, 2), rs.rs_op_box_indices(S0.op, l, j, 2))
            e0 = rs.rs_op_box_matrix(S0.op, l, j, 2)
            if e0.size:
                worst = max(worst, _rel(rs.rs_op_box_matrix(S1.op, l, j, 2), e0))
    print("largest relative E difference between the forms: %.2e" % worst)
    assert worst <= 1e-10
    f = W.rhs_normal(n, 17, nrhs=3)
    x0, x1 = S0.solve(f), S1.solve(f)
    assert _rel(x1, x0) <= 1e-12
    F = oracle_mod.Factorization(n, leaf, 1e-10, a=a)
    assert _rel(x1, F.solve(f)) <= 1e-9


def test_bad_gemm_form_is_rejected(rs):
    with pytest.raises(RuntimeError):
        rs.Solver(W.grid_points(16), 4, eps=1e-10, opts=_opts(rs, 2))
