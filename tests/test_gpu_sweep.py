"""The symmetric sweep inverse (F^{-1}, E and the root of the real symmetric Laplace kernel,
no pivoting, m^3 flops) against pivoted Gauss-Jordan (2 m^3 flops) on the same operator, and
its fallback when a block is not positive definite.

Both inversions see the same F (the ID phase is deterministic), so leaf inverses agree to
cond(F) u ~ 1e-14; blocks above the leaves also carry the children's E, which differ by the
same order amplified through T (|T| ~ 1/eps at worst): tolerance 1e-9.
"""
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


def _rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


def _factor(rs, n, leaf, eps, a, spd, panel=0):
    o = rs.rs_opts_default()
    o.spd_inverse = spd
    o.sweep_panel = panel
    return rs.Solver(W.grid_points(n), leaf, a=a, eps=eps, opts=o)


@pytest.mark.parametrize("panel", [8, 16])
@pytest.mark.parametrize("n,leaf,eps", [(32, 8, 1e-10), (64, 8, 1e-10), (64, 16, 1e-6), (8, 2, 0.0)])
def test_sweep_matches_pivoted_gauss_jordan(rs, n, leaf, eps, panel):
    """Panels of 8 and of 16 columns (a block of 8 x 8 or 16 x 16 pivots per step)."""
    a = W.coeff_a_batched(n)
    S1 = _factor(rs, n, leaf, eps, a, 1, panel)
    S0 = _factor(rs, n, leaf, eps, a, 0)
    assert S1.stats()["spd_fallbacks"] == 0
    d = S1.stats()["depth"]
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S1.op, l, j) == rs.rs_op_box_sizes(S0.op, l, j)
            tol = 1e-12 if l == d else 1e-9
            f1, f0 = rs.rs_op_box_matrix(S1.op, l, j, 1), rs.rs_op_box_matrix(S0.op, l, j, 1)
            assert _rel(f1, f0) <= tol, ("Finv", l, j, _rel(f1, f0))
            np.testing.assert_array_equal(f1, f1.T)          # the sweep writes an exactly symmetric inverse
            e1, e0 = rs.rs_op_box_matrix(S1.op, l, j, 2), rs.rs_op_box_matrix(S0.op, l, j, 2)
            if e0.size:
                assert _rel(e1, e0) <= 1e-9, ("E", l, j, _rel(e1, e0))
    r1, r0 = rs.rs_op_root_matrix(S1.op), rs.rs_op_root_matrix(S0.op)
    assert _rel(r1, r0) <= 1e-9
    f = W.rhs_uniform(n, 4)
    assert _rel(S1.solve(f), S0.solve(f)) <= 1e-11


def test_not_positive_definite_falls_back(rs, oracle_mod):
    """a = -1: A = -I + K is negative definite, so the sweep stops at its first pivot on every
    level and the level is redone with pivoted Gauss-Jordan; the result is the oracle's."""
    n, leaf, eps = 32, 8, 1e-10
    a = -np.ones(n * n)
    S = _factor(rs, n, leaf, eps, a, 1)
    st = S.stats()
    assert st["spd_fallbacks"] == 2 * st["depth"] + 1          # F and E per level, and the root
    f = W.rhs_uniform(n, 5)
    xo = oracle_mod.Factorization(n, leaf, eps, a=a).solve(f)
    assert _rel(S.solve(f), xo) <= 1e-9


def test_indefinite_level_falls_back(rs, oracle_mod):
    """a = -0.05: A is indefinite; whichever blocks the sweep rejects are redone, and the
    solution still matches the oracle's pivoted factorization."""
    n, leaf, eps = 32, 8, 1e-10
    a = np.full(n * n, -0.05)
    S = _factor(rs, n, leaf, eps, a, 1)
    f = W.rhs_uniform(n, 6)
    xo = oracle_mod.Factorization(n, leaf, eps, a=a).solve(f)
    assert _rel(S.solve(f), xo) <= 1e-9


def test_bad_panel_width_is_refused(rs):
    with pytest.raises(RuntimeError):
        _factor(rs, 16, 4, 1e-10, None, 1, 12)
