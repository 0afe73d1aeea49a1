"""opts.per_box = 1 launches every factor and solve kernel for one box at a time (the unbatched
form the per-level launches are measured against).  It runs the same arithmetic per box --
only the CTA counts, and with them the solve's summation blocks, differ -- so ranks and
skeletons are identical and solutions agree to rounding."""
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


def _solver(rs, n, leaf, per_box, **kw):
    o = rs.rs_opts_default()
    o.per_box = per_box
    return rs.Solver(W.grid_points(n), leaf, eps=1e-10, opts=o, **kw)


@pytest.mark.parametrize("n,leaf", [(32, 8), (64, 8)])
def test_per_box_matches_batched_laplace(rs, oracle_mod, n, leaf):
    a = W.coeff_a_batched(n)
    S1 = _solver(rs, n, leaf, 1, a=a)
    S0 = _solver(rs, n, leaf, 0, a=a)
    d = S0.stats()["depth"]
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S1.op, l, j) == rs.rs_op_box_sizes(S0.op, l, j)
            np.testing.assert_array_equal(rs.rs_op_box_indices(S1.op, l, j, 2), rs.rs_op_box_indices(S0.op, l, j, 2))
    f = W.rhs_normal(n, 8, nrhs=3)
    x1, x0 = S1.solve(f), S0.solve(f)
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
    xo = oracle_mod.Factorization(n, leaf, 1e-10, a=a).solve(f)
    assert np.linalg.norm(x1 - xo) <= 1e-9 * np.linalg.norm(xo)


def test_per_box_helmholtz_c128(rs):
    n, leaf, kappa = 32, 8, 10.0
    b = W.coeff_b_gaussian(n)
    S1 = _solver(rs, n, leaf, 1, kappa=kappa, b=b)
    S0 = _solver(rs, n, leaf, 0, kappa=kappa, b=b)
    f = W.rhs_plane_wave(n, kappa)
    x1, x0 = S1.solve(f), S0.solve(f)
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
