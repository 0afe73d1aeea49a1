"""Helmholtz / Lippmann-Schwinger (Sec. 5.3-5.4): sigma + kappa^2 b (i/4) int H0(kappa|x-y|) sigma = f,
factored in the symmetric form of Eq. (5.6) (diagonal similarity by kappa sqrt(b)).

RS_C128: complex128 factorization compared with the oracle (ranks, skeletons and index lists
exactly; solutions to 1e-9).  RS_C64_REFINED: complex64 factorization at eps = 1e-5 refined to
1e-10 with the complex128 direct-sum residual; compared with the dense complex solve.  The
solution tolerance there is cond(A) x (r_gpu + r_ref) with cond(A) measured on the dense
matrix (about 2e1 at kappa = 25 on these grids), i.e. 1e-8.
"""
import numpy as np
import pytest

import _dense as D
from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu
KAPPA = 25.0


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    return P


def _opts(P, prec, tol=1e-10):
    o = P.rs_opts_default()
    o.precision = prec
    o.refine_tol = tol
    o.refine_max_iter = 12
    return o


@pytest.mark.parametrize("n,leaf", [(16, 4), (32, 8)])
def test_c128_matches_oracle(P, oracle_mod, n, leaf):
    b = W.coeff_b_gaussian(n)
    F = oracle_mod.Factorization(n, leaf, 1e-10, b=b, kind=1, kappa=KAPPA)
    S = P.Solver(W.grid_points(n), leaf, eps=1e-10, kappa=KAPPA, b=b, opts=_opts(P, P.RS_C128))
    mism = []
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            assert P.rs_op_box_sizes(S.op, l, j) == F.sizes(l, j), (l, j)
            np.testing.assert_array_equal(P.rs_op_box_indices(S.op, l, j, 0), F.active(l, j))
            np.testing.assert_array_equal(P.rs_op_box_indices(S.op, l, j, 1), F.near(l, j))
            if not np.array_equal(P.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j)):
                mism.append((l, j))
    assert not mism
    d = F.depth
    fi = P.rs_op_box_matrix(S.op, d, 0, 1, cplx=True)
    assert np.linalg.norm(fi - F.Finv(d, 0)) <= 1e-11 * np.linalg.norm(fi)
    f = W.rhs_plane_wave(n, KAPPA)
    x = S.solve(f)
    xo = F.solve(f)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)


def test_c64_refined_matches_dense(P, oracle_mod):
    n, leaf = 64, 16
    b = W.coeff_b_gaussian(n)
    S = P.Solver(W.grid_points(n), leaf, eps=1e-5, kappa=KAPPA, b=b, opts=_opts(P, P.RS_C64_REFINED))
    f = W.rhs_plane_wave(n, KAPPA)
    x = S.solve(f)
    st = P.rs_op_stats(S.op)
    assert st["refine_residual"] <= 1e-10 and st["refine_iters"] >= 2
    A = D.helmholtz(n, KAPPA, b)
    xd = np.linalg.solve(A, f)
    assert np.linalg.norm(A @ x - f) <= 1e-10 * np.linalg.norm(f) * 1.01
    assert np.linalg.norm(x - xd) <= 1e-8 * np.linalg.norm(xd)
    rel = P.rs_residual(S.op, np.ascontiguousarray(x), np.ascontiguousarray(f), 1)[0]
    want = np.linalg.norm(oracle_mod.matvec(n, x, b=b, kind=1, kappa=KAPPA) - f) / np.linalg.norm(f)
    assert abs(rel - want) <= 1e-13


@pytest.mark.slow
def test_lippmann_schwinger_full_size(P, oracle_mod):
    """256 x 256 grid (N = 65536), kappa = 25, b = exp(-40 |x - (1/2,1/2)|^2), f = exp(i kappa x1):
    complex64 factor at eps = 1e-5, refined to 1e-10 with the complex128 residual, against the
    oracle's complex128 factorization of the same problem (eps 1e-10) refined by its own
    brute-force residual to 1e-12.  Two solutions with residuals r1, r2 differ by at most
    cond(A) (r1 + r2); cond(A) is about 2e1 at kappa = 25 (measured on the dense matrix of
    the smaller grids), so 1e-8 is asserted with both residuals stated in the message."""
    import torch
    cfg = W.WORKLOADS["helmholtz_ls"]
    n, leaf = cfg["n"], cfg["leaf"]
    b = W.coeff_b_gaussian(n)
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, eps=cfg["eps"], opts=_opts(P, P.RS_C64_REFINED), kappa=KAPPA, b=b)
    try:
        f = W.rhs_plane_wave(n, KAPPA)
        fd = torch.from_numpy(f).cuda()
        xd = torch.empty_like(fd)
        P.rs_solve(op, fd, 1, xd, torch.cuda.current_stream())
        st = P.rs_op_stats(op)
        assert st["refine_residual"] <= 1e-10
        x = xd.cpu().numpy()
        rows = np.random.default_rng(5).choice(n * n, 96, replace=False)
        r = oracle_mod.matvec_rows(n, x, rows, b=b, kind=1, kappa=KAPPA) - f[rows]
        assert np.linalg.norm(r) <= 10 * 1e-10 * np.linalg.norm(f[rows])
        orc = oracle_mod.Factorization(n, leaf, 1e-10, b=b, kind=1, kappa=KAPPA)
        xo, r_orc, _ = oracle_mod.solve_refined(orc, f, tol=1e-12, max_iter=4)
        assert r_orc <= 1e-12
        diff = np.linalg.norm(x - xo) / np.linalg.norm(xo)
        assert diff <= 1e-8, "difference %.2e; residuals: GPU %.2e, oracle %.2e" % (
            diff, st["refine_residual"], r_orc)
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)
