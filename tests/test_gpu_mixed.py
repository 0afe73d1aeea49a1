"""Mixed precision (S9): FP32 factorization at a looser eps, FP64 pivot norms and panel
arithmetic, and iterative refinement with the FP64 direct-sum residual (the paper's round of
refinement, Sec. 5.3-5.4, repeated to a tolerance).

The mixed path is compared on solutions only: its FP32 ranks need not equal the FP64
oracle's.  Both sides refine to their own residual bound; two solutions with relative
residuals r1, r2 differ by at most cond(A) (r1 + r2), and cond(A) ~ 1.13 here, so with
r_gpu <= 1e-10 and r_oracle <= 1e-12 the tolerance is 1e-9.
"""
import os

import numpy as np
import pytest

import _dense as D
from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    return P


def _mixed_opts(P, tol=1e-10):
    o = P.rs_opts_default()
    o.precision = P.RS_MIXED_FP32
    o.refine_tol = tol
    o.refine_max_iter = 10
    return o


def test_residual_matches_brute_force(P, oracle_mod):
    n = 32
    tree = P.rs_build_tree(W.grid_points(n), 8)
    op = P.rs_factor(tree, eps=1e-10)
    try:
        a = None
        rng = np.random.default_rng(4)
        x = np.asfortranarray(rng.standard_normal((n * n, 3)))
        f = np.asfortranarray(rng.standard_normal((n * n, 3)))
        rel = P.rs_residual(op, x, f, 3)
        r = f - oracle_mod.matvec(n, x)
        want = np.linalg.norm(r, axis=0) / np.linalg.norm(f, axis=0)
        np.testing.assert_allclose(rel, want, rtol=1e-12)
        # a tiny residual: x = the oracle's refined solution
        Fo = oracle_mod.Factorization(n, 8, 1e-10)
        f1 = W.rhs_uniform(n, 0)
        x1, r1, _ = oracle_mod.solve_refined(Fo, f1, tol=1e-14)
        rel1 = P.rs_residual(op, np.asfortranarray(x1), np.asfortranarray(f1), 1)[0]
        assert abs(rel1 - r1) <= 1e-14
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)


@pytest.mark.parametrize("n,leaf,avar", [(64, 8, False), (64, 16, True), (128, 16, False)])
def test_mixed_refined_solution_matches_oracle(P, oracle_mod, n, leaf, avar):
    eps = 1e-6
    a = W.coeff_a_batched(n) if avar else None
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, a=a, eps=eps, opts=_mixed_opts(P))
    try:
        f = W.rhs_uniform(n, 2)
        x = np.zeros(n * n)
        P.rs_solve(op, np.ascontiguousarray(f), 1, x)
        st = P.rs_op_stats(op)
        assert st["refine_residual"] <= 1e-10 and 1 <= st["refine_iters"] <= 10
        Fo = oracle_mod.Factorization(n, leaf, eps, a=a)
        xo, ro, _ = oracle_mod.solve_refined(Fo, f, tol=1e-12)
        assert ro <= 1e-12
        assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
        res = np.linalg.norm(oracle_mod.matvec(n, x, a=a) - f) / np.linalg.norm(f)
        assert res <= 1e-10
        if n <= 64:
            xd = np.linalg.solve(D.laplace(n, a), f)
            assert np.linalg.norm(x - xd) <= 1e-9 * np.linalg.norm(xd)
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)


def test_mixed_multi_rhs_device_and_nonconvergence(P):
    import torch
    n, leaf = 64, 8
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, eps=1e-6, opts=_mixed_opts(P))
    try:
        F = W.rhs_normal(n, 3, nrhs=3)
        f = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
        x = torch.empty_like(f)
        P.rs_solve(op, f, 3, x, torch.cuda.current_stream())
        rel = P.rs_residual(op, x, f, 3)
        assert (rel <= 1e-10).all()
    finally:
        P.rs_free(op)
    # one low-precision solve cannot reach 1e-14: the call reports RS_E_NOT_CONVERGED
    o = _mixed_opts(P, tol=1e-14)
    o.refine_max_iter = 1
    op = P.rs_factor(tree, eps=1e-6, opts=o)
    try:
        x = np.zeros(n * n)
        with pytest.raises(P.RsError) as e:
            P.rs_solve(op, W.rhs_uniform(n, 2), 1, x)
        assert e.value.code == P.RS_E_NOT_CONVERGED
        assert np.isfinite(x).all() and np.linalg.norm(x) > 0
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)


@pytest.mark.slow
def test_mixed_full_size_sampled_residual(P, oracle_mod):
    """The mixed workload at full size: 1024 x 1024 grid (N = 1048576), leaves 16 x 16,
    eps 1e-6 FP32 factor, refinement to 1e-10, f ~ U[-1,1] (seed 2).

    Checked against the oracle's FP64 solution of the same problem (eps 1e-10, stored for 2048
    sampled rows by tests/golden/make_laplace_mixed_sample.py, which calls only the oracle):
    two solutions with residuals r1, r2 differ by at most |A^{-1}| (r1 + r2) |f|, and A =
    I + (a positive operator) has |A^{-1}| <= 1, so with r1 <= 1e-10 (the refinement target)
    and the oracle's r2 (stated in the file, ~1e-13) the sampled relative difference is held to
    1e-9.  The true residual on 128 of those rows, computed entry by entry by the oracle, is
    held to the 1e-10 target itself."""
    import torch
    cfg = W.WORKLOADS["laplace_mixed"]
    n, leaf = cfg["n"], cfg["leaf"]
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, eps=cfg["eps"], opts=_mixed_opts(P), stream=torch.cuda.current_stream())
    try:
        f = W.rhs_uniform(n, cfg["seed"])
        fd = torch.from_numpy(f).cuda()
        xd = torch.empty_like(fd)
        P.rs_solve(op, fd, 1, xd, torch.cuda.current_stream())
        st = P.rs_op_stats(op)
        assert st["refine_residual"] <= 1e-10
        x = xd.cpu().numpy()
        gold = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "laplace_mixed_1024_oracle_sample.txt"))
        rows = gold[:, 0].astype(np.int64)
        xo = gold[:, 1]
        diff = np.linalg.norm(x[rows] - xo) / np.linalg.norm(xo)
        assert diff <= 1e-9, diff
        sub = rows[:128]
        r = oracle_mod.matvec_rows(n, x, sub) - f[sub]
        assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(f[sub])
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)
