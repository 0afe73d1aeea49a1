"""rs_fwd_apply (the forward apply through the HSS form the factorization's IDs define) on the
GPU: against the brute-force matvec (exact without truncation, within 10 eps with it; for
Helmholtz in the symmetric form), against the oracle's forward apply of the same HSS form, and
against the factorization itself (rs_solve inverts it to rounding) -- in every precision, with
several right-hand sides on device buffers, in the translation-invariant modes, at full size
(512^2, varying a) on sampled rows, and the operators it must refuse."""
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


def test_fwd_exact_without_truncation(rs, oracle_mod):
    n = 8
    S = rs.Solver(W.grid_points(n), 2, eps=0.0)
    x = W.rhs_normal(n, 1, nrhs=3)
    assert _rel(S.fwd_apply(x), oracle_mod.matvec(n, x)) <= 1e-13


@pytest.mark.parametrize("n,leaf,eps", [(16, 4, 1e-10), (32, 8, 1e-10), (64, 8, 1e-10), (64, 16, 1e-5), (128, 16, 1e-10)])
def test_fwd_matches_brute_force_and_oracle(rs, oracle_mod, n, leaf, eps):
    a = W.coeff_a_batched(n)
    S = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps)
    x = W.rhs_normal(n, 2, nrhs=5)
    y = S.fwd_apply(x)
    yr = oracle_mod.matvec(n, x, a=a)
    assert _rel(y, yr) <= 10 * eps
    if n <= 64:
        yo = oracle_mod.Factorization(n, leaf, eps, a=a).fwd_apply(x)
        assert _rel(y, yo) <= 10 * eps
    f = W.rhs_uniform(n, 4)
    assert _rel(S.fwd_apply(S.solve(f)), f) <= 1e-12


def test_fwd_device_buffers_and_order(rs, oracle_mod):
    import torch
    n, leaf = 32, 8
    order = W.shuffled(n, 3)
    S = rs.Solver(W.grid_points(n)[order], leaf, eps=1e-10)
    X = W.rhs_normal(n, 5, nrhs=3)
    xin = np.ascontiguousarray(X[order].T)                 # (nrhs, N) rows = column-major N x nrhs
    xd = torch.from_numpy(xin).cuda()
    yd = torch.empty_like(xd)
    rs.rs_fwd_apply(S.op, xd, 3, yd, torch.cuda.current_stream())
    torch.cuda.synchronize()
    y = yd.cpu().numpy().T
    yr = oracle_mod.matvec(n, X)[order]
    assert _rel(y, yr) <= 1e-9


def test_fwd_helmholtz_c128_and_low_precision(rs, oracle_mod):
    n, leaf, kappa = 32, 8, 25.0
    b = W.coeff_b_gaussian(n)
    s = kappa * np.sqrt(b)
    x = W.rhs_plane_wave(n, kappa)
    yr = oracle_mod.matvec(n, x, b=b, kind=1, kappa=kappa)
    o = rs.rs_opts_default()
    o.precision = rs.RS_C128
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10, kappa=kappa, b=b, opts=o)
    y = S.fwd_apply(x)
    assert _rel(y / s, yr / s) <= 1e-9
    assert _rel(S.fwd_apply(S.solve(x)), x) <= 1e-11
    o.precision = rs.RS_C64_REFINED
    S64 = rs.Solver(W.grid_points(n), leaf, eps=1e-5, kappa=kappa, b=b, opts=o)
    assert _rel(S64.fwd_apply(x) / s, yr / s) <= 1e-4
    n = 64
    om = rs.rs_opts_default()
    om.precision = rs.RS_MIXED_FP32
    Sm = rs.Solver(W.grid_points(n), 8, eps=1e-6, opts=om)
    v = W.rhs_normal(n, 7)
    assert _rel(Sm.fwd_apply(v), oracle_mod.matvec(n, v)) <= 1e-5


@pytest.mark.parametrize("mode", [1, 2])
def test_fwd_translation_invariant(rs, oracle_mod, mode):
    n, leaf = 64, 8
    o = rs.rs_opts_default()
    o.translation_invariant = mode
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10, opts=o)
    x = W.rhs_normal(n, 8, nrhs=2)
    assert _rel(S.fwd_apply(x), oracle_mod.matvec(n, x)) <= 1e-9
    assert _rel(S.fwd_apply(S.solve(x)), x) <= 1e-12


def test_fwd_refuses_compressed_operators(rs):
    n = 64
    o = rs.rs_opts_default()
    o.k_cut = 32
    S = rs.Solver(W.grid_points(n), 8, eps=1e-10, opts=o)
    if S.stats()["compressed_boxes"] > 0:
        with pytest.raises(RuntimeError):
            S.fwd_apply(np.ones(n * n))


@pytest.mark.slow
def test_fwd_full_size(rs, oracle_mod):
    import torch
    cfg = W.WORKLOADS["laplace_batched"]
    n, leaf, eps = cfg["n"], cfg["leaf"], cfg["eps"]
    a = W.coeff_a_batched(n)
    st = torch.cuda.current_stream()
    tree = rs.rs_build_tree(W.grid_points(n), leaf)
    try:
        op = rs.rs_factor(tree, a=a, eps=eps, stream=st)
        try:
            X = W.rhs_normal(n, 9, nrhs=2)
            xd = torch.from_numpy(np.ascontiguousarray(X.T)).cuda()
            yd = torch.empty_like(xd)
            rs.rs_fwd_apply(op, xd, 2, yd, st)
            zd = torch.empty_like(xd)
            rs.rs_solve(op, yd, 2, zd, st)             # A^{-1} (A x) = x for the HSS pair
            torch.cuda.synchronize()
            y = yd.cpu().numpy().T
            z = zd.cpu().numpy().T
        finally:
            rs.rs_free(op)
    finally:
        rs.rs_free_tree(tree)
    assert _rel(z, X) <= 1e-11
    rows = np.random.default_rng(6).choice(n * n, 64, replace=False)
    yr = oracle_mod.matvec_rows(n, X, rows, a=a)
    assert _rel(y[rows], yr) <= 10 * eps
