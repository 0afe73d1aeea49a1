"""The forms of the column-pivoted QR of Eq. 2.1 (opts.cpqr_variant): two passes per step with
4 or 8 rows per lane in flight, the look-ahead form (one pass per step, the update of step s
fused with the dot products of step s+1), and the form that keeps the open-column lists in
global memory (taken by itself for boxes too large for shared memory), and the form that keeps
each box in the shared memory of one thread-block cluster (variant 4; levels whose boxes do not
fit 16 CTAs take the default), and the form that processes eight columns per warp pass with
one reduction and one bookkeeping pass per eight (variant 5), the two-rows-in-flight form
capped at the registers of five CTAs per SM (variant 6), and the blocked forms that defer the
trailing updates over panels of 16 or 8 steps (variants 7, 8; real scalars, complex operators
take the default form).  Each is forced on every level and checked
against the oracle: identical ranks and skeleton sets, solutions within the 1e-9 bound of the
FP64 path.  The cases cover several CTAs per box (64^2 grids and up), boxes whose rank test
stops the factorisation before min(r, m) (eps = 1e-5, and the extra group barrier the
look-ahead form takes there), full rank (eps = 0), every scalar type, and the full-size
workload at sampled rows."""
import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2, 3, 4, 5, 6, 7, 8]


@pytest.fixture(scope="module")
def rs():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    P.lib()
    return P


def _opts(rs, variant, precision=None):
    o = rs.rs_opts_default()
    o.cpqr_variant = variant
    if precision is not None:
        o.precision = precision
    return o


def _rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("n,leaf,eps", [(32, 8, 1e-10), (64, 8, 1e-10), (64, 16, 1e-5), (8, 2, 0.0)])
def test_variant_matches_oracle_laplace(rs, oracle_mod, variant, n, leaf, eps):
    a = W.coeff_a_batched(n)
    F = oracle_mod.Factorization(n, leaf, eps, a=a)
    S = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps, opts=_opts(rs, variant))
    mism = []
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S.op, l, j) == F.sizes(l, j), (l, j)
            if not np.array_equal(rs.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j)):
                mism.append((l, j))
    assert not mism, "skeleton sets differ at %s" % mism
    f = W.rhs_normal(n, 5, nrhs=2)
    x = S.solve(f)
    xo = F.solve(f)
    tol = 1e-9 if eps <= 1e-10 else 1e-3
    assert _rel(x, xo) <= tol


@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7, 8])
def test_variant_matches_default_128(rs, variant):
    """128^2 grid, leaves 16^2: Y blocks of several hundred rows and columns, so every loop
    of the kernels (full blocks of rows, leftover rows, paired and single columns) runs."""
    n, leaf, eps = 128, 16, 1e-10
    a = W.coeff_a_batched(n)
    S0 = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps, opts=_opts(rs, 0))
    S1 = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps, opts=_opts(rs, variant))
    d = S0.stats()["depth"]
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S1.op, l, j) == rs.rs_op_box_sizes(S0.op, l, j), (l, j)
    f = W.rhs_normal(n, 6, nrhs=3)
    assert _rel(S1.solve(f), S0.solve(f)) <= 1e-11


def test_look_ahead_helmholtz_c128_and_c64(rs, oracle_mod):
    n, leaf, kappa = 32, 8, 25.0
    b = W.coeff_b_gaussian(n)
    F = oracle_mod.Factorization(n, leaf, 1e-10, b=b, kind=1, kappa=kappa)
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10, kappa=kappa, b=b, opts=_opts(rs, 2, rs.RS_C128))
    mism = []
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S.op, l, j) == F.sizes(l, j), (l, j)
            if not np.array_equal(rs.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j)):
                mism.append((l, j))
    assert not mism
    f = W.rhs_plane_wave(n, kappa)
    assert _rel(S.solve(f), F.solve(f)) <= 1e-9
    o = _opts(rs, 2, rs.RS_C64_REFINED)
    o.refine_max_iter = 12
    S32 = rs.Solver(W.grid_points(n), leaf, eps=1e-5, kappa=kappa, b=b, opts=o)
    x = S32.solve(f)
    res = _rel(oracle_mod.matvec(n, x, b=b, kind=1, kappa=kappa), f)
    assert res <= 1e-10 * 1.01


@pytest.mark.parametrize("variant", [4, 5, 7])
@pytest.mark.parametrize("n,leaf", [(32, 8), (64, 16)])
def test_variant_helmholtz_c128_and_c64(rs, oracle_mod, n, leaf, variant):
    kappa = 25.0
    b = W.coeff_b_gaussian(n)
    F = oracle_mod.Factorization(n, leaf, 1e-10, b=b, kind=1, kappa=kappa)
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10, kappa=kappa, b=b, opts=_opts(rs, variant, rs.RS_C128))
    mism = []
    for l in range(F.depth, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S.op, l, j) == F.sizes(l, j), (l, j)
            if not np.array_equal(rs.rs_op_box_indices(S.op, l, j, 2), F.skel(l, j)):
                mism.append((l, j))
    assert not mism
    f = W.rhs_plane_wave(n, kappa)
    assert _rel(S.solve(f), F.solve(f)) <= 1e-9
    o = _opts(rs, variant, rs.RS_C64_REFINED)
    o.refine_max_iter = 12
    S32 = rs.Solver(W.grid_points(n), leaf, eps=1e-5, kappa=kappa, b=b, opts=o)
    x = S32.solve(f)
    res = _rel(oracle_mod.matvec(n, x, b=b, kind=1, kappa=kappa), f)
    assert res <= 1e-10 * 1.01


@pytest.mark.parametrize("variant", [2, 4, 5, 7, 8])
def test_variant_mixed_fp32(rs, oracle_mod, variant):
    n, leaf = 64, 8
    a = W.coeff_a_batched(n)
    S = rs.Solver(W.grid_points(n), leaf, a=a, eps=1e-6, opts=_opts(rs, variant, rs.RS_MIXED_FP32))
    f = W.rhs_normal(n, 9, nrhs=2)
    x = S.solve(f)
    for c in range(2):
        assert _rel(oracle_mod.matvec(n, x[:, c], a=a), f[:, c]) <= 1e-10 * 1.01


def test_bad_variant_is_rejected(rs):
    o = _opts(rs, 9)
    with pytest.raises(RuntimeError):
        rs.Solver(W.grid_points(16), 4, eps=1e-10, opts=o)


@pytest.mark.slow
def test_look_ahead_full_size_sampled_residual(rs, oracle_mod):
    import torch
    cfg = W.WORKLOADS["laplace_batched"]
    n, leaf, eps = cfg["n"], cfg["leaf"], cfg["eps"]
    a = W.coeff_a_batched(n)
    F = W.rhs_normal(n, cfg["seed"], nrhs=2)
    st = torch.cuda.current_stream()
    tree = rs.rs_build_tree(W.grid_points(n), leaf)
    try:
        op = rs.rs_factor(tree, a=a, eps=eps, opts=_opts(rs, 2), stream=st)
        try:
            f_dev = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
            x_dev = torch.empty_like(f_dev)
            rs.rs_solve(op, f_dev, 2, x_dev, st)
            torch.cuda.synchronize()
            x = x_dev.cpu().numpy().T.copy()
        finally:
            rs.rs_free(op)
    finally:
        rs.rs_free_tree(tree)
    rows = np.random.default_rng(4).choice(n * n, 128, replace=False)
    Ax = oracle_mod.matvec_rows(n, x, rows, a=a)
    for c in range(F.shape[1]):
        assert np.linalg.norm(Ax[:, c] - F[rows, c]) / np.linalg.norm(F[rows, c]) <= 10 * eps
