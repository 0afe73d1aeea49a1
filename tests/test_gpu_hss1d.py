"""Extra compression of Sec. 3 on the GPU vs the CPU oracle, through the C ABI.

Standalone HSS1D (rs_hss1d_*): the same matrix, order, leaf size and eps go to both sides, so
the tree (position ranges), every node's rank and skeleton (integers) must be identical, and
the applies must agree to rounding (the stored blocks are entries of M or ID coefficients of
well-separated blocks, |T| = O(1)).

Compressed factorization (opts.k_cut): the compressed blocks come from each side's own dense
blocks, which agree only to ~1e-7 relative above the leaves (T = R11^{-1} R12 amplifies
rounding by up to 1/eps), so ranks decided in floating point may differ near the threshold;
the integer structure (which boxes, orders, tree depths, position ranges) must be equal, the
ranks within a few of the oracle's with the stored sizes within 2%, and the solutions within
the FP64 tolerance.
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


def _rel(x, y):
    return np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-300)


def _semiseparable(rng, n):
    u, v, p, q = rng.standard_normal((4, n))
    return np.tril(np.outer(u, v), -1) + np.triu(np.outer(p, q), 1) + np.diag(2.0 + rng.uniform(0, 1, n))


def _curve_kernel(n, kappa=None):
    t = 2 * np.pi * (np.arange(n) + 0.5) / n
    P = np.stack([np.cos(t), 0.7 * np.sin(t)], 1)
    r = np.linalg.norm(P[:, None] - P[None], axis=2)
    np.fill_diagonal(r, 1.0)
    if kappa is None:
        M = np.log(r) / n
        np.fill_diagonal(M, 2.0)
        return M
    from scipy.special import hankel1
    M = 0.25j * hankel1(0, kappa * r) / n
    np.fill_diagonal(M, 1.0 + 0.1j)
    return M


MATS = [("semisep", 300, 20, 1e-13, False), ("logcurve", 400, 32, 1e-10, False), ("logcurve", 400, 32, 1e-6, True),
        ("hankel", 300, 24, 1e-10, False), ("random", 157, 16, 0.0, False), ("random", 40, 64, 1e-10, False)]


@pytest.mark.parametrize("kind,n,leaf,eps,permuted", MATS)
def test_standalone_matches_oracle(rs, oracle_mod, kind, n, leaf, eps, permuted):
    rng = np.random.default_rng(n)
    M = {"semisep": lambda: _semiseparable(rng, n), "logcurve": lambda: _curve_kernel(n),
         "hankel": lambda: _curve_kernel(n, 20.0), "random": lambda: rng.standard_normal((n, n))}[kind]()
    order = rng.permutation(n) if permuted else None
    ho = oracle_mod.HSS1D(M, order=order, leaf=leaf, eps=eps)
    h = rs.rs_hss1d_build(M, order=order, leaf=leaf, eps=eps)
    try:
        depth, entries, _ = rs.rs_hss1d_info(h)
        assert depth == ho.depth
        assert entries == ho.entries()
        levels = [(0, 0)] if depth == 0 else [(l, j) for l in range(1, depth + 1) for j in range(2 ** l)]
        for l, j in levels:
            lo, hi, a, k, sk = rs.rs_hss1d_node(h, l, j)
            if depth > 0:
                olo, ohi, oa, ok, osk, _ = ho.node(l, j)
                assert (lo, hi, a, k) == (olo, ohi, oa, ok), (l, j)
                np.testing.assert_array_equal(sk, osk)
        X = rng.standard_normal((n, 3)) + (1j * rng.standard_normal((n, 3)) if np.iscomplexobj(M) else 0)
        Xf = np.asfortranarray(X)
        Y = np.zeros_like(Xf)
        rs.rs_hss1d_apply(h, Xf, 3, Y)
        assert _rel(Y, ho.apply(X)) <= 1e-12
        assert _rel(Y, M @ X) <= 10 * max(eps, 1e-15)
    finally:
        rs.rs_hss1d_free(h)


def test_standalone_device_buffers_and_errors(rs):
    import torch
    n = 256
    M = _curve_kernel(n)
    h = rs.rs_hss1d_build(M, leaf=32, eps=1e-10)
    try:
        X = torch.randn(4, n, dtype=torch.float64, device="cuda")      # column-major n x 4
        Y = torch.empty_like(X)
        rs.rs_hss1d_apply(h, X, 4, Y)
        torch.cuda.synchronize()
        ref = M @ X.cpu().numpy().T
        assert _rel(Y.cpu().numpy().T, ref) <= 1e-9
        with pytest.raises(rs.RsError):
            rs.rs_hss1d_apply(h, X, 4, X)
        with pytest.raises(rs.RsError):
            rs.rs_hss1d_node(h, 9, 0)
    finally:
        rs.rs_hss1d_free(h)
    with pytest.raises(rs.RsError):
        rs.rs_hss1d_build(M, order=np.zeros(n, dtype=np.int64), leaf=32)
    with pytest.raises(rs.RsError):
        rs.rs_hss1d_build(M, leaf=0)


# ------------------------------------------------------------------ compressed factorization

def _opts(rs, k_cut, hss_leaf, precision=0):
    o = rs.rs_opts_default()
    o.k_cut, o.hss_leaf, o.precision = k_cut, hss_leaf, precision
    return o


@pytest.mark.parametrize("n,leaf,k_cut,hss_leaf", [(64, 8, 80, 32), (64, 16, 150, 48), (128, 16, 200, 64)])
def test_compressed_factorization_matches_oracle(rs, oracle_mod, n, leaf, k_cut, hss_leaf):
    eps = 1e-10
    Fo = oracle_mod.Factorization(n, leaf, eps, k_cut=k_cut, hss_leaf=hss_leaf, threads=0)
    S = rs.Solver(W.grid_points(n), leaf, eps=eps, opts=_opts(rs, k_cut, hss_leaf))
    Sd = rs.Solver(W.grid_points(n), leaf, eps=eps)
    st = S.stats()
    ncomp, worst, ksum, kdiff = 0, 0, 0, 0
    for l in range(1, Fo.depth + 1):
        for j in range(2 ** l):
            m, k, _, _ = Fo.sizes(l, j)
            comp = Fo.box_hss(l, j, 2) is not None
            assert comp == (k > k_cut)
            if not comp:
                with pytest.raises(rs.RsError):
                    rs.rs_op_box_form(S.op, l, j, 0)
                continue
            ncomp += 1
            np.testing.assert_array_equal(rs.rs_op_box_order(S.op, l, j, 0), Fo.order(l, j, 0))
            np.testing.assert_array_equal(rs.rs_op_box_order(S.op, l, j, 1), Fo.order(l, j, 1))
            for which in (0, 1, 2):
                depth, _, nodes = rs.rs_op_box_form(S.op, l, j, which)
                h = Fo.box_hss(l, j, which)
                assert depth == h.depth
                if depth > 0:
                    on = np.array([h.node(ll, jj)[:4] for ll in range(1, depth + 1) for jj in range(2 ** ll)])
                    np.testing.assert_array_equal(nodes[:, :2], on[:, :2])       # position ranges
                    worst = max(worst, int(np.abs(nodes[:, 3] - on[:, 3]).max()))
                    ksum += int(on[:, 3].sum())
                    kdiff += int(np.abs(nodes[:, 3] - on[:, 3]).sum())
            for which, w in ((3, 0), (4, 1), (5, 2)):
                depth, _, nodes = rs.rs_op_box_form(S.op, l, j, which)
                assert depth == -1
                worst = max(worst, abs(int(nodes[0, 3]) - Fo.lr_rank(l, j, w)))
    assert ncomp == st["compressed_boxes"] > 0
    assert worst <= 4 and kdiff <= 0.02 * ksum, (worst, kdiff, ksum)
    c_gpu = st["bytes_compressed"] / 8
    c_or, _ = Fo.compressed_entries()
    assert abs(c_gpu - c_or) <= 0.02 * c_or
    assert 0 < st["bytes_compressed"] < st["bytes_dense_replaced"]
    f = W.rhs_uniform(n, 0)
    x = S.solve(f)
    assert _rel(x, Fo.solve(f)) <= SOL_TOL
    assert _rel(x, Sd.solve(f)) <= 10 * eps
    res = rs.rs_residual(S.op, np.asfortranarray(x), np.asfortranarray(f), 1)[0]
    assert res <= 10 * eps


def test_compressed_multi_rhs_device_and_noalloc(rs):
    import torch
    n, leaf, eps = 64, 8, 1e-10
    S = rs.Solver(W.grid_points(n), leaf, eps=eps, opts=_opts(rs, 60, 32))
    Sd = rs.Solver(W.grid_points(n), leaf, eps=eps)
    F = torch.from_numpy(W.rhs_normal(n, 1, nrhs=5).T.copy()).cuda()    # (nrhs, N): column-major N x nrhs
    X = S.solve(F)
    Xd = Sd.solve(F)
    X2 = torch.empty_like(F)
    rs.rs_solve_noalloc(S.op, F, 5, X2)
    torch.cuda.synchronize()
    assert torch.equal(X, X2)
    assert (torch.linalg.norm(X - Xd) / torch.linalg.norm(Xd)).item() <= 10 * eps
    with pytest.raises(rs.RsError):
        rs.rs_op_box_matrix(S.op, 1, 0, 1)            # dense blocks released for level 1
    with pytest.raises(rs.RsError):
        rs.rs_server_create([S.op], 1 << 26)


def test_compressed_mixed_precision_refines(rs):
    n, leaf = 128, 16
    o = _opts(rs, 100, 32, precision=rs.RS_MIXED_FP32)
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-6, opts=o)
    f = W.rhs_uniform(n, 2)
    x = S.solve(f)
    st = S.stats()
    assert st["compressed_boxes"] > 0 and st["refine_residual"] <= 1e-10
    res = rs.rs_residual(S.op, np.asfortranarray(x), np.asfortranarray(f), 1)[0]
    assert res <= 1e-10


def test_compressed_helmholtz(rs, oracle_mod):
    n, leaf, kappa = 32, 8, 10.0
    b = W.coeff_b_gaussian(n)
    f = W.rhs_plane_wave(n, kappa)
    x0 = oracle_mod.Factorization(n, leaf, 1e-10, b=b, kind=oracle_mod.HELMHOLTZ, kappa=kappa).solve(f)
    pts = W.grid_points(n)
    S = rs.Solver(pts, leaf, eps=1e-10, opts=_opts(rs, 40, 16), kappa=kappa, b=b)
    x = S.solve(f)
    assert S.stats()["compressed_boxes"] > 0
    assert _rel(x, x0) <= 1e-5        # eps-relative block errors amplified by the apply's cancellation
    o = _opts(rs, 40, 16, precision=rs.RS_C64_REFINED)
    S2 = rs.Solver(pts, leaf, eps=1e-5, opts=o, kappa=kappa, b=b)
    x2 = S2.solve(f)
    assert S2.stats()["refine_residual"] <= 1e-10
    assert _rel(x2, x0) <= 1e-8
