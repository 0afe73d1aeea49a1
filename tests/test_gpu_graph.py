"""rs_solve replayed from a CUDA graph (opts.solve_graph = 1, the default) against the same
apply launched kernel by kernel (solve_graph = 0): the graph holds the same launches, so the
results are bit-identical, across repeated calls, different nrhs (one graph each) and
workspace growth (which retires the older graphs)."""
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


def _solver(rs, n, leaf, graph, **kw):
    o = rs.rs_opts_default()
    o.solve_graph = graph
    return rs.Solver(W.grid_points(n), leaf, eps=1e-10, opts=o, **kw)


def test_graph_replay_is_bit_identical(rs):
    import torch
    n, leaf = 64, 8
    Sg = _solver(rs, n, leaf, 1)
    Sk = _solver(rs, n, leaf, 0)
    for nrhs in (1, 4, 2, 4, 9, 1):          # cache hits, new nrhs, workspace growth at 9
        f = torch.from_numpy(np.ascontiguousarray(W.rhs_normal(n, 20 + nrhs, nrhs=nrhs).T)).cuda()
        xg = Sg.solve(f)
        xk = Sk.solve(f)
        torch.cuda.synchronize()
        assert torch.equal(xg, xk), nrhs


def test_graph_launch_count_matches_direct_launches(rs):
    import torch
    n, leaf = 32, 8
    Sg = _solver(rs, n, leaf, 1)
    Sk = _solver(rs, n, leaf, 0)
    f = torch.from_numpy(np.ascontiguousarray(W.rhs_normal(n, 3, nrhs=2).T)).cuda()
    Sg.solve(f)                               # capture
    counts = []
    for S in (Sg, Sk):
        c0 = rs.rs_launch_count()
        S.solve(f)
        torch.cuda.synchronize()
        counts.append(rs.rs_launch_count() - c0)
    assert counts[0] == counts[1] > 0


def test_graph_helmholtz_c128(rs):
    n, leaf, kappa = 32, 8, 10.0
    b = W.coeff_b_gaussian(n)
    Sg = _solver(rs, n, leaf, 1, kappa=kappa, b=b)
    Sk = _solver(rs, n, leaf, 0, kappa=kappa, b=b)
    f = W.rhs_plane_wave(n, kappa)
    np.testing.assert_array_equal(Sg.solve(f), Sk.solve(f))
