"""rs_autotune on a small operator: it fills the table for every level, the tuned
factorization gives the same ranks and (up to the rounding order of the CPQR variants) the
same solution, and the table survives a save / clear / load cycle."""
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


def test_autotune_fills_table_and_keeps_results(rs, tmp_path):
    n, leaf, eps = 64, 8, 1e-10
    a = W.coeff_a_batched(n)
    rs.rs_tune_clear()
    S0 = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps)
    f = W.rhs_uniform(n, 7)
    x0 = S0.solve(f)
    tree = rs.rs_build_tree(W.grid_points(n), leaf)
    try:
        path = tmp_path / "tune.json"
        rep = rs.rs_autotune(tree, a=a, eps=eps, path=path)
    finally:
        rs.rs_free_tree(tree)
    d = S0.stats()["depth"]
    assert rep["candidates"] >= 4 and rep["keys_set"] >= d
    assert rep["default_factor_ms"] > 0 and rep["tuned_factor_ms"] > 0
    assert rs.rs_tune_count() > 0 and path.exists()
    S1 = rs.Solver(W.grid_points(n), leaf, a=a, eps=eps)
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert rs.rs_op_box_sizes(S1.op, l, j) == rs.rs_op_box_sizes(S0.op, l, j)
    x1 = S1.solve(f)
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
    cnt = rs.rs_tune_count()
    rs.rs_tune_clear()
    rs.rs_tune_load(path)
    assert rs.rs_tune_count() == cnt
    rs.rs_tune_clear()
