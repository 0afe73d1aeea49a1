"""The batched Laplace workload at full size (512 x 512 grid, leaves 16 x 16, eps 1e-10,
a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2), 4 RHS), in the launch configuration the benchmark
times (device buffers on the current torch stream, the autotuned launch shapes when a table
is loaded), against the oracle's factorization of the same workload over the whole tree
(Algorithm 1 with the E of Algorithm 2, every level, all host cores) and its inverse apply
(Algorithm 6).

- every box of every level: sizes (m, k, r, near rows), active sets and skeleton sets
  identical (integer results, bit-exact);
- factor blocks on sampled boxes of every level (every box of levels 1-2) and the root
  inverse, within the block tolerances derived in test_blocks_match_oracle_on_every_level;
- the 4-RHS solution within the 1e-9 FP64 tolerance of the oracle's solution;
- the true residual on sampled rows (computed entry by entry by the oracle) within 10 eps.
"""
import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def full(oracle_mod):
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    cfg = W.WORKLOADS["laplace_batched"]
    n, leaf, eps, nrhs = cfg["n"], cfg["leaf"], cfg["eps"], cfg["nrhs"]
    a = W.coeff_a_batched(n)
    F = W.rhs_normal(n, cfg["seed"], nrhs=nrhs)
    st = torch.cuda.current_stream()
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, a=a, eps=eps, stream=st)
    f_dev = torch.from_numpy(np.ascontiguousarray(F.T)).cuda()
    x_dev = torch.empty_like(f_dev)
    P.rs_solve(op, f_dev, nrhs, x_dev, st)
    torch.cuda.synchronize()
    x = x_dev.cpu().numpy().T.copy()
    orc = oracle_mod.Factorization(n, leaf, eps, a=a)
    yield dict(P=P, op=op, n=n, a=a, F=F, x=x, eps=eps, orc=orc, d=orc.depth)
    P.rs_free(op)
    P.rs_free_tree(tree)


def test_every_level_matches_oracle(full):
    P, op, orc, d = full["P"], full["op"], full["orc"], full["d"]
    mism = []
    for l in range(d, 0, -1):
        for j in range(2 ** l):
            assert P.rs_op_box_sizes(op, l, j) == orc.sizes(l, j), (l, j)
            np.testing.assert_array_equal(P.rs_op_box_indices(op, l, j, 0), orc.active(l, j))
            if not np.array_equal(P.rs_op_box_indices(op, l, j, 2), orc.skel(l, j)):
                mism.append((l, j))
    assert not mism, "skeleton sets differ at %s" % mism[:20]


def test_blocks_match_oracle_on_every_level(full):
    """Block tolerances.  A leaf's F^{-1} involves no T: 1e-11 (as in test_gpu_parity).  T =
    R11^{-1} R12 with |R_kk| / |R_11| ~ eps carries rounding differences of R amplified by up
    to 1/eps: 100 u / eps = 1e-4.  E, F^{-1} above the leaves and the root inverse are built
    from the children's T and E, so they carry those differences too; at this size their
    condition numbers reach 1e4 (|F^{-1}| ~ 4e3 at level 1) and the small-grid bound of 1e-6
    no longer holds, so they are held to T's bound, 1e-4.  The solution itself is held to
    1e-9 below.  The largest observed difference per kind is printed."""
    P, op, orc, d = full["P"], full["op"], full["orc"], full["d"]
    rng = np.random.default_rng(0)
    worst = {"Finv_leaf": 0.0, "Finv": 0.0, "E": 0.0, "T": 0.0}
    bad = []

    def rel(a, b, floor=0.0):
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(a), floor))

    for l in range(d, 0, -1):
        boxes = range(2 ** l) if l <= 2 else rng.choice(2 ** l, 3, replace=False)
        for j in boxes:
            kf = "Finv_leaf" if l == d else "Finv"
            checks = [(kf, rel(P.rs_op_box_matrix(op, l, j, 1), orc.Finv(l, j)), 1e-11 if l == d else 1e-4),
                      ("E", rel(P.rs_op_box_matrix(op, l, j, 2), orc.E(l, j)), 1e-4)]
            t = P.rs_op_box_matrix(op, l, j, 0)
            if t.size:
                checks.append(("T", rel(t, orc.T(l, j), 1.0), 1e-4))
            for kind, v, tol in checks:
                worst[kind] = max(worst[kind], v)
                if not v <= tol:
                    bad.append((kind, l, int(j), v))
    r = P.rs_op_root_matrix(op)
    root = rel(r, orc.root_inv())
    print("largest relative block differences:", worst, "root inverse %.2e" % root)
    assert not bad, bad[:10]
    assert root <= 1e-4


def test_solution_matches_oracle(full):
    x, F, orc = full["x"], full["F"], full["orc"]
    xo = orc.solve(F)
    for c in range(F.shape[1]):
        rel = np.linalg.norm(x[:, c] - xo[:, c]) / np.linalg.norm(xo[:, c])
        assert rel <= 1e-9, (c, rel)


def test_sampled_residual(full, oracle_mod):
    n, x, F, a, eps = full["n"], full["x"], full["F"], full["a"], full["eps"]
    rows = np.random.default_rng(2).choice(n * n, 256, replace=False)
    Ax = oracle_mod.matvec_rows(n, x, rows, a=a)
    for c in range(F.shape[1]):
        r = np.linalg.norm(Ax[:, c] - F[rows, c]) / np.linalg.norm(F[rows, c])
        assert r <= 10 * eps, (c, r)


def test_stats_are_consistent(full):
    s = full["P"].rs_op_stats(full["op"])
    assert s["depth"] == full["d"] and s["n_side"] == full["n"]
    assert s["flops_factor"] > 0 and s["bytes_factors"] > 0 and s["root_m"] == full["orc"].root_inv().shape[0]
