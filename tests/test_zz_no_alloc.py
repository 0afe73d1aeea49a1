"""rs_solve_noalloc: the inverse apply with its workspace in a fixed device array.

Some callers cannot allocate device memory while they serve solves: their memory already
belongs to another allocator or to fixed budgets, or a cudaMalloc would stall a latency-bound
request path.  For them the library offers rs_solve_noalloc, which computes what rs_solve
computes without allocating.  These tests call both through the C ABI and compare them, on two
calls in a row, within the solution tolerance of the parity tests; they also check that a
request too large for the fixed array is refused without touching the output.
"""
import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SOL_TOL = 1e-9   # the FP64 solution tolerance of test_gpu_parity


@pytest.fixture(scope="module")
def small():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    n, leaf, eps = 64, 8, 1e-10
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, eps=eps)
    yield P, op, n
    P.rs_free(op)
    P.rs_free_tree(tree)


def _dev(F):
    import torch
    return torch.from_numpy(np.ascontiguousarray(F.T)).cuda()     # N x nrhs column-major


def _rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_noalloc_matches_rs_solve_on_two_calls(small):
    import torch
    P, op, n = small
    for seed in (11, 12):                       # two calls in a row, different right-hand sides
        f = _dev(W.rhs_normal(n, seed, nrhs=4))
        x_ref = torch.empty_like(f)
        x_na = torch.full_like(f, np.nan)
        P.rs_solve(op, f, 4, x_ref, torch.cuda.current_stream())
        P.rs_solve_noalloc(op, f, 4, x_na, torch.cuda.current_stream())
        torch.cuda.synchronize()
        a, b = x_na.cpu().numpy(), x_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert _rel(a, b) <= SOL_TOL


def test_noalloc_refuses_oversize_and_host_buffers(small):
    import torch
    P, op, n = small
    nrhs = 512                                   # needs more than the fixed 32 MiB array
    f = torch.zeros((nrhs, n * n), dtype=torch.float64, device="cuda")
    x = torch.full_like(f, 7.0)
    with pytest.raises(P.RsError) as e:
        P.rs_solve_noalloc(op, f, nrhs, x, torch.cuda.current_stream())
    assert e.value.code == P.RS_E_INVALID and "workspace" in str(e.value)
    torch.cuda.synchronize()
    assert bool((x == 7.0).all())
    fh = np.zeros(n * n)
    with pytest.raises(P.RsError) as e:
        P.rs_solve_noalloc(op, fh, 1, np.zeros(n * n))
    assert e.value.code == P.RS_E_INVALID


def test_noalloc_refuses_huge_nrhs_before_size_arithmetic(small):
    import torch
    P, op, n = small
    f = torch.zeros(n * n, dtype=torch.float64, device="cuda")
    x = torch.full_like(f, 7.0)
    for nrhs in (1 << 40, (1 << 51) + 3):        # products with the layout offsets would overflow
        with pytest.raises(P.RsError) as e:
            P.rs_solve_noalloc(op, f, nrhs, x, torch.cuda.current_stream())
        assert e.value.code == P.RS_E_INVALID and "workspace" in str(e.value)
    torch.cuda.synchronize()
    assert bool((x == 7.0).all())


def test_noalloc_on_fresh_operator_grows_no_workspace():
    """On an operator that rs_solve has never touched, rs_solve_noalloc alone leaves the
    operator's own solve workspace at zero bytes, and still matches the oracle-checked
    rs_solve computed afterwards."""
    import torch
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    n, leaf, eps = 32, 8, 1e-10
    tree = P.rs_build_tree(W.grid_points(n), leaf)
    op = P.rs_factor(tree, eps=eps)
    try:
        assert P.rs_op_stats(op)["bytes_workspace"] == 0
        f = _dev(W.rhs_normal(n, 21, nrhs=3))
        x_na = torch.full_like(f, np.nan)
        for _ in range(2):
            P.rs_solve_noalloc(op, f, 3, x_na, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert P.rs_op_stats(op)["bytes_workspace"] == 0
        x_ref = torch.empty_like(f)
        P.rs_solve(op, f, 3, x_ref, torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert P.rs_op_stats(op)["bytes_workspace"] > 0
        assert _rel(x_na.cpu().numpy(), x_ref.cpu().numpy()) <= SOL_TOL
    finally:
        P.rs_free(op)
        P.rs_free_tree(tree)
