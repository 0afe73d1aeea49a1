"""Failure detection without a GPU fault: a device-side wait that nothing will ever release
(one CTA at the group barrier of the cooperative kernels, with a target of two arrivals) must
end by its iteration limit, report RS_E_TIMEOUT to the host, and leave the CUDA context usable
for the next factorization and solve."""
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


@pytest.mark.parametrize("limit", [1, 1000, 100000])
def test_wait_ends_by_its_limit_and_context_survives(rs, oracle_mod, limit):
    with pytest.raises(rs.RsError) as e:
        rs.rs_wait_check(limit)
    assert e.value.code == rs.RS_E_TIMEOUT
    n, leaf = 16, 4
    S = rs.Solver(W.grid_points(n), leaf, eps=1e-10)
    f = W.rhs_uniform(n, 1)
    xo = oracle_mod.Factorization(n, leaf, 1e-10).solve(f)
    assert np.linalg.norm(S.solve(f) - xo) <= 1e-9 * np.linalg.norm(xo)


def test_limit_must_be_positive(rs):
    with pytest.raises(rs.RsError) as e:
        rs.rs_wait_check(0)
    assert e.value.code == rs.RS_E_INVALID
