"""Serving (S11): continuous batching of inverse applies over resident factorizations.

Requests of different operators and RHS counts are admitted while others run, share launches
tick by tick, and must give the same result as rs_solve alone (the same per-request
arithmetic: identical bits expected, 1e-13 asserted), and every served result must match
the oracle's inverse apply within the 1e-9 FP64 solution tolerance.  Admission respects the memory budget,
and host-side failures (bad arguments, an operator freed while referenced, a request that
can never fit) are reported as error codes, with no GPU fault involved.
"""
import time

import numpy as np
import pytest

from paper_1303_5466_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SPECS = [(32, 8), (64, 8), (64, 16)]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    from paper_1303_5466_gb300 import build as B
    B.build()
    import paper_1303_5466_gb300 as P
    trees, ops = [], []
    for n, leaf in SPECS:
        t = P.rs_build_tree(W.grid_points(n), leaf)
        trees.append(t)
        ops.append(P.rs_factor(t, eps=1e-10))
    yield P, ops
    for o in ops:
        P.rs_free(o)
    for t in trees:
        P.rs_free_tree(t)


def _requests(count, seed, max_rhs=8):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        k = int(rng.integers(0, len(SPECS)))
        nrhs = int(rng.integers(1, max_rhs + 1))
        n = SPECS[k][0]
        out.append((k, nrhs, rng.standard_normal((nrhs, n * n))))
    return out


def _alone(P, ops, reqs):
    import torch
    st = torch.cuda.current_stream()
    xs = []
    for k, nrhs, F in reqs:
        f = torch.from_numpy(F).cuda()
        x = torch.empty_like(f)
        P.rs_solve(ops[k], f, nrhs, x, st)
        torch.cuda.synchronize()
        xs.append(x.cpu().numpy())
    return xs


def test_results_equal_alone_and_in_the_mix(env):
    import torch
    P, ops = env
    reqs = _requests(40, 3)
    ref = _alone(P, ops, reqs)
    srv = P.rs_server_create(ops, 256 << 20, max_inflight=16)
    try:
        fs = [torch.from_numpy(F).cuda() for _, _, F in reqs]
        xs = [torch.full_like(f, np.nan) for f in fs]
        torch.cuda.synchronize()
        tickets = []
        for i, (k, nrhs, _) in enumerate(reqs):
            tickets.append(P.rs_server_submit(srv, k, fs[i], nrhs, xs[i]))
            if i == 19:
                time.sleep(0.01)          # the second half arrives while the first runs
        P.rs_server_drain(srv, 120.0)
        done = P.rs_server_poll(srv, 1024)
        assert sorted(done) == sorted(tickets)
        st = P.rs_server_stats(srv)
        assert st["completed"] == 40 and st["rhs_completed"] == sum(r[1] for r in reqs)
        assert st["peak_inflight"] > 1          # requests really shared ticks
        worst = 0.0
        for x, r in zip(xs, ref):
            got = x.cpu().numpy()
            worst = max(worst, float(np.abs(got - r).max() / np.abs(r).max()))
        assert worst <= 1e-13, worst
        lat = P.rs_server_latencies(srv)
        assert len(lat) == 40 and (lat > 0).all()
    finally:
        P.rs_server_free(srv)


def test_served_results_match_oracle(env, oracle_mod):
    """Every request served in the mix (several operators, 1-64 right-hand sides, arriving while
    others run) is compared with the oracle's inverse apply of the same operator (Algorithm 6
    over the oracle's own factorization) within the 1e-9 FP64 solution tolerance."""
    import torch
    P, ops = env
    orc = [oracle_mod.Factorization(n, leaf, 1e-10) for n, leaf in SPECS]
    reqs = _requests(30, 11, max_rhs=64)
    srv = P.rs_server_create(ops, 512 << 20, max_inflight=16)
    try:
        fs = [torch.from_numpy(F).cuda() for _, _, F in reqs]
        xs = [torch.full_like(f, np.nan) for f in fs]
        torch.cuda.synchronize()
        for i, (k, nrhs, _) in enumerate(reqs):
            P.rs_server_submit(srv, k, fs[i], nrhs, xs[i])
            if i == 14:
                time.sleep(0.01)          # the second half arrives while the first runs
        P.rs_server_drain(srv, 120.0)
        torch.cuda.synchronize()
        assert P.rs_server_stats(srv)["peak_inflight"] > 1
        for (k, nrhs, F), x in zip(reqs, xs):
            got = x.cpu().numpy()                       # (nrhs, N): column-major N x nrhs
            want = orc[k].solve(np.ascontiguousarray(F.T)).reshape(-1, nrhs).T
            for c in range(nrhs):
                rel = np.linalg.norm(got[c] - want[c]) / np.linalg.norm(want[c])
                assert rel <= 1e-9, (k, nrhs, c, rel)
    finally:
        P.rs_server_free(srv)


def test_memory_budget_limits_admission(env):
    import torch
    P, ops = env
    reqs = [(1, 4, F) for (_, _, F) in _requests(10, 5, max_rhs=1)]
    n = SPECS[1][0]
    reqs = [(1, 4, np.random.default_rng(i).standard_normal((4, n * n))) for i in range(10)]
    ref = _alone(P, ops, reqs)
    # workspace of one 4-RHS request on the 64 x 64 operator is below 2 MiB: room for two
    srv = P.rs_server_create(ops, 4 << 20, max_inflight=16)
    try:
        fs = [torch.from_numpy(F).cuda() for _, _, F in reqs]
        xs = [torch.empty_like(f) for f in fs]
        torch.cuda.synchronize()
        for i, (k, nrhs, _) in enumerate(reqs):
            P.rs_server_submit(srv, k, fs[i], nrhs, xs[i])
        P.rs_server_drain(srv, 120.0)
        st = P.rs_server_stats(srv)
        assert st["completed"] == 10 and 1 <= st["peak_inflight"] <= 2
        for x, r in zip(xs, ref):
            assert np.abs(x.cpu().numpy() - r).max() <= 1e-13 * np.abs(r).max()
    finally:
        P.rs_server_free(srv)


def test_host_side_failures(env):
    import torch
    P, ops = env
    srv = P.rs_server_create(ops, 1 << 20, max_inflight=4)
    try:
        f = torch.zeros((1, 64 * 64), dtype=torch.float64, device="cuda")
        x = torch.zeros_like(f)
        with pytest.raises(P.RsError) as e:
            P.rs_server_submit(srv, 7, f, 1, x)            # no such operator
        assert e.value.code == P.RS_E_INVALID
        big = torch.zeros((64, 64 * 64), dtype=torch.float64, device="cuda")
        with pytest.raises(P.RsError) as e:
            P.rs_server_submit(srv, 1, big, 64, torch.zeros_like(big))   # never fits 1 MiB
        assert e.value.code == P.RS_E_NOMEM
        with pytest.raises(P.RsError) as e:
            P.rs_free(ops[0])                               # still referenced by the server
        assert e.value.code == P.RS_E_INVALID
        with pytest.raises(P.RsError):
            P.rs_server_submit(srv, 0, np.zeros(32 * 32), 1, np.zeros(32 * 32))   # host buffers
    finally:
        P.rs_server_free(srv)


def test_translation_invariant_operators_in_the_mix(env):
    """Operators factored in the translation-invariant modes (their boxes share one stored set
    of blocks per class or per level) are served like any other: same results as rs_solve."""
    import torch
    P, _ = env
    trees, ops = [], []
    try:
        for mode, (n, leaf) in zip((1, 2, 0), SPECS):
            t = P.rs_build_tree(W.grid_points(n), leaf)
            trees.append(t)
            o = P.rs_opts_default()
            o.translation_invariant = mode
            ops.append(P.rs_factor(t, eps=1e-10, opts=o))
        reqs = _requests(24, 5)
        ref = _alone(P, ops, reqs)
        srv = P.rs_server_create(ops, 256 << 20, max_inflight=8)
        try:
            fs = [torch.from_numpy(F).cuda() for _, _, F in reqs]
            xs = [torch.full_like(f, np.nan) for f in fs]
            torch.cuda.synchronize()
            for i, (k, nrhs, _) in enumerate(reqs):
                P.rs_server_submit(srv, k, fs[i], nrhs, xs[i])
            P.rs_server_drain(srv, 120.0)
            torch.cuda.synchronize()
            for i in range(len(reqs)):
                x = xs[i].cpu().numpy()
                assert np.linalg.norm(x - ref[i]) <= 1e-13 * np.linalg.norm(ref[i])
        finally:
            P.rs_server_free(srv)
    finally:
        for o in ops:
            P.rs_free(o)
        for t in trees:
            P.rs_free_tree(t)
