"""Pins of the oracle's forward apply: y = A x through the HSS form that the factorization's
IDs define (off-diagonal blocks L_i A(sk_i, sk_j) R_j, nested level by level; Sec. 2.2 with the
telescoping form of Eq. 2.9).  Checked against the brute-force matvec (exact without
truncation, within 10 eps with it), and against the factorization itself: the factor is the
exact inverse of this compressed operator, so applying it to A^{-1} f returns f to rounding
whatever eps is.  The planted mistake 9 (T dropped from the upward pass) fails the
brute-force pin in test_oracle.py."""
import numpy as np
import pytest

import _dense as D
from paper_1303_5466_gb300 import workloads as W


def _rel(x, y):
    return np.linalg.norm(x - y) / np.linalg.norm(y)


def test_fwd_exact_without_truncation(oracle_mod):
    n = 8
    F = oracle_mod.Factorization(n, 2, 0.0)
    x = W.rhs_normal(n, 1, nrhs=3)
    assert _rel(F.fwd_apply(x), D.laplace(n) @ x) <= 1e-14


@pytest.mark.parametrize("n,leaf,eps", [(16, 4, 1e-10), (32, 8, 1e-10), (64, 8, 1e-10), (64, 16, 1e-5)])
def test_fwd_within_eps_of_brute_force(oracle_mod, n, leaf, eps):
    a = W.coeff_a_batched(n)
    F = oracle_mod.Factorization(n, leaf, eps, a=a)
    x = W.rhs_normal(n, 2, nrhs=2)
    assert _rel(F.fwd_apply(x), oracle_mod.matvec(n, x, a=a)) <= 10 * eps


@pytest.mark.parametrize("n,leaf,eps", [(16, 4, 1e-10), (64, 8, 1e-10), (64, 16, 1e-5)])
def test_factor_inverts_the_hss_form(oracle_mod, n, leaf, eps):
    F = oracle_mod.Factorization(n, leaf, eps)
    f = W.rhs_uniform(n, 4)
    assert _rel(F.fwd_apply(F.solve(f)), f) <= 1e-12


def test_fwd_helmholtz(oracle_mod):
    """The IDs are taken on the symmetric form A_s = S^{-1} A S (S = diag(kappa sqrt b)), so the
    eps bound holds there: with b = 1 directly, with the Gaussian b (S spanning four decades)
    on S^{-1} y."""
    n, leaf, kappa = 32, 8, 25.0
    x = W.rhs_plane_wave(n, kappa)
    F1 = oracle_mod.Factorization(n, leaf, 1e-10, kind=1, kappa=kappa)
    assert _rel(F1.fwd_apply(x), oracle_mod.matvec(n, x, kind=1, kappa=kappa)) <= 10 * 1e-10
    b = W.coeff_b_gaussian(n)
    s = kappa * np.sqrt(b)
    F = oracle_mod.Factorization(n, leaf, 1e-10, kind=1, kappa=kappa, b=b)
    y, yr = F.fwd_apply(x), oracle_mod.matvec(n, x, b=b, kind=1, kappa=kappa)
    assert _rel(y / s, yr / s) <= 10 * 1e-10
    assert _rel(F.fwd_apply(F.solve(x)), x) <= 1e-11


def test_fwd_translation_invariant(oracle_mod):
    n, leaf = 32, 8
    F = oracle_mod.Factorization(n, leaf, 1e-10, ti=True)
    x = W.rhs_normal(n, 6)
    assert _rel(F.fwd_apply(x), D.laplace(n) @ x) <= 1e-9
    assert _rel(F.fwd_apply(F.solve(x)), x) <= 1e-12


def test_fwd_refuses_compressed_and_partial(oracle_mod):
    n = 32
    Fk = oracle_mod.Factorization(n, 8, 1e-10, k_cut=16)
    with pytest.raises(RuntimeError):
        Fk.fwd_apply(np.ones(n * n))
    Fp = oracle_mod.Factorization(n, 8, 1e-10, max_levels=2)
    with pytest.raises(RuntimeError):
        Fp.fwd_apply(np.ones(n * n))
