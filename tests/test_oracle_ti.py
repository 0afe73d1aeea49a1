"""Pins of the oracle's translation-invariant mode (Sec. 5: with a and b constant, one set of
matrix blocks per level).  Its factorization is checked against what does not depend on it:
the dense LU solve (eps = 1e-10: within the 1e-9 bound of the FP64 path; eps = 0 on boxes the
ID cannot compress: to rounding), the structure the mode claims (every box of a level a
translate of box 0: the same sizes, skeletons shifted by the box offset, identical blocks),
the Helmholtz form against the dense complex solve, and the inputs it must refuse.  The
planted mistake 8 (template rows from box 0's own corner neighbourhood) is caught by the
dense-LU pin in test_oracle.py."""
import numpy as np
import pytest

import _dense as D
from paper_1303_5466_gb300 import workloads as W


@pytest.mark.parametrize("n,leaf", [(16, 4), (32, 8), (64, 8)])
def test_ti_matches_dense_lu(oracle_mod, n, leaf):
    F = oracle_mod.Factorization(n, leaf, 1e-10, ti=True)
    f = W.rhs_uniform(n, 0)
    xd = np.linalg.solve(D.laplace(n), f)
    assert np.linalg.norm(F.solve(f) - xd) <= 1e-9 * np.linalg.norm(xd)


def test_ti_exact_without_truncation(oracle_mod):
    n, leaf = 8, 2
    F = oracle_mod.Factorization(n, leaf, 0.0, ti=True)
    f = W.rhs_normal(n, 1, nrhs=2)
    xd = np.linalg.solve(D.laplace(n), f)
    assert np.linalg.norm(F.solve(f) - xd) <= 1e-12 * np.linalg.norm(xd)


def test_ti_boxes_are_translates(oracle_mod):
    n, leaf = 32, 4
    F = oracle_mod.Factorization(n, leaf, 1e-10, ti=True)
    for l in range(F.depth, 0, -1):
        s0 = F.sizes(l, 0)
        sk0, act0 = F.skel(l, 0), F.active(l, 0)
        T0, Fi0, E0 = F.T(l, 0), F.Finv(l, 0), F.E(l, 0)
        for j in range(1, 2 ** l):
            assert F.sizes(l, j) == s0
            act = F.active(l, j)
            shift = act[0] - act0[0]
            np.testing.assert_array_equal(act - act0, shift)
            np.testing.assert_array_equal(F.skel(l, j) - sk0, shift)
            if j in (1, 2 ** l - 1):
                np.testing.assert_array_equal(F.T(l, j), T0)
                np.testing.assert_array_equal(F.Finv(l, j), Fi0)
                np.testing.assert_array_equal(F.E(l, j), E0)


def test_ti_skeleton_covers_interior_boxes(oracle_mod):
    """The template stands for an interior box: on a grid with interior boxes at the finest
    level, its rank there equals that of an interior box of the per-box factorization."""
    n, leaf = 64, 8
    Ft = oracle_mod.Factorization(n, leaf, 1e-10, ti=True)
    Fn = oracle_mod.Factorization(n, leaf, 1e-10)
    d = Ft.depth
    ks = [Fn.sizes(d, j)[1] for j in range(2 ** d)]
    assert Ft.sizes(d, 0)[1] == max(ks)


def test_ti_helmholtz_matches_dense(oracle_mod):
    n, leaf, kappa = 32, 8, 25.0
    F = oracle_mod.Factorization(n, leaf, 1e-10, kind=1, kappa=kappa, ti=True)
    f = W.rhs_plane_wave(n, kappa)
    A = D.helmholtz(n, kappa, np.ones(n * n))
    xd = np.linalg.solve(A, f)
    assert np.linalg.norm(F.solve(f) - xd) <= 1e-9 * np.linalg.norm(xd)


def test_ti_refuses_varying_coefficients(oracle_mod):
    n = 16
    with pytest.raises(RuntimeError):
        oracle_mod.Factorization(n, 4, 1e-10, a=W.coeff_a_batched(n), ti=True)
    with pytest.raises(RuntimeError):
        oracle_mod.Factorization(n, 4, 1e-10, kind=1, kappa=10.0, b=W.coeff_b_gaussian(n), ti=True)
    with pytest.raises(RuntimeError):
        oracle_mod.Factorization(n, 4, 1e-10, ti=True, k_cut=8)
    # a constant a other than 1 is translation invariant too
    a = np.full(n * n, 2.5)
    F = oracle_mod.Factorization(n, 4, 1e-10, a=a, ti=True)
    f = W.rhs_uniform(n, 3)
    xd = np.linalg.solve(D.laplace(n, a), f)
    assert np.linalg.norm(F.solve(f) - xd) <= 1e-9 * np.linalg.norm(xd)
