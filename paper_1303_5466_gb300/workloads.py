"""Seeded synthetic inputs for the solver and its tests.

This module only draws inputs: grid points, coefficient fields and right-hand sides.  It
holds none of the solver's arithmetic, so the CUDA library and the CPU oracle can both be
fed from it.  Every generator is deterministic given its seed.

Workloads (all on the cell-centre grid x = ((i1+1/2)h, (i2+1/2)h) of [0,1]^2, h = 1/n,
grid order g = i1 + n*i2):
  laplace_small   n=64,   leaf 8,  eps 1e-10, a = 1,                      f ~ U[-1,1]  (seed 0)
  laplace_batched n=512,  leaf 16, eps 1e-10, a = 1 + 0.5 sin(2 pi x1) cos(2 pi x2),
                                                                           4 RHS ~ N(0,1) (seed 1)
  laplace_mixed   n=1024, leaf 16, eps 1e-6 (FP32 factor) + FP64 refinement, f ~ U[-1,1] (seed 2)
  serving         n = 128, 256, 512, leaf 16, eps 1e-10; Poisson stream of 10k requests (seed 3)
  helmholtz_ls    n=256,  leaf 16, kappa 25, b = exp(-40 |x - (1/2,1/2)|^2), f = exp(i kappa x1)
  helmholtz_ls_plateau  n=256, leaf 16, kappa 25, the test problem's b of Sec. 5.4 (a plateau
                  b = 1 with a tanh fall-off at the boundary; coeff_b_plateau), f = exp(i kappa x1):
                  the iterative solver with the b = 1 preconditioner
"""
import numpy as np

WORKLOADS = {
    "laplace_small": dict(n=64, leaf=8, eps=1e-10, nrhs=1, seed=0),
    "laplace_batched": dict(n=512, leaf=16, eps=1e-10, nrhs=4, seed=1),
    "laplace_mixed": dict(n=1024, leaf=16, eps=1e-6, nrhs=1, seed=2),
    # a quarter-size copy of laplace_batched for profiling runs (same leaf, eps, a, RHS recipe)
    "laplace_n256": dict(n=256, leaf=16, eps=1e-10, nrhs=4, seed=1),
    "helmholtz_ls": dict(n=256, leaf=16, eps=1e-5, nrhs=1, seed=None, kappa=25.0),
    "helmholtz_ls_plateau": dict(n=256, leaf=16, eps=1e-10, nrhs=1, seed=None, kappa=25.0),
}


def grid_points(n):
    """(N, 2) float64 cell centres in grid order g = i1 + n*i2."""
    h = 1.0 / n
    i = (np.arange(n, dtype=np.float64) + 0.5) * h
    x1 = np.tile(i, n)
    x2 = np.repeat(i, n)
    return np.stack([x1, x2], axis=1)


def coeff_a_batched(n):
    """a(x) = 1 + 0.5 sin(2 pi x1) cos(2 pi x2) on the grid (the batched Laplace workload)."""
    p = grid_points(n)
    return 1.0 + 0.5 * np.sin(2 * np.pi * p[:, 0]) * np.cos(2 * np.pi * p[:, 1])


def coeff_b_gaussian(n, width=40.0):
    """b(x) = exp(-width |x - (1/2, 1/2)|^2) on the grid (the Lippmann-Schwinger workload)."""
    p = grid_points(n)
    return np.exp(-width * ((p[:, 0] - 0.5) ** 2 + (p[:, 1] - 0.5) ** 2))


def coeff_b_plateau(n, D=20.0, e=0.1):
    """The scatterer of the Lippmann-Schwinger test problem of Sec. 5.4, without its k^2 factor
    (the kernel carries kappa^2): b = (1/4)(1 + tanh D(1 - e - |xi1|))(1 + tanh D(1 - e - |xi2|))
    with xi = 2x - 1 mapping [0,1]^2 onto the paper's [-1,1]^2.  b is 1 on most of the square and
    falls off in a layer at its boundary (D and e are not given in the paper)."""
    p = grid_points(n)
    xi1, xi2 = 2.0 * p[:, 0] - 1.0, 2.0 * p[:, 1] - 1.0
    return 0.25 * (1.0 + np.tanh(D * (1.0 - e - np.abs(xi1)))) * (1.0 + np.tanh(D * (1.0 - e - np.abs(xi2))))


def rhs_uniform(n, seed, nrhs=1):
    """f ~ U[-1, 1], (N,) for nrhs == 1 else (N, nrhs) with column c drawn c-th."""
    rng = np.random.default_rng(seed)
    N = n * n
    if nrhs == 1:
        return rng.uniform(-1.0, 1.0, N)
    return np.ascontiguousarray(rng.uniform(-1.0, 1.0, (nrhs, N)).T)


def rhs_normal(n, seed, nrhs=1):
    """f ~ N(0, 1), drawn as an (nrhs, N) block and returned as (N, nrhs)."""
    rng = np.random.default_rng(seed)
    F = rng.standard_normal((nrhs, n * n))
    return F[0].copy() if nrhs == 1 else np.ascontiguousarray(F.T)


def rhs_plane_wave(n, kappa):
    """f = exp(i kappa x1) on the grid (complex128)."""
    p = grid_points(n)
    return np.exp(1j * kappa * p[:, 0])


def shuffled(n, seed):
    """A seeded permutation of the grid order, for tests of arbitrary input order."""
    return np.random.default_rng(seed).permutation(n * n)
