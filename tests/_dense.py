"""Dense Nystrom matrices built with numpy/scipy, independently of the oracle and the library.

The diagonal comes from scipy quadrature of the kernel over the cell, not from the closed
forms the oracle uses, so a dense solve with these matrices is an independent check of
the whole discretisation (Sec. 5: A_ij = a(x_i) delta_ij + h^2 b(x_i) K(|x_i - x_j|)).
"""
import functools

import numpy as np
from scipy import integrate, special


@functools.lru_cache(maxsize=None)
def cell_integral_log(h):
    """int_{[-h/2,h/2]^2} log|y| dy by adaptive quadrature (integrable corner singularity)."""
    f = lambda y, x: 0.5 * np.log(x * x + y * y)
    v, _ = integrate.dblquad(f, 0.0, h / 2, 0.0, h / 2, epsabs=1e-15, epsrel=1e-13)
    return 4.0 * v


@functools.lru_cache(maxsize=None)
def cell_integral_h0(h, kappa):
    """int over the h x h cell of H0^(1)(kappa |y|) dy, in polar coordinates over 8 triangles."""
    def part(fn):
        g = lambda r, th: fn(kappa * r) * r
        v, _ = integrate.dblquad(g, 0.0, np.pi / 4, 0.0, lambda th: 0.5 * h / np.cos(th),
                                 epsabs=1e-15, epsrel=1e-13)
        return 8.0 * v
    return complex(part(special.j0), part(special.y0))


def grid(n):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    return np.tile(c, n), np.repeat(c, n), h


def laplace(n, a=None):
    x, y, h = grid(n)
    N = n * n
    d2 = (x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2
    np.fill_diagonal(d2, 1.0)
    A = -(h * h / (2 * np.pi)) * 0.5 * np.log(d2)
    av = np.ones(N) if a is None else np.asarray(a, float)
    A[np.arange(N), np.arange(N)] = av - cell_integral_log(h) / (2 * np.pi)
    return A


def helmholtz(n, kappa, b, a=None):
    """A = a I + kappa^2 diag(b) (i/4) H0(kappa r) h^2, with the cell integral on the diagonal."""
    x, y, h = grid(n)
    N = n * n
    r = np.sqrt((x[:, None] - x[None, :]) ** 2 + (y[:, None] - y[None, :]) ** 2)
    np.fill_diagonal(r, 1.0)
    K = 0.25j * special.hankel1(0, kappa * r) * h * h
    K[np.arange(N), np.arange(N)] = 0.25j * cell_integral_h0(h, kappa)
    av = np.ones(N) if a is None else np.asarray(a, float)
    return np.diag(av.astype(complex)) + (kappa * kappa * np.asarray(b, float))[:, None] * K


def square_log_potential(px, py):
    """int_{[0,1]^2} log|p - y| dy in closed form (antiderivative of (1/2) log(u^2 + v^2))."""
    def F(u, v):
        s = 0.0
        if u != 0.0 or v != 0.0:
            s += u * v * np.log(u * u + v * v)
        s -= 3.0 * u * v
        if u != 0.0:
            s += u * u * np.arctan(v / u)
        if v != 0.0:
            s += v * v * np.arctan(u / v)
        return 0.5 * s
    tot = 0.0
    for (u, su) in ((1.0 - px, 1), (-px, -1)):
        for (v, sv) in ((1.0 - py, 1), (-py, -1)):
            tot += su * sv * F(u, v)
    return tot
