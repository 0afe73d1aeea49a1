"""ctypes wrapper of the C oracle (rs_oracle.c).  Test infrastructure only.

The oracle follows the paper step by step (Algorithm 1 with the E formula of Algorithm 2,
the inverse apply of Algorithm 6, proxy-accelerated IDs of Sec. 2.2).  It shares no code
with the CUDA library.  ``build()`` compiles it with gcc; ``-ffp-contract=off`` keeps its
rounding the same on x86 and Arm hosts.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, f) for f in ("rs_oracle.c", "ro_core.inc", "rs_oracle.h")]
_LIB = os.path.join(_HERE, "librs_oracle.so")
_lib = None

LAPLACE, HELMHOLTZ = 0, 1


def build(force=False, plant=0, out=None):
    """Compile librs_oracle.so next to the sources if it is missing or stale.

    ``plant`` != 0 builds a copy with a deliberate mistake (see ro_core.inc) into ``out``;
    the tests use it to show that the pins catch such a mistake."""
    target = out or _LIB
    stale = not os.path.exists(target) or any(os.path.getmtime(s) > os.path.getmtime(target) for s in _SRC)
    if force or stale or plant:
        tmp = target + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-ffp-contract=off", "-fopenmp",
               "-DRO_PLANT=%d" % plant, "-o", tmp, os.path.join(_HERE, "rs_oracle.c"), "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, target)
    return target


class _Opts(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa", C.c_double), ("proxy_points", C.c_int),
                ("proxy_radius_factor", C.c_double), ("near_all", C.c_int),
                ("threads", C.c_int), ("max_levels", C.c_int)]


def load(path):
    """Load an oracle build at ``path`` (the default build or a planted-mistake copy)."""
    L = C.CDLL(path)
    _declare(L)
    return L


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = load(_LIB)
    return _lib


def use(L):
    """Route this module's calls to another oracle build (tests of planted mistakes)."""
    global _lib
    old, _lib = _lib, L
    return old


def _declare(L):
    dp, ip, i64p = C.POINTER(C.c_double), C.POINTER(C.c_int), C.POINTER(C.c_int64)
    L.ro_opts_default.argtypes = [C.POINTER(_Opts)]
    L.ro_laplace_cell_integral.restype = C.c_double
    L.ro_laplace_cell_integral.argtypes = [C.c_double]
    L.ro_helmholtz_cell_integral.argtypes = [C.c_double, C.c_double, C.c_int, dp, dp]
    L.ro_gauss_legendre.argtypes = [C.c_int, dp, dp]
    L.ro_id.argtypes = [C.c_int, dp, C.c_int, C.c_int, C.c_double, ip, ip, dp]
    L.ro_inverse.argtypes = [C.c_int, dp, C.c_int, dp]
    L.ro_factor.argtypes = [C.c_int, C.c_int, dp, dp, C.c_double, C.POINTER(_Opts), C.POINTER(C.c_void_p)]
    L.ro_solve.argtypes = [C.c_void_p, dp, C.c_int, dp]
    L.ro_free.argtypes = [C.c_void_p]
    L.ro_depth.argtypes = [C.c_void_p]
    L.ro_box_sizes.argtypes = [C.c_void_p, C.c_int, C.c_int, ip, ip, ip, ip]
    for nm in ("ro_box_active", "ro_box_skel", "ro_box_near"):
        getattr(L, nm).argtypes = [C.c_void_p, C.c_int, C.c_int, i64p]
    for nm in ("ro_box_T", "ro_box_Finv", "ro_box_E"):
        getattr(L, nm).argtypes = [C.c_void_p, C.c_int, C.c_int, dp]
    L.ro_root_size.argtypes = [C.c_void_p]
    L.ro_root_inv.argtypes = [C.c_void_p, dp]
    L.ro_matvec.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, dp, C.c_int, dp]
    L.ro_matvec_rows.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, dp, C.c_int, i64p, C.c_int, dp]
    L.ro_entry.argtypes = [C.c_int, C.c_int, C.c_double, dp, dp, C.c_int64, C.c_int64, dp, dp]


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _f64(a, n=None):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


def laplace_cell_integral(h):
    """Integral of log|y - x| over the h x h cell centred at x."""
    return lib().ro_laplace_cell_integral(h)


def helmholtz_cell_integral(h, kappa, nodes=32):
    """Integral of H0^(1)(kappa |y - x|) over the h x h cell centred at x (complex)."""
    re, im = C.c_double(), C.c_double()
    lib().ro_helmholtz_cell_integral(h, kappa, nodes, C.byref(re), C.byref(im))
    return complex(re.value, im.value)


def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    lib().ro_gauss_legendre(n, _dp(x), _dp(w))
    return x, w


def interp_decomp(Y, eps):
    """ID of Y (r x m, real or complex): returns (k, perm, T) with T in pivot order."""
    cplx = np.iscomplexobj(Y)
    Y = np.ascontiguousarray(Y, dtype=np.complex128 if cplx else np.float64)
    r, m = Y.shape
    perm = np.zeros(m, dtype=np.int32)
    T = np.zeros(max(m * m, 1), dtype=Y.dtype)
    k = C.c_int()
    rc = lib().ro_id(int(cplx), Y.ctypes.data_as(C.POINTER(C.c_double)), r, m, eps, C.byref(k),
                     perm.ctypes.data_as(C.POINTER(C.c_int)), T.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise RuntimeError("ro_id failed: %d" % rc)
    k = k.value
    return k, perm, T[: k * (m - k)].reshape(k, m - k)


def inverse(A):
    cplx = np.iscomplexobj(A)
    A = np.ascontiguousarray(A, dtype=np.complex128 if cplx else np.float64)
    m = A.shape[0]
    out = np.zeros_like(A)
    rc = lib().ro_inverse(int(cplx), A.ctypes.data_as(C.POINTER(C.c_double)), m,
                          out.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise np.linalg.LinAlgError("ro_inverse failed: %d" % rc)
    return out


class Factorization:
    """Dense-block HSS inverse built by ro_factor (Algorithm 1)."""

    def __init__(self, n, leaf, eps, a=None, b=None, kind=LAPLACE, kappa=0.0, proxy_points=64,
                 proxy_radius_factor=1.5, near_all=False, threads=0, max_levels=0):
        L = self._L = lib()
        o = _Opts()
        L.ro_opts_default(C.byref(o))
        o.kind, o.kappa, o.proxy_points = kind, kappa, proxy_points
        o.proxy_radius_factor, o.near_all, o.threads = proxy_radius_factor, int(near_all), threads
        o.max_levels = max_levels
        self.n, self.leaf, self.eps, self.kind, self.kappa = n, leaf, eps, kind, kappa
        N = n * n
        self.a, self.b = _f64(a, N), _f64(b, N)
        p = C.c_void_p()
        rc = L.ro_factor(n, leaf, _dp(self.a), _dp(self.b), eps, C.byref(o), C.byref(p))
        if rc:
            raise RuntimeError("ro_factor failed: %d" % rc)
        self._p = p
        self.depth = L.ro_depth(p)

    def __del__(self):
        if getattr(self, "_p", None):
            self._L.ro_free(self._p)
            self._p = None

    @property
    def cplx(self):
        return self.kind == HELMHOLTZ

    def solve(self, f):
        """x = A^{-1} f by Algorithm 6.  f: (N,) or (N, nrhs) in grid order."""
        N = self.n * self.n
        f = np.asarray(f)
        one = f.ndim == 1
        F = f.reshape(N, -1)
        dt = np.complex128 if self.cplx else np.float64
        Fc = np.asfortranarray(F.astype(dt))
        X = np.zeros_like(Fc)
        rc = self._L.ro_solve(self._p, Fc.ctypes.data_as(C.POINTER(C.c_double)), F.shape[1],
                            X.ctypes.data_as(C.POINTER(C.c_double)))
        if rc:
            raise RuntimeError("ro_solve failed: %d" % rc)
        return X[:, 0] if one else np.ascontiguousarray(X)

    def sizes(self, level, box):
        m, k, r, nn = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        if self._L.ro_box_sizes(self._p, level, box, C.byref(m), C.byref(k), C.byref(r), C.byref(nn)):
            raise IndexError((level, box))
        return m.value, k.value, r.value, nn.value

    def _ints(self, fn, level, box, cnt):
        out = np.zeros(max(cnt, 1), dtype=np.int64)
        getattr(self._L, fn)(self._p, level, box, out.ctypes.data_as(C.POINTER(C.c_int64)))
        return out[:cnt]

    def _mat(self, fn, level, box, shape):
        dt = np.complex128 if self.cplx else np.float64
        out = np.zeros(max(shape[0] * shape[1], 1), dtype=dt)
        getattr(self._L, fn)(self._p, level, box, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out[: shape[0] * shape[1]].reshape(shape)

    def active(self, level, box):
        return self._ints("ro_box_active", level, box, self.sizes(level, box)[0])

    def skel(self, level, box):
        return self._ints("ro_box_skel", level, box, self.sizes(level, box)[1])

    def near(self, level, box):
        return self._ints("ro_box_near", level, box, self.sizes(level, box)[3])

    def T(self, level, box):
        m, k, _, _ = self.sizes(level, box)
        return self._mat("ro_box_T", level, box, (k, m - k))

    def Finv(self, level, box):
        m = self.sizes(level, box)[0]
        return self._mat("ro_box_Finv", level, box, (m, m))

    def E(self, level, box):
        k = self.sizes(level, box)[1]
        return self._mat("ro_box_E", level, box, (k, k))

    def root_inv(self):
        m = self._L.ro_root_size(self._p)
        dt = np.complex128 if self.cplx else np.float64
        out = np.zeros(m * m, dtype=dt)
        self._L.ro_root_inv(self._p, out.ctypes.data_as(C.POINTER(C.c_double)))
        return out.reshape(m, m)


def matvec(n, x, a=None, b=None, kind=LAPLACE, kappa=0.0):
    """Brute-force y = A x over all N^2 entries (x: (N,) or (N, nrhs), grid order)."""
    N = n * n
    x = np.asarray(x)
    one = x.ndim == 1
    dt = np.complex128 if kind == HELMHOLTZ else np.float64
    X = np.asfortranarray(x.reshape(N, -1).astype(dt))
    Y = np.zeros_like(X)
    a, b = _f64(a, N), _f64(b, N)
    rc = lib().ro_matvec(n, kind, kappa, _dp(a), _dp(b), X.ctypes.data_as(C.POINTER(C.c_double)), X.shape[1],
                         Y.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise RuntimeError("ro_matvec failed")
    return Y[:, 0] if one else np.ascontiguousarray(Y)


def matvec_rows(n, x, rows, a=None, b=None, kind=LAPLACE, kappa=0.0):
    """Rows `rows` of A x, computed entry by entry.  Returns (len(rows),) or (len(rows), nrhs)."""
    N = n * n
    x = np.asarray(x)
    one = x.ndim == 1
    dt = np.complex128 if kind == HELMHOLTZ else np.float64
    X = np.asfortranarray(x.reshape(N, -1).astype(dt))
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    Y = np.zeros((len(rows), X.shape[1]), dtype=dt, order="F")
    a, b = _f64(a, N), _f64(b, N)
    rc = lib().ro_matvec_rows(n, kind, kappa, _dp(a), _dp(b), X.ctypes.data_as(C.POINTER(C.c_double)), X.shape[1],
                              rows.ctypes.data_as(C.POINTER(C.c_int64)), len(rows),
                              Y.ctypes.data_as(C.POINTER(C.c_double)))
    if rc:
        raise RuntimeError("ro_matvec_rows failed")
    return Y[:, 0] if one else np.ascontiguousarray(Y)


def entry(n, g, gp, a=None, b=None, kind=LAPLACE, kappa=0.0):
    N = n * n
    a, b = _f64(a, N), _f64(b, N)
    re, im = C.c_double(), C.c_double()
    lib().ro_entry(n, kind, kappa, _dp(a), _dp(b), g, gp, C.byref(re), C.byref(im))
    return complex(re.value, im.value) if kind == HELMHOLTZ else re.value


def solve_refined(F, f, tol=1e-12, max_iter=30):
    """Iterative refinement of Sec. 5.3/5.4 around the oracle factorization F: x = 0, then
    x += F.solve(r), r = f - A x (brute-force matvec) until |r| / |f| <= tol.
    Returns (x, relative residual, solves made)."""
    f = np.asarray(f)
    x = np.zeros_like(f, dtype=np.complex128 if F.cplx else np.float64)
    r = f.astype(x.dtype)
    nf = np.linalg.norm(f)
    rel = 1.0
    for it in range(1, max_iter + 1):
        x = x + F.solve(r)
        r = f - matvec(F.n, x, a=F.a, b=F.b, kind=F.kind, kappa=F.kappa)
        rel = np.linalg.norm(r) / nf
        if rel <= tol:
            return x, rel, it
    return x, rel, max_iter
