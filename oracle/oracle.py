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
                ("threads", C.c_int), ("max_levels", C.c_int), ("k_cut", C.c_int), ("hss_leaf", C.c_int),
                ("hss_eps", C.c_double), ("ti", C.c_int)]


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
    L.ro_fwd_apply.argtypes = [C.c_void_p, dp, C.c_int, dp]
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
    L.ro_hss1d_build.argtypes = [C.c_int, dp, C.c_int, ip, C.c_int, C.c_double, C.POINTER(C.c_void_p)]
    L.ro_hss1d_apply.argtypes = [C.c_void_p, dp, C.c_int, dp]
    L.ro_hss1d_depth.argtypes = [C.c_void_p]
    L.ro_hss1d_node.argtypes = [C.c_void_p, C.c_int, C.c_int, ip, ip, ip, ip, ip, dp]
    L.ro_hss1d_entries.argtypes = [C.c_void_p]
    L.ro_hss1d_entries.restype = C.c_int64
    L.ro_hss1d_free.argtypes = [C.c_void_p]
    L.ro_box_hss.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.ro_box_hss.restype = C.c_void_p
    L.ro_box_lr_rank.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int]
    L.ro_box_order.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, ip]
    L.ro_compressed_entries.argtypes = [C.c_void_p, i64p]
    L.ro_compressed_entries.restype = C.c_int64


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


class HSS1D:
    """HSS1D form (Sec. 3.2) of an explicit square matrix built by ro_hss1d_build."""

    def __init__(self, M, order=None, leaf=64, eps=1e-10, _handle=None, _owner=None):
        L = self._L = lib()
        if _handle is not None:
            self._p, self._own, self._owner = _handle, False, _owner
        else:
            self.cplx = np.iscomplexobj(M)
            M = np.ascontiguousarray(M, dtype=np.complex128 if self.cplx else np.float64)
            n = M.shape[0]
            o = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
            p = C.c_void_p()
            rc = L.ro_hss1d_build(int(self.cplx), M.ctypes.data_as(C.POINTER(C.c_double)), n,
                                  None if o is None else o.ctypes.data_as(C.POINTER(C.c_int)), leaf, eps,
                                  C.byref(p))
            if rc:
                raise RuntimeError("ro_hss1d_build failed: %d" % rc)
            self._p, self._own = p, True
        self.depth = L.ro_hss1d_depth(self._p)

    def __del__(self):
        if getattr(self, "_own", False) and getattr(self, "_p", None):
            self._L.ro_hss1d_free(self._p)
            self._p = None

    def node(self, level, j):
        """(lo, hi, a, k, skeleton rows, T) of node (level, j)."""
        lo, hi, a, k = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        if self._L.ro_hss1d_node(self._p, level, j, C.byref(lo), C.byref(hi), C.byref(a), C.byref(k), None, None):
            raise IndexError((level, j))
        sk = np.zeros(max(k.value, 1), dtype=np.int32)
        dt = np.complex128 if self.cplx else np.float64
        T = np.zeros(max(k.value * (a.value - k.value), 1), dtype=dt)
        self._L.ro_hss1d_node(self._p, level, j, None, None, None, None, sk.ctypes.data_as(C.POINTER(C.c_int)),
                              T.ctypes.data_as(C.POINTER(C.c_double)))
        return (lo.value, hi.value, a.value, k.value, sk[: k.value],
                T[: k.value * (a.value - k.value)].reshape(k.value, a.value - k.value))

    def entries(self):
        return self._L.ro_hss1d_entries(self._p)

    def apply(self, x):
        x = np.asarray(x)
        one = x.ndim == 1
        dt = np.complex128 if self.cplx else np.float64
        X = np.ascontiguousarray(x.reshape(x.shape[0], -1), dtype=dt)
        Y = np.zeros_like(X)
        if self._L.ro_hss1d_apply(self._p, X.ctypes.data_as(C.POINTER(C.c_double)), X.shape[1],
                                  Y.ctypes.data_as(C.POINTER(C.c_double))):
            raise RuntimeError("ro_hss1d_apply failed")
        return Y[:, 0] if one else Y


class Factorization:
    """Dense-block HSS inverse built by ro_factor (Algorithm 1)."""

    def __init__(self, n, leaf, eps, a=None, b=None, kind=LAPLACE, kappa=0.0, proxy_points=64,
                 proxy_radius_factor=1.5, near_all=False, threads=0, max_levels=0, k_cut=0, hss_leaf=64,
                 hss_eps=0.0, ti=False):
        L = self._L = lib()
        o = _Opts()
        L.ro_opts_default(C.byref(o))
        o.kind, o.kappa, o.proxy_points = kind, kappa, proxy_points
        o.proxy_radius_factor, o.near_all, o.threads = proxy_radius_factor, int(near_all), threads
        o.max_levels, o.k_cut, o.hss_leaf, o.hss_eps = max_levels, k_cut, hss_leaf, hss_eps
        o.ti = int(ti)
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

    def fwd_apply(self, x):
        """y = A x through the HSS form the factorization's IDs define (O(N), error ~ eps).
        x: (N,) or (N, nrhs) in grid order."""
        N = self.n * self.n
        x = np.asarray(x)
        one = x.ndim == 1
        X = x.reshape(N, -1)
        dt = np.complex128 if self.cplx else np.float64
        Xc = np.asfortranarray(X.astype(dt))
        Y = np.zeros_like(Xc)
        rc = self._L.ro_fwd_apply(self._p, Xc.ctypes.data_as(C.POINTER(C.c_double)), X.shape[1],
                                  Y.ctypes.data_as(C.POINTER(C.c_double)))
        if rc:
            raise RuntimeError("ro_fwd_apply failed: %d" % rc)
        return Y[:, 0] if one else np.ascontiguousarray(Y)

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

    def box_hss(self, level, box, which):
        """HSS1D form of phi^{sk} (which 0), phi^{rs} (1) or E (2) of a compressed box, or None."""
        p = self._L.ro_box_hss(self._p, level, box, which)
        if not p:
            return None
        h = HSS1D(None, _handle=C.c_void_p(p), _owner=self)
        h.cplx = self.cplx
        return h

    def lr_rank(self, level, box, which):
        """Rank of the low-rank phi^{s<-r} (0), phi^{r<-s} (1) or T (2) of a compressed box (-1: dense)."""
        return self._L.ro_box_lr_rank(self._p, level, box, which)

    def order(self, level, box, which):
        """Sec. 3.1 order: skeleton indices cyclically (which 0) or residual indices along the interface (1)."""
        m, k, _, _ = self.sizes(level, box)
        cnt = k if which == 0 else m - k
        out = np.zeros(max(cnt, 1), dtype=np.int32)
        if self._L.ro_box_order(self._p, level, box, which, out.ctypes.data_as(C.POINTER(C.c_int))):
            raise IndexError((level, box))
        return out[:cnt]

    def compressed_entries(self):
        """(stored scalars of the compressed forms, scalars the same blocks take densely)."""
        d = C.c_int64()
        c = self._L.ro_compressed_entries(self._p, C.byref(d))
        return c, d.value

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
