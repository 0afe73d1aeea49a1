"""GB300-native recursive-skeletonization direct solver for 2D volume integral equations
(Corona, Martinsson & Zorin, arXiv:1303.5466).

This module is a thin ctypes binding of the C ABI in ``include/rs.h``: the functions carry the
same names and only marshal arguments.  Every floating-point step runs in the CUDA kernels of
``librs.so``; there is no CPU fallback, and importing the binding fails loudly when the
library has not been built (``python -m paper_1303_5466_gb300.build`` or
``__graft_entry__.build()``).

Vectors passed to ``rs_solve`` are N x nrhs column-major in the caller's point order: a numpy
array of shape (N,) or a Fortran-ordered (N, nrhs) array for host memory, or a torch CUDA
tensor of shape (N,) or a C-contiguous (nrhs, N) tensor for device memory.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librs.so")

RS_OK, RS_E_INVALID, RS_E_NOT_GRID, RS_E_NOMEM = 0, -1, -2, -3
RS_E_SINGULAR, RS_E_NOT_CONVERGED, RS_E_TIMEOUT, RS_E_CUDA = -4, -5, -6, -7
RS_LAPLACE, RS_HELMHOLTZ = 0, 1
RS_FP64, RS_MIXED_FP32, RS_C64_REFINED, RS_C128 = 0, 1, 2, 3
PROF_CLASSES = ("assemble_Y", "cpqr", "id_T", "assemble_F", "inv_F", "gemm_E", "inv_E", "inv_root", "solve")


class RsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("rs error %d: %s" % (code, msg))
        self.code = code


class rs_kernel(C.Structure):
    _fields_ = [("kind", C.c_int), ("kappa", C.c_double), ("b", C.POINTER(C.c_double))]


class rs_opts(C.Structure):
    _fields_ = [("proxy_points", C.c_int), ("proxy_radius_factor", C.c_double), ("precision", C.c_int),
                ("refine_tol", C.c_double), ("refine_max_iter", C.c_int), ("k_cut", C.c_int64),
                ("spin_limit", C.c_int64), ("profile", C.c_int), ("hss_leaf", C.c_int),
                ("hss_eps", C.c_double), ("solve_graph", C.c_int),
                ("per_box", C.c_int), ("spd_inverse", C.c_int), ("cpqr_variant", C.c_int),
                ("translation_invariant", C.c_int), ("sweep_panel", C.c_int), ("forward_only", C.c_int),
                ("gemm_form", C.c_int)]


class rs_stats(C.Structure):
    _fields_ = [("depth", C.c_int), ("n_side", C.c_int64), ("root_m", C.c_int64), ("bytes_factors", C.c_int64),
                ("bytes_workspace", C.c_int64), ("flops_factor", C.c_double), ("flops_solve_per_rhs", C.c_double),
                ("bytes_solve", C.c_double), ("ms_tree", C.c_double), ("ms_inverse", C.c_double),
                ("refine_iters", C.c_int), ("refine_residual", C.c_double), ("compressed_boxes", C.c_int64),
                ("bytes_compressed", C.c_int64), ("bytes_dense_replaced", C.c_int64), ("ms_compress", C.c_double),
                ("spd_fallbacks", C.c_int), ("refine_fp64_sums", C.c_int)]


class rs_tune_report(C.Structure):
    _fields_ = [("candidates", C.c_int), ("keys_set", C.c_int), ("default_factor_ms", C.c_double),
                ("tuned_factor_ms", C.c_double)]


_lib = None


def lib():
    """The loaded librs.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("librs.so is not built (%s); run paper_1303_5466_gb300.build.build()" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, dp, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int64)
        L.rs_opts_default.argtypes = [C.POINTER(rs_opts)]
        L.rs_opts_default.restype = None
        L.rs_last_error.restype = C.c_char_p
        L.rs_build_tree.argtypes = [dp, C.c_int64, C.c_int, C.POINTER(vp)]
        L.rs_free_tree.argtypes = [vp]
        L.rs_free_tree.restype = None
        L.rs_tree_info.argtypes = [vp, i64p, C.POINTER(C.c_int), i64p]
        L.rs_tree_level_sets.argtypes = [vp, C.c_int, i64p, i64p, C.c_double, i64p, i64p, i64p, i64p]
        L.rs_factor.argtypes = [vp, C.POINTER(rs_kernel), dp, C.c_double, C.POINTER(rs_opts), vp, C.POINTER(vp)]
        L.rs_solve.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.rs_fwd_apply.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.rs_wait_check.argtypes = [C.c_int64, vp]
        L.rs_fp64_probe.argtypes = [C.c_int, dp, vp]
        L.rs_bicgstab.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, C.POINTER(C.c_int),
                                  C.POINTER(C.c_double), vp]
        L.rs_free.argtypes = [vp]
        L.rs_server_create.argtypes = [C.POINTER(vp), C.c_int, C.c_size_t, C.c_int, C.POINTER(vp)]
        L.rs_server_submit.argtypes = [vp, C.c_int, vp, C.c_int64, vp, C.POINTER(C.c_uint64)]
        L.rs_server_poll.argtypes = [vp, C.POINTER(C.c_uint64), C.c_int, C.POINTER(C.c_int)]
        L.rs_server_drain.argtypes = [vp, C.c_double]
        L.rs_server_stats.argtypes = [vp, i64p, i64p, i64p, i64p, i64p]
        L.rs_server_latencies.argtypes = [vp, dp, C.c_int64, i64p]
        L.rs_server_free.argtypes = [vp]
        L.rs_server_free.restype = None
        L.rs_solve_noalloc.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.rs_residual.argtypes = [vp, vp, vp, C.c_int64, dp, vp]
        L.rs_op_stats.argtypes = [vp, C.POINTER(rs_stats)]
        L.rs_op_box_sizes.argtypes = [vp, C.c_int, C.c_int, i64p, i64p, i64p, i64p]
        L.rs_op_box_indices.argtypes = [vp, C.c_int, C.c_int, C.c_int, i64p]
        L.rs_op_box_matrix.argtypes = [vp, C.c_int, C.c_int, C.c_int, dp]
        L.rs_op_root_matrix.argtypes = [vp, dp]
        L.rs_op_profile.argtypes = [vp, C.c_int, dp, dp, dp, i64p]
        L.rs_launch_count.restype = C.c_int64
        L.rs_launch_count.argtypes = []
        L.rs_op_box_order.argtypes = [vp, C.c_int, C.c_int, C.c_int, i64p]
        L.rs_tree_box_order.argtypes = [vp, C.c_int, C.c_int, C.c_int, i64p, C.c_int64, i64p]
        L.rs_op_box_form.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_int), i64p, i64p]
        L.rs_hss1d_build.argtypes = [vp, C.c_int64, C.c_int, i64p, C.c_int, C.c_double, vp, C.POINTER(vp)]
        L.rs_hss1d_apply.argtypes = [vp, vp, C.c_int64, vp, vp]
        L.rs_hss1d_info.argtypes = [vp, C.POINTER(C.c_int), i64p, i64p]
        L.rs_hss1d_node.argtypes = [vp, C.c_int, C.c_int, i64p, i64p, i64p, i64p, i64p]
        L.rs_hss1d_free.argtypes = [vp]
        L.rs_op_profile_level.argtypes = [vp, C.c_int, C.c_int, dp]
        L.rs_autotune.argtypes = [vp, C.POINTER(rs_kernel), dp, C.c_double, C.POINTER(rs_opts), vp, C.c_char_p,
                                  C.POINTER(rs_tune_report)]
        L.rs_tune_save.argtypes = [C.c_char_p]
        L.rs_tune_load.argtypes = [C.c_char_p]
        L.rs_tune_clear.argtypes = []
        L.rs_tune_count.argtypes = []
        _lib = L
    return _lib


def _check(rc):
    if rc != RS_OK:
        raise RsError(rc, rs_last_error())
    return rc


def _dp(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _i64p(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_int64))


def rs_last_error():
    return lib().rs_last_error().decode()


def rs_opts_default():
    o = rs_opts()
    lib().rs_opts_default(C.byref(o))
    return o


def rs_build_tree(points, leaf_side):
    """points: (N, 2) float64 host array.  Returns the tree handle (c_void_p)."""
    pts = np.ascontiguousarray(points, dtype=np.float64)
    out = C.c_void_p()
    _check(lib().rs_build_tree(_dp(pts), pts.shape[0], int(leaf_side), C.byref(out)))
    return out


def rs_free_tree(tree):
    lib().rs_free_tree(tree)


def rs_tree_info(tree, N=None):
    n, d = C.c_int64(), C.c_int()
    g = np.zeros(N, dtype=np.int64) if N else None
    _check(lib().rs_tree_info(tree, C.byref(n), C.byref(d), _i64p(g)))
    return n.value, d.value, g


def rs_tree_level_sets(tree, level, child_k=None, child_skel=None, proxy_radius_factor=1.5):
    """Host bookkeeping of one level: (m, act, nnear, near) as int64 arrays."""
    nb = 1 << level
    ck = None if child_k is None else np.ascontiguousarray(child_k, dtype=np.int64)
    cs = None if child_skel is None else np.ascontiguousarray(child_skel, dtype=np.int64)
    m, nn = np.zeros(nb, np.int64), np.zeros(nb, np.int64)
    _check(lib().rs_tree_level_sets(tree, level, _i64p(ck), _i64p(cs), proxy_radius_factor, _i64p(m), None,
                                    _i64p(nn), None))
    act, near = np.zeros(max(int(m.sum()), 1), np.int64), np.zeros(max(int(nn.sum()), 1), np.int64)
    _check(lib().rs_tree_level_sets(tree, level, _i64p(ck), _i64p(cs), proxy_radius_factor, _i64p(m), _i64p(act),
                                    _i64p(nn), _i64p(near)))
    return m, act[: int(m.sum())], nn, near[: int(nn.sum())]


def rs_factor(tree, kernel=None, a=None, eps=1e-10, opts=None, stream=None, kappa=None, b=None):
    """Factor the operator.  Laplace by default; pass kappa (and b, N values in input order) for
    the Helmholtz kernel, or a ready rs_kernel as `kernel`.  Returns the op handle."""
    bv = None
    if kappa is not None:
        bv = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        k = rs_kernel(RS_HELMHOLTZ, float(kappa), _dp(bv))
    else:
        k = kernel if kernel is not None else rs_kernel(RS_LAPLACE, 0.0, None)
    av = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    o = opts if opts is not None else rs_opts_default()
    out = C.c_void_p()
    _check(lib().rs_factor(tree, C.byref(k), _dp(av), float(eps), C.byref(o), _stream(stream), C.byref(out)))
    return out


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(int(s.cuda_stream))


def _ptr(v):
    if hasattr(v, "data_ptr"):
        return C.c_void_p(v.data_ptr())
    return C.c_void_p(v.ctypes.data)


def rs_solve(op, f, nrhs, x, stream=None):
    """x = A^{-1} f; f and x are both host (numpy) or both device (torch CUDA) buffers holding
    N x nrhs column-major values in input order."""
    _check(lib().rs_solve(op, _ptr(f), int(nrhs), _ptr(x), _stream(stream)))


def rs_fwd_apply(op, x, nrhs, y, stream=None):
    """y = A x through the HSS form the factorization's IDs define (O(N); x, y: both host or
    both device, N x nrhs column-major in input order)."""
    _check(lib().rs_fwd_apply(op, _ptr(x), int(nrhs), _ptr(y), _stream(stream)))


def rs_bicgstab(A, M, f, x, tol=1e-10, max_iter=100, stream=None):
    """x = A^{-1} f by BiCGstab with the right preconditioner M^{-1} (Sec. 5.4); f, x device
    buffers (torch CUDA, N values).  Returns (iterations, relative residual).  Raises RsError
    (RS_E_NOT_CONVERGED) when max_iter is reached."""
    it, rel = C.c_int(), C.c_double()
    _check(lib().rs_bicgstab(A, M, _ptr(f), _ptr(x), float(tol), int(max_iter), C.byref(it), C.byref(rel),
                             _stream(stream)))
    return it.value, rel.value


def rs_wait_check(limit, stream=None):
    """A device-side wait that cannot complete, bounded by `limit` polls: raises RsError with
    code RS_E_TIMEOUT, the expected outcome."""
    _check(lib().rs_wait_check(int(limit), _stream(stream)))


RS_PROBE_DFMA, RS_PROBE_DMMA, RS_PROBE_BF16_MMA = 0, 1, 2


def rs_fp64_probe(kind, stream=None):
    """Measured throughput (TFLOP/s) of DFMA chains (RS_PROBE_DFMA), mma.sync f64 matrix
    instructions (RS_PROBE_DMMA) or bf16 mma.sync products (RS_PROBE_BF16_MMA) on the current
    device."""
    out = C.c_double()
    _check(lib().rs_fp64_probe(int(kind), C.byref(out), _stream(stream)))
    return out.value


def rs_solve_noalloc(op, f, nrhs, x, stream=None):
    """As rs_solve, with the workspace in the library's fixed device array (no allocation);
    f and x must be device buffers."""
    _check(lib().rs_solve_noalloc(op, _ptr(f), int(nrhs), _ptr(x), _stream(stream)))


def rs_residual(op, x, f, nrhs, stream=None):
    """Relative FP64 residuals |f - A x| / |f| per column (x, f: both host or both device)."""
    out = np.zeros(int(nrhs))
    _check(lib().rs_residual(op, _ptr(x), _ptr(f), int(nrhs), _dp(out), _stream(stream)))
    return out


def rs_free(op):
    _check(lib().rs_free(op))


def rs_server_create(ops, mem_budget_bytes, max_inflight=64):
    arr = (C.c_void_p * len(ops))(*[o.value if hasattr(o, "value") else o for o in ops])
    out = C.c_void_p()
    _check(lib().rs_server_create(arr, len(ops), int(mem_budget_bytes), int(max_inflight), C.byref(out)))
    return out


def rs_server_submit(server, op_index, f, nrhs, x):
    """Queue x = A^{-1} f (device buffers, N x nrhs column-major); returns the ticket."""
    t = C.c_uint64()
    _check(lib().rs_server_submit(server, int(op_index), _ptr(f), int(nrhs), _ptr(x), C.byref(t)))
    return t.value


def rs_server_poll(server, max_tickets=1024):
    buf = (C.c_uint64 * max_tickets)()
    n = C.c_int()
    _check(lib().rs_server_poll(server, buf, max_tickets, C.byref(n)))
    return list(buf[: n.value])


def rs_server_drain(server, timeout_s=600.0):
    _check(lib().rs_server_drain(server, float(timeout_s)))


def rs_server_stats(server):
    v = [C.c_int64() for _ in range(5)]
    _check(lib().rs_server_stats(server, *[C.byref(x) for x in v]))
    return dict(zip(("submitted", "completed", "rhs_completed", "ticks", "peak_inflight"), [x.value for x in v]))


def rs_server_latencies(server):
    n = C.c_int64()
    _check(lib().rs_server_latencies(server, None, 0, C.byref(n)))
    out = np.zeros(max(n.value, 1))
    _check(lib().rs_server_latencies(server, _dp(out), n.value, C.byref(n)))
    return out[: n.value]


def rs_server_free(server):
    lib().rs_server_free(server)


def rs_op_stats(op):
    s = rs_stats()
    _check(lib().rs_op_stats(op, C.byref(s)))
    return {name: getattr(s, name) for name, _ in rs_stats._fields_}


def rs_op_profile(op):
    """Per-class kernel times (opts.profile): {name: (ms, work, bytes, launches)}."""
    out = {}
    for cls, name in enumerate(PROF_CLASSES):
        ms, w, b, n = C.c_double(), C.c_double(), C.c_double(), C.c_int64()
        _check(lib().rs_op_profile(op, cls, C.byref(ms), C.byref(w), C.byref(b), C.byref(n)))
        out[name] = (ms.value, w.value, b.value, n.value)
    return out


def rs_op_profile_level(op, cls_name, level):
    """Event time (ms) of one profile class at one tree level (opts.profile)."""
    ms = C.c_double()
    _check(lib().rs_op_profile_level(op, PROF_CLASSES.index(cls_name), int(level), C.byref(ms)))
    return ms.value


def rs_autotune(tree, kernel=None, a=None, eps=1e-10, opts=None, stream=None, path=None, kappa=None, b=None):
    """Time the candidate launch settings on this operator and fill the tuning table (and
    `path`, JSON, if given).  Returns the report as a dict."""
    if kappa is not None:
        bv = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        k = rs_kernel(RS_HELMHOLTZ, float(kappa), _dp(bv))
    else:
        k = kernel if kernel is not None else rs_kernel(RS_LAPLACE, 0.0, None)
    av = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    o = opts if opts is not None else rs_opts_default()
    rep = rs_tune_report()
    _check(lib().rs_autotune(tree, C.byref(k), _dp(av), float(eps), C.byref(o), _stream(stream),
                             None if path is None else str(path).encode(), C.byref(rep)))
    return {name: getattr(rep, name) for name, _ in rs_tune_report._fields_}


def rs_tune_save(path):
    _check(lib().rs_tune_save(str(path).encode()))


def rs_tune_load(path):
    _check(lib().rs_tune_load(str(path).encode()))


def rs_tune_clear():
    _check(lib().rs_tune_clear())


def rs_tune_count():
    return int(lib().rs_tune_count())


def rs_launch_count():
    return lib().rs_launch_count()


def rs_op_box_sizes(op, level, box):
    m, k, r, nn = C.c_int64(), C.c_int64(), C.c_int64(), C.c_int64()
    _check(lib().rs_op_box_sizes(op, level, box, C.byref(m), C.byref(k), C.byref(r), C.byref(nn)))
    return m.value, k.value, r.value, nn.value


def rs_op_box_indices(op, level, box, which):
    m, k, _, nn = rs_op_box_sizes(op, level, box)
    cnt = (m, nn, k)[which]
    out = np.zeros(max(cnt, 1), dtype=np.int64)
    _check(lib().rs_op_box_indices(op, level, box, which, _i64p(out)))
    return out[:cnt]


def rs_op_box_matrix(op, level, box, which, cplx=False):
    """T (which 0), F^{-1} (1) or E (2) of one box; complex operators need cplx=True."""
    m, k, _, _ = rs_op_box_sizes(op, level, box)
    shape = ((k, m - k), (m, m), (k, k))[which]
    c = 2 if cplx else 1
    out = np.zeros(max(c * shape[0] * shape[1], 2))
    _check(lib().rs_op_box_matrix(op, level, box, which, _dp(out)))
    out = out[: c * shape[0] * shape[1]]
    return (out.view(np.complex128) if cplx else out).reshape(shape)


def rs_op_root_matrix(op, cplx=False):
    m = rs_op_stats(op)["root_m"]
    c = 2 if cplx else 1
    out = np.zeros(c * m * m)
    _check(lib().rs_op_root_matrix(op, _dp(out)))
    return (out.view(np.complex128) if cplx else out).reshape(m, m)


def rs_op_box_order(op, level, box, which):
    """Sec. 3.1 order of a box: skeleton indices cyclically (which 0), residual indices along
    the interface (1)."""
    m, k, _, _ = rs_op_box_sizes(op, level, box)
    cnt = k if which == 0 else m - k
    out = np.zeros(max(cnt, 1), dtype=np.int64)
    _check(lib().rs_op_box_order(op, level, box, which, _i64p(out)))
    return out[:cnt]


def rs_tree_box_order(tree, level, box, which, g):
    """Sec. 3.1 order of the grid points g of box (level, box): cyclic (which 0) or along the
    interface (1); returns the index into g at each position."""
    gv = np.ascontiguousarray(g, dtype=np.int64)
    out = np.zeros(max(len(gv), 1), dtype=np.int64)
    _check(lib().rs_tree_box_order(tree, level, box, which, _i64p(gv), len(gv), _i64p(out)))
    return out[: len(gv)]


def rs_op_box_form(op, level, box, which):
    """Compressed form of a box block (which 0 phi_ss, 1 phi_rr, 2 E, 3 phi_sr, 4 phi_rs, 5 T):
    (depth, entries, nodes) with nodes an (n, 4) array of (lo, hi, a, k)."""
    d, e = C.c_int(), C.c_int64()
    _check(lib().rs_op_box_form(op, level, box, which, C.byref(d), C.byref(e), None))
    cnt = 1 if d.value <= 0 else (1 << (d.value + 1)) - 2
    nodes = np.zeros(4 * cnt, dtype=np.int64)
    _check(lib().rs_op_box_form(op, level, box, which, C.byref(d), C.byref(e), _i64p(nodes)))
    return d.value, e.value, nodes.reshape(cnt, 4)


def rs_hss1d_build(M, order=None, leaf=64, eps=1e-10, stream=None):
    """HSS1D form of the square matrix M: a numpy array (real or complex), or a torch CUDA
    tensor whose contiguous storage is M column-major (i.e. the tensor holds M^T).  Returns the
    handle."""
    if hasattr(M, "data_ptr"):
        n = int(M.shape[0])
        cplx = bool(M.is_complex())
        ptr = C.c_void_p(M.data_ptr())
    else:
        cplx = np.iscomplexobj(M)
        Mf = np.asfortranarray(M, dtype=np.complex128 if cplx else np.float64)
        n = Mf.shape[0]
        ptr = C.c_void_p(Mf.ctypes.data)
    o = None if order is None else np.ascontiguousarray(order, dtype=np.int64)
    out = C.c_void_p()
    _check(lib().rs_hss1d_build(ptr, n, int(cplx), _i64p(o), int(leaf), float(eps), _stream(stream), C.byref(out)))
    return out


def rs_hss1d_apply(h, x, nrhs, y, stream=None):
    """y = M x (n x nrhs column-major; both host numpy or both device torch)."""
    _check(lib().rs_hss1d_apply(h, _ptr(x), int(nrhs), _ptr(y), _stream(stream)))


def rs_hss1d_info(h):
    d, e, b = C.c_int(), C.c_int64(), C.c_int64()
    _check(lib().rs_hss1d_info(h, C.byref(d), C.byref(e), C.byref(b)))
    return d.value, e.value, b.value


def rs_hss1d_node(h, level, node):
    """(lo, hi, a, k, skeleton rows) of one node."""
    v = [C.c_int64() for _ in range(4)]
    _check(lib().rs_hss1d_node(h, level, node, *[C.byref(x) for x in v], None))
    k = v[3].value
    sk = np.zeros(max(k, 1), dtype=np.int64)
    _check(lib().rs_hss1d_node(h, level, node, None, None, None, None, _i64p(sk)))
    return v[0].value, v[1].value, v[2].value, k, sk[:k]


def rs_hss1d_free(h):
    _check(lib().rs_hss1d_free(h))


class Solver:
    """Convenience owner of a tree and its factorization (frees both on deletion)."""

    def __init__(self, points, leaf_side, a=None, eps=1e-10, kernel=None, opts=None, stream=None, kappa=None, b=None):
        self.N = int(np.asarray(points).shape[0])
        self.complex = kappa is not None
        self.tree = rs_build_tree(points, leaf_side)
        self.op = None
        self.op = rs_factor(self.tree, kernel=kernel, a=a, eps=eps, opts=opts, stream=stream, kappa=kappa, b=b)

    def solve(self, f, stream=None):
        """f: numpy (N,) / (N, nrhs), or torch CUDA (N,) / (nrhs, N).  Returns x of the same kind."""
        if hasattr(f, "data_ptr"):
            import torch
            fc = f.contiguous()
            nrhs = 1 if fc.dim() == 1 else fc.shape[0]
            x = torch.empty_like(fc)
            rs_solve(self.op, fc, nrhs, x, stream if stream is not None else torch.cuda.current_stream())
            return x
        fa = np.asarray(f, dtype=np.complex128 if self.complex else np.float64)
        nrhs = 1 if fa.ndim == 1 else fa.shape[1]
        fa = np.asfortranarray(fa)
        x = np.zeros_like(fa, order="F")
        rs_solve(self.op, fa, nrhs, x, stream)
        return x

    def fwd_apply(self, v):
        """A v through the HSS form of the factorization (numpy (N,) / (N, nrhs))."""
        va = np.asfortranarray(np.asarray(v, dtype=np.complex128 if self.complex else np.float64))
        nrhs = 1 if va.ndim == 1 else va.shape[1]
        y = np.zeros_like(va, order="F")
        rs_fwd_apply(self.op, va, nrhs, y)
        return y

    def stats(self):
        return rs_op_stats(self.op)

    def __del__(self):
        if getattr(self, "op", None):
            rs_free(self.op)
            self.op = None
        if getattr(self, "tree", None):
            rs_free_tree(self.tree)
            self.tree = None
