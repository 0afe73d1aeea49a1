"""The C ABI on CPU: every declared symbol is exported, argument errors are reported, and the
host bookkeeping of the tree (Sec. 2.2) is bit-exact with the oracle at every level."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_1303_5466_gb300 import build as B
from paper_1303_5466_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def rs():
    B.build()
    import paper_1303_5466_gb300 as P
    P.lib()
    return P


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rs_[a-z0-9_]+)\s*\(", txt))
    return sorted(names)


def test_every_declared_symbol_is_exported(rs):
    names = _declared()
    assert "rs_factor" in names and "rs_solve" in names and "rs_build_tree" in names
    L = C.CDLL(rs.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing


def test_build_tree_rejects_bad_input(rs):
    pts = W.grid_points(16)
    with pytest.raises(rs.RsError) as e:
        rs.rs_build_tree(pts[:-1], 4)
    assert e.value.code == rs.RS_E_INVALID
    bad = pts.copy()
    bad[3, 0] += 0.3 / 16
    with pytest.raises(rs.RsError) as e:
        rs.rs_build_tree(bad, 4)
    assert e.value.code == rs.RS_E_NOT_GRID
    dup = pts.copy()
    dup[5] = dup[6]
    with pytest.raises(rs.RsError) as e:
        rs.rs_build_tree(dup, 4)
    assert e.value.code == rs.RS_E_NOT_GRID
    with pytest.raises(rs.RsError) as e:
        rs.rs_build_tree(pts, 5)                 # 16 / 5 not an integer
    assert e.value.code == rs.RS_E_INVALID
    with pytest.raises(rs.RsError) as e:
        rs.rs_build_tree(pts, 16)                # one leaf: no tree
    assert e.value.code == rs.RS_E_INVALID
    with pytest.raises(rs.RsError):
        rs.rs_build_tree(np.zeros((0, 2)), 4)    # empty


def test_tree_info_and_input_permutation(rs):
    n = 16
    perm = W.shuffled(n, 4)
    pts = W.grid_points(n)[perm]
    t = rs.rs_build_tree(pts, 4)
    try:
        nn, d, g = rs.rs_tree_info(t, n * n)
        assert nn == n and d == 4
        np.testing.assert_array_equal(g, perm)
    finally:
        rs.rs_free_tree(t)


@pytest.mark.parametrize("n,leaf", [(32, 8), (64, 16), (32, 4)])
def test_level_bookkeeping_matches_oracle(rs, oracle_mod, n, leaf):
    """Active sets and near rows of every box at every level, given the oracle's skeletons
    of the level below, are identical (integers, in order) to the oracle's."""
    F = oracle_mod.Factorization(n, leaf, 1e-10)
    t = rs.rs_build_tree(W.grid_points(n), leaf)
    try:
        for l in range(F.depth, 0, -1):
            if l == F.depth:
                m, act, nn, near = rs.rs_tree_level_sets(t, l)
            else:
                ck = np.array([F.sizes(l + 1, j)[1] for j in range(2 ** (l + 1))], dtype=np.int64)
                cs = np.concatenate([F.skel(l + 1, j) for j in range(2 ** (l + 1))])
                m, act, nn, near = rs.rs_tree_level_sets(t, l, ck, cs)
            ao = np.concatenate([[0], np.cumsum(m)])
            no = np.concatenate([[0], np.cumsum(nn)])
            for j in range(2 ** l):
                np.testing.assert_array_equal(act[ao[j]:ao[j + 1]], F.active(l, j))
                np.testing.assert_array_equal(near[no[j]:no[j + 1]], F.near(l, j))
    finally:
        rs.rs_free_tree(t)


@pytest.mark.parametrize("n,leaf", [(64, 8), (32, 4)])
def test_compression_orders_match_oracle(rs, oracle_mod, n, leaf):
    """Orders of Sec. 3.1 (skeleton around the box, residual along the interface) for the
    oracle's skeleton and residual points of every box: identical integers on both sides."""
    F = oracle_mod.Factorization(n, leaf, 1e-10)
    t = rs.rs_build_tree(W.grid_points(n), leaf)
    try:
        for l in range(1, F.depth + 1):
            for j in range(2 ** l):
                sk = F.skel(l, j)
                np.testing.assert_array_equal(rs.rs_tree_box_order(t, l, j, 0, sk), F.order(l, j, 0))
                sks = set(sk.tolist())
                rsg = np.array([g for g in F.active(l, j) if g not in sks], dtype=np.int64)
                np.testing.assert_array_equal(rs.rs_tree_box_order(t, l, j, 1, rsg), F.order(l, j, 1))
        with pytest.raises(rs.RsError):
            rs.rs_tree_box_order(t, 1, 0, 0, np.array([n * n], dtype=np.int64))
    finally:
        rs.rs_free_tree(t)


def test_struct_layouts_match_the_header(rs, tmp_path):
    """The ctypes mirrors of rs_kernel, rs_opts, rs_stats and rs_tune_report have the size and the
    field offsets that a C compiler gives the structs of include/rs.h (a field missing on either
    side, or out of order, fails), and rs_opts_default fills the documented defaults of the
    fields added last."""
    import subprocess
    structs = [rs.rs_kernel, rs.rs_opts, rs.rs_stats, rs.rs_tune_report]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "rs.h"', "int main(void) {"]
    for S in structs:
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (S.__name__, S.__name__))
        for name, _ in S._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (S.__name__, name, S.__name__, name))
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = dict(l.split() for l in subprocess.run([str(exe)], check=True, capture_output=True,
                                                  text=True).stdout.splitlines())
    for S in structs:
        assert int(out[S.__name__]) == C.sizeof(S), S.__name__
        for name, _ in S._fields_:
            assert int(out["%s.%s" % (S.__name__, name)]) == getattr(S, name).offset, (S.__name__, name)
    o = rs.rs_opts_default()
    assert o.gemm_form == 1 and o.forward_only == 0 and o.cpqr_variant == -1
