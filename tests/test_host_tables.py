"""Host tabulation of the library's trees (pic_tree_tabulate: no GPU
needed) against the oracle's tables on uniform and unbalanced 2D/3D trees:
the finite-element grid (non-hanging vertices, hanging-vertex expansions of
every leaf corner, vertex loads and stiffness diagonals; Section 4 tree, the
d-linear grid of Section 3) and the PIDT owner vertices (Algorithms 2-3)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

TREES = [
    pytest.param(2, lambda: W.uniform_tree_flags(2, 3), id="2d-uniform"),
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), id="2d-adaptive-a"),
    pytest.param(2, lambda: W.random_tree_flags(2, 6, 0.2, 11, min_depth=1), id="2d-adaptive-b"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 2), id="3d-uniform"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), id="3d-adaptive-a"),
    pytest.param(3, lambda: W.random_tree_flags(3, 4, 0.05, 9, min_depth=2), id="3d-adaptive-b"),
]


def _lib_or_skip():
    try:
        return pic.load()
    except Exception as exc:  # pragma: no cover - the library is built by build()
        pytest.skip(f"library not built: {exc}")


@pytest.mark.parametrize("d,flags_fn", TREES)
def test_host_tables_match_oracle(d, flags_fn):
    _lib_or_skip()
    flags = flags_fn()
    tab = pic.tree_tables(d, flags)
    ot = oracle.Tree(d, flags)
    assert tab["n_leaves"] == ot.n_leaves and tab["depth"] == ot.depth
    assert np.array_equal(tab["vertex_pos"], ot.vertex_pos())
    lev, j = ot.pidt_vertices()
    assert np.array_equal(tab["pidt_level"], lev) and np.array_equal(tab["pidt_j"], j)
    if tab["uniform"]:
        return
    ptr, vid, w = ot.corner_expansion()
    assert np.array_equal(tab["cexp_ptr"], ptr) and np.array_equal(tab["cexp_vid"], vid)
    assert np.allclose(tab["cexp_w"], w, rtol=1e-14, atol=0)
    ion, diag = ot.vertex_aux()
    assert np.allclose(tab["ion_load"], ion, rtol=1e-12, atol=0)
    assert np.allclose(tab["diag"], diag, rtol=1e-12, atol=0)
    # hanging vertices exist in these trees and are expanded onto several vertices
    assert (np.diff(ptr) > 1).any()


def test_host_tables_reject_malformed_tree():
    _lib_or_skip()
    with pytest.raises(pic.PicError):
        pic.tree_tables(3, np.array([1, 0, 0], np.uint8))  # a refined root without 27 children


@pytest.mark.parametrize("d,flags_fn", [TREES[2], TREES[5]])
def test_host_tables_do_not_depend_on_thread_count(d, flags_fn, monkeypatch):
    """The threaded tabulation (radix sorts, chunked passes) gives the same
    tables with one host thread as with several."""
    _lib_or_skip()
    flags = flags_fn()
    monkeypatch.setenv("PIC_HOST_THREADS", "1")
    one = pic.tree_tables(d, flags)
    monkeypatch.setenv("PIC_HOST_THREADS", "7")
    seven = pic.tree_tables(d, flags)
    assert one.keys() == seven.keys()
    for k in one:
        assert np.array_equal(np.asarray(one[k]), np.asarray(seven[k])), k


def test_host_tables_reject_adaptive_trees_deeper_than_level_12():
    _lib_or_skip()
    # a chain of first children refined down to level 13 in 2D
    flags = []
    for level in range(13):
        flags += [1] + [0] * (8 if level else 0)
    flags += [0] * 9
    with pytest.raises(pic.PicError):
        pic.tree_tables(2, np.array(flags, np.uint8))
