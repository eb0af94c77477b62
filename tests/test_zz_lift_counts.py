"""Lift, drop and tunneller counts of the steps (pic_count_lifts /
pic_lift_counts) against the oracle: the oracle runs the same steps and
counts, for every particle, the lifts and drops between its leaf (PIT,
Algorithm 1) or owner vertex (PIDT, Algorithms 2-3 read as a count) before and
after each step, and whether its new leaf touches its old one (the closed
forms are pinned on the CPU in tests/test_oracle_pins.py and
tests/test_oracle_pins_fp32.py).  Totals must agree exactly, and counting must
not change the steps."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

CASES = [
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), pic.FP64, id="2d-adaptive-fp64"),
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), pic.FP32_SPLIT, id="2d-adaptive-split"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 3), pic.FP32_SPLIT, id="3d-brick-split"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), pic.FP64, id="3d-adaptive-fp64"),
]


def oracle_leaf_by_id(tree, st, split):
    leaf = st.leaf if split else tree.pit_owner(st.x)
    out = np.empty(len(leaf), np.int64)
    out[st.ids] = leaf
    return out


def oracle_key_by_id(st):
    out = np.empty(len(st.key), np.int64)
    out[st.ids] = st.key
    return out


@pytest.mark.parametrize("d,flags_fn,precision", CASES)
def test_lift_counts_match_oracle(d, flags_fn, precision):
    flags = flags_fn()
    n = 40_000
    x, v = W.random_particles(d, n, 17, vmax=0.5)  # tunnelling: several cells per step
    q = -1.0 / n
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=pic.PIT, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    ot = oracle.Tree(d, flags)
    st = (oracle.State32 if split else oracle.State64)(ot, x, v, prm)
    kw = dict(scheme=pic.PIT, precision=precision, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    g = pic.Pic(d, flags, x, v, **kw)
    plain = pic.Pic(d, flags, x, v, **kw)
    g.count_lifts(True)
    lifts = drops = tun = 0
    for _ in range(3):
        before = oracle_leaf_by_id(ot, st, split)
        st.step(0.1)
        after = oracle_leaf_by_id(ot, st, split)
        li, dr = ot.pit_lifts(before, after)
        lifts += int(li.sum())
        drops += int(dr.sum())
        tun += int(ot.tunnellers(before, after).sum())
        g.step(0.1)
        plain.step(0.1)
    g.sync()
    plain.sync()
    assert lifts > 0 and tun > 0
    assert g.lift_counts() == (lifts, drops, tun, 3)
    assert g.stats().tunnellers == tun
    for u, w in zip(g.get_state(), plain.get_state()):
        assert np.array_equal(u, w)
    assert np.array_equal(g.bins()[1], st.ids)
    g.count_lifts(True)  # restart from zero
    assert g.lift_counts() == (0, 0, 0, 0)
    g.step_fixed_field(0.0)  # nobody moves
    assert g.lift_counts() == (0, 0, 0, 1)
    g.count_lifts(False)
    assert g.stats().tunnellers == -1
    with pytest.raises(pic.PicError):
        g.lift_counts()


PIDT_CASES = [
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), pic.FP64, id="2d-adaptive-fp64"),
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), pic.FP32_SPLIT, id="2d-adaptive-split"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 3), pic.FP32_SPLIT, id="3d-uniform-split"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), pic.FP64, id="3d-adaptive-fp64"),
]


@pytest.mark.parametrize("d,flags_fn,precision", PIDT_CASES)
def test_pidt_lift_counts_match_oracle(d, flags_fn, precision):
    flags = flags_fn()
    n = 40_000
    x, v = W.random_particles(d, n, 19, vmax=0.5)
    q = -1.0 / n
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=pic.PIDT, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    ot = oracle.Tree(d, flags)
    st = (oracle.State32 if split else oracle.State64)(ot, x, v, prm)
    kw = dict(scheme=pic.PIDT, precision=precision, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    g = pic.Pic(d, flags, x, v, **kw)
    plain = pic.Pic(d, flags, x, v, **kw)
    g.count_lifts(True)
    lifts = drops = tun = 0
    for _ in range(3):
        leaf0, key0 = oracle_leaf_by_id(ot, st, split), oracle_key_by_id(st)
        st.step(0.1)
        leaf1, key1 = oracle_leaf_by_id(ot, st, split), oracle_key_by_id(st)
        li, dr = ot.pidt_lifts(leaf0, key0, key1)
        lifts += int(li.sum())
        drops += int(dr.sum())
        tun += int(ot.tunnellers(leaf0, leaf1).sum())
        g.step(0.1)
        plain.step(0.1)
    g.sync()
    plain.sync()
    assert lifts > 0 and tun > 0
    assert g.lift_counts() == (lifts, drops, tun, 3)
    for u, w in zip(g.get_state(), plain.get_state()):
        assert np.array_equal(u, w)
    assert np.array_equal(g.bins()[1], st.ids)


def test_lift_counting_needs_ids():
    flags = W.uniform_tree_flags(2, 3)
    x, v = W.random_particles(2, 1000, 3)
    with pytest.raises(pic.PicError):
        pic.Pic(2, flags, x, v, track_ids=False).count_lifts(True)
