"""The particle-handling step of the paper's experiments (pic_step_particles:
no field, reflecting or periodic walls, artificial flops, dynamic ppc
refinement) against the oracle: keys, bucket order and state bit for bit
(FP64 positions within 1e-12), on adaptive 2D and 3D trees, PIT and PIDT,
FP64 and split, with particles that tunnel and bounce off the walls."""
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


def compare(g, st, split):
    g.sync()
    start, ids = g.bins()
    assert np.array_equal(ids, st.ids)
    assert np.array_equal(g.keys(), st.key)
    if split:
        leaf, o, v = g.get_state()
        assert np.array_equal(leaf, st.leaf) and np.array_equal(o, st.o) and np.array_equal(v, st.v)
    else:
        x, v = g.particles()
        assert np.max(np.abs(x - st.x)) <= 1e-12 and np.array_equal(np.sign(v), np.sign(st.v))
        assert np.max(np.abs(v - st.v)) <= 1e-12


CASES = [
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), id="2d-adaptive"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), id="3d-adaptive"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 3), id="3d-uniform"),
]


@pytest.mark.parametrize("d,flags_fn", CASES)
@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
@pytest.mark.parametrize("reflect", [True, False])
def test_particle_steps_match_oracle(d, flags_fn, scheme, precision, reflect):
    flags = flags_fn()
    w = W.particle_handling(d, 30_000, seed=41)
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=scheme, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    st = (oracle.State32 if split else oracle.State64)(oracle.Tree(d, flags), w.x, w.v, prm)
    g = pic.Pic(d, flags, w.x, w.v, scheme=scheme, precision=precision, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    for dt in (0.02, 0.3, 1.7):   # within a cell, several cells, several wall hits
        st.move(dt, 1 if reflect else 0)
        g.step_particles(dt, reflect=reflect)
        compare(g, st, split)


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_breaking_dam_with_ppc_refinement_every_step(precision):
    """The (0, 0.1)^d start spreading through the box, the tree re-refined by
    the ppc criterion before every step (refine on overrun, coarsen when the
    union stays within ppc), as in the paper's dynamic-AMR experiments."""
    d, ppc, dmin, dmax = 2, 40, 1, 6
    w = W.particle_handling(d, 20_000, dam=True, seed=42)
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=pic.PIT, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    st = (oracle.State32 if split else oracle.State64)(oracle.Tree(d, w.flags), w.x, w.v, prm)
    g = pic.Pic(d, w.flags, w.x, w.v, scheme=pic.PIT, precision=precision, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    for _ in range(4):
        g.adapt(ppc, dmin, dmax)
        flags = (oracle.retree32(st.tree, st.leaf, st.o, ppc, dmin, dmax) if split
                 else oracle.retree64(d, st.x, ppc, dmin, dmax))
        assert np.array_equal(g.tree_flags(), flags)
        nt = oracle.Tree(d, flags)
        if split:
            st.tree.rebin32_into(nt, st.leaf, st.o)
        st.tree = nt
        del st.key
        st.rebin()
        st.move(0.05, 1)
        g.step_particles(0.05, reflect=True)
        compare(g, st, split)
    assert len(flags) > 10


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_artificial_flops_change_nothing(precision):
    d = 3
    flags = W.random_tree_flags(d, 3, 0.3, 6, min_depth=1)
    w = W.particle_handling(d, 20_000, seed=43)
    kw = dict(scheme=pic.PIT, precision=precision, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    a = pic.Pic(d, flags, w.x, w.v, **kw)
    b = pic.Pic(d, flags, w.x, w.v, **kw)
    for _ in range(2):
        a.step_particles(0.1, reflect=True, flops=0)
        b.step_particles(0.1, reflect=True, flops=4096)
    a.sync()
    b.sync()
    for u, v in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, v)
    with pytest.raises(pic.PicError):
        a.step_particles(0.1, flops=-1)
    assert a.lib.pic_step_particles(a.h, 0.1, 7, 0) == -1   # no such boundary


def test_lift_counts_of_particle_steps():
    """Lifts and drops of Algorithm 1 for the particle-handling move equal the
    oracle's closed form per particle, summed."""
    d = 2
    flags = W.random_tree_flags(d, 5, 0.3, 5, min_depth=2)
    w = W.particle_handling(d, 20_000, seed=44)
    prm = oracle.Params(scheme=pic.PIT, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    ot = oracle.Tree(d, flags)
    st = oracle.State64(ot, w.x, w.v, prm)
    g = pic.Pic(d, flags, w.x, w.v, scheme=pic.PIT, precision=pic.FP64, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    g.count_lifts(True)
    lifts = drops = tun = 0
    for dt in (0.01, 0.1):
        before = np.empty(w.n, np.int64)
        before[st.ids] = ot.pit_owner(st.x)
        st.move(dt, 1)
        after = np.empty(w.n, np.int64)
        after[st.ids] = ot.pit_owner(st.x)
        li, dr = ot.pit_lifts(before, after)
        lifts += int(li.sum())
        drops += int(dr.sum())
        tun += int(ot.tunnellers(before, after).sum())
        g.step_particles(dt, reflect=True)
    assert g.lift_counts() == (lifts, drops, tun, 2)


def test_brick_handle_alternates_field_and_particle_steps():
    """On a handle that runs the brick path (uniform 3D tree, split, PIT) the
    field-free step takes the generic re-bin; field steps before and after it
    stay bit-identical to the oracle."""
    d, n = 3, 60_000
    flags = W.uniform_tree_flags(d, 3)
    x, v = W.random_particles(d, n, 45, vmax=0.05)
    kw = dict(scheme=pic.PIT, q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=3, omega=0.8)
    g = pic.Pic(d, flags, x, v, precision=pic.FP32_SPLIT, **kw)
    assert g.info().brick == 1
    st = oracle.State32(oracle.Tree(d, flags), x, v, oracle.Params(**kw))
    for s in range(4):
        if s % 2:
            st.move(0.1, 1)
            g.step_particles(0.1, reflect=True)
        else:
            st.step(0.05)
            g.step(0.05)
        compare(g, st, True)


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_pidt_lift_counts_across_refinements(precision):
    """PIDT lifts, drops and tunnellers of particle steps with the tree
    re-refined by ppc before every step: each step counts on the tree it ran
    on (the owner-vertex tables follow every new tree)."""
    d, ppc, dmin, dmax = 2, 40, 1, 6
    w = W.particle_handling(d, 20_000, dam=True, seed=46)
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=pic.PIDT, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    st = (oracle.State32 if split else oracle.State64)(oracle.Tree(d, w.flags), w.x, w.v, prm)
    g = pic.Pic(d, w.flags, w.x, w.v, scheme=pic.PIDT, precision=precision, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    g.count_lifts(True)

    def by_id(a):
        out = np.empty(len(a), np.int64)
        out[st.ids] = a
        return out

    lifts = drops = tun = 0
    sizes = set()
    for _ in range(4):
        g.adapt(ppc, dmin, dmax)
        flags = (oracle.retree32(st.tree, st.leaf, st.o, ppc, dmin, dmax) if split
                 else oracle.retree64(d, st.x, ppc, dmin, dmax))
        nt = oracle.Tree(d, flags)
        sizes.add(nt.n_leaves)
        if split:
            st.tree.rebin32_into(nt, st.leaf, st.o)
        st.tree = nt
        del st.key
        st.rebin()
        leaf0 = by_id(st.leaf if split else nt.pit_owner(st.x))
        key0 = by_id(st.key)
        st.move(0.08, 1)
        leaf1 = by_id(st.leaf if split else nt.pit_owner(st.x))
        li, dr = nt.pidt_lifts(leaf0, key0, by_id(st.key))
        lifts += int(li.sum())
        drops += int(dr.sum())
        tun += int(nt.tunnellers(leaf0, leaf1).sum())
        g.step_particles(0.08, reflect=True)
        compare(g, st, split)
    assert len(sizes) > 1 and lifts > 0
    assert g.lift_counts() == (lifts, drops, tun, 4)
