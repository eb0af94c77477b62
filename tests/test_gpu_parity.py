"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Keys, buckets and integer state are compared bit for bit; FP64 floats within
1e-12 relative (they are expected bit-identical: both sides use the same
operation order with no fused multiply-add); FP32 split results within a few
FP32 ulps of the mirror.
"""
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

REL64 = 1e-12


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    scale = max(np.max(np.abs(b)), 1e-300)
    return float(np.max(np.abs(a - b)) / scale) if a.size else 0.0


def make(d, flags, x, v, scheme, precision, **kw):
    return pic.Pic(d, flags, x, v, scheme=scheme, precision=precision, **kw)


def random_case(d, depth, p, seed, n, vmax=0.05, min_depth=1):
    flags = W.random_tree_flags(d, depth, p, seed, min_depth=min_depth)
    x, v = W.random_particles(d, n, seed, vmax=vmax)
    return flags, x, v


TREES = [
    pytest.param(2, lambda: W.uniform_tree_flags(2, 3), id="2d-uniform-d3"),
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), id="2d-adaptive-d5"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 2), id="3d-uniform-d2"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 3), id="3d-uniform-d3"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), id="3d-adaptive-d3"),
]


# ---------------------------------------------------------------------------
# tables
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,flags_fn", TREES)
def test_tables_match_oracle(d, flags_fn):
    flags = flags_fn()
    x, v = W.random_particles(d, 1000, 1)
    ot = oracle.Tree(d, flags)
    g = make(d, flags, x, v, pic.PIT, pic.FP64)
    lev, co = g.leaf_table()
    olev, oco = ot.leaf_info()
    assert np.array_equal(lev, olev) and np.array_equal(co, oco)
    assert np.array_equal(g.vertex_table(), ot.vertex_pos())
    gp = make(d, flags, x, v, pic.PIDT, pic.FP64)
    plev, pj = gp.pidt_table()
    oplev, opj = ot.pidt_vertices()
    assert np.array_equal(plev, oplev) and np.array_equal(pj, opj)


# ---------------------------------------------------------------------------
# a1/a2 keys and a6 buckets at creation
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
@pytest.mark.parametrize("d,flags_fn", TREES)
def test_initial_keys_and_buckets(d, flags_fn, scheme, precision):
    flags = flags_fn()
    n = 70_001  # several tiles and a ragged tail
    x, v = W.random_particles(d, n, 7)
    # particles on faces and at the wrap-around point
    x[:, :27] = (np.arange(27) % 9)[None, :] / 9.0
    x[:, 27] = 1.0 - 1e-17
    x[:, 28] = -0.25
    ot = oracle.Tree(d, flags)
    prm = oracle.Params(scheme=scheme)
    st = oracle.State64(ot, x, v, prm) if precision == pic.FP64 else oracle.State32(ot, x, v, prm)
    g = make(d, flags, x, v, scheme, precision)
    keys = g.keys()
    start, ids = g.bins()
    assert np.array_equal(ids, st.ids)                     # same storage order
    assert np.array_equal(keys, st.key)                    # bit-exact keys
    nb = 1 << d if scheme == pic.PIDT else 1
    assert np.array_equal(start, st.start[::nb])
    if precision == pic.FP32_SPLIT:
        leaf, o, vf = g.get_state()
        assert np.array_equal(leaf, st.leaf)
        assert np.array_equal(o, st.o) and np.array_equal(vf, st.v)
    else:
        xs, vs = g.particles()
        assert np.array_equal(xs, st.x) and np.array_equal(vs, st.v)


# ---------------------------------------------------------------------------
# one full step: deposit, solve, field, gather + push, re-bin
# ---------------------------------------------------------------------------

def compare_step64(g, st, d):
    Qo, tot, res, Eo = st.step(0.1)
    g.step(0.1)
    g.sync()
    return Qo, Eo


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("d,flags_fn", TREES)
def test_fp64_steps_match_oracle(d, flags_fn, scheme):
    flags = flags_fn()
    n = 40_000
    x, v = W.random_particles(d, n, 11, vmax=0.5)   # tunnelling: up to ~5 finest cells per step
    q = -1.0 / n
    prm = oracle.Params(scheme=scheme, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    ot = oracle.Tree(d, flags)
    st = oracle.State64(ot, x, v, prm)
    g = make(d, flags, x, v, scheme, pic.FP64, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    for step in range(3):
        Qo, tot, res, Eo = st.step(0.1)
        Qg_before = g.deposit()
        assert rel_err(Qg_before, Qo) <= REL64, f"deposit step {step}"
        g.step(0.1)
        g.sync()
        assert rel_err(g.potential(), st.V) <= REL64, f"potential step {step}"
        assert rel_err(g.field(), Eo) <= REL64, f"field step {step}"
        keys = g.keys()
        start, ids = g.bins()
        assert np.array_equal(ids, st.ids), f"storage order step {step}"
        assert np.array_equal(keys, st.key), f"keys step {step}"
        xs, vs = g.particles()
        assert rel_err(xs, st.x) <= REL64 and rel_err(vs, st.v) <= REL64
        s = g.stats()
        assert abs(s.total_charge - tot) <= 1e-12
        assert s.error == 0


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("d,flags_fn", TREES)
def test_split_steps_match_mirror(d, flags_fn, scheme):
    flags = flags_fn()
    n = 40_000
    x, v = W.random_particles(d, n, 12, vmax=0.5)
    q = -1.0 / n
    prm = oracle.Params(scheme=scheme, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    ot = oracle.Tree(d, flags)
    st = oracle.State32(ot, x, v, prm)
    g = make(d, flags, x, v, scheme, pic.FP32_SPLIT, q=q, qm=-1.0, ion=1.0, sweeps=30, omega=0.8)
    for step in range(3):
        Qo, tot, res, Eo = st.step(0.1)
        g.step(0.1)
        g.sync()
        # field arithmetic is FP32 with the same operation order
        assert rel_err(g.field(), Eo) <= 1e-5, f"field step {step}"
        leaf, o, vf = g.get_state()
        start, ids = g.bins()
        assert np.array_equal(ids, st.ids), f"storage order step {step}"
        assert np.array_equal(g.keys(), st.key), f"keys step {step}"
        assert np.array_equal(leaf, st.leaf)
        assert np.array_equal(o, st.o) and np.array_equal(vf, st.v)


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------

def test_empty_particle_set():
    flags = W.uniform_tree_flags(2, 2)
    x = np.zeros((2, 0))
    g = make(2, flags, x, x.copy(), pic.PIT, pic.FP64, q=0.0)
    g.step(0.1)
    g.sync()
    start, ids = g.bins()
    assert start[-1] == 0 and ids.size == 0


def test_malformed_tree_rejected():
    with pytest.raises(pic.PicError) as e:
        make(2, np.array([1, 0, 0], np.uint8), np.zeros((2, 1)), np.zeros((2, 1)), pic.PIT, pic.FP64)
    assert e.value.code == -1


def test_nonfinite_input_rejected():
    x = np.full((2, 4), 0.5)
    x[0, 2] = np.nan
    with pytest.raises(pic.PicError) as e:
        make(2, W.uniform_tree_flags(2, 2), x, np.zeros((2, 4)), pic.PIT, pic.FP64)
    assert e.value.code == -3


def test_device_inputs_and_determinism():
    """Device-resident input gives the same result, and two runs agree bit for bit."""
    d = 2
    flags = W.random_tree_flags(2, 5, 0.3, 9, min_depth=2)
    x, v = W.random_particles(d, 30_000, 9, vmax=0.3)
    outs = []
    for dev in (False, True, True):
        xi = torch.from_numpy(x).cuda() if dev else x
        vi = torch.from_numpy(v).cuda() if dev else v
        g = make(d, flags, xi, vi, pic.PIT, pic.FP32_SPLIT, q=-1.0 / 30_000, sweeps=10)
        for _ in range(3):
            g.step(0.1)
        g.sync()
        outs.append((g.get_state(), g.bins(), g.deposit()))
    for o in outs[1:]:
        for a, b in zip(o[0], outs[0][0]):
            assert np.array_equal(a, b)
        assert np.array_equal(o[1][1], outs[0][1][1])
        assert np.array_equal(o[2], outs[0][2])


# ---------------------------------------------------------------------------
# brick path (uniform trees, PIT, split) against the generic path
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,depth,n,vmax", [(2, 4, 150_001, 2.0), (3, 3, 120_001, 0.3),
                                            (3, 4, 200_003, 2.0), (2, 3, 11_664, 0.05),
                                            (2, 3, 150_001, 0.3),     # every brick over the on-chip capacity
                                            (3, 3, 193_536, 0.3),     # every brick over it (27 bricks of 7,168)
                                            (3, 3, 170_100, 0.3),     # about one brick in ten over it
                                            (3, 3, 172_800, 0.3)])    # bricks at the capacity (2 x 3,200) on both sides
def test_brick_path_bit_identical_to_generic(d, depth, n, vmax):
    """Same state, bucket offsets and ids after several steps, with particles
    that stay, move to neighbour bricks and tunnel across several bricks."""
    flags = W.uniform_tree_flags(d, depth)
    x, v = W.random_particles(d, n, 31 + depth, vmax=vmax)
    kw = dict(q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=5, omega=0.8)
    fast = make(d, flags, x, v, pic.PIT, pic.FP32_SPLIT, path=pic.PATH_AUTO, **kw)
    slow = make(d, flags, x, v, pic.PIT, pic.FP32_SPLIT, path=pic.PATH_GENERIC, **kw)
    assert fast.info().brick == 1 and slow.info().brick == 0
    for step in range(3):
        fast.step(0.1)
        slow.step(0.1)
        fast.sync()
        slow.sync()
        for a, b in zip(fast.get_state(), slow.get_state()):
            assert np.array_equal(a, b), f"state differs at step {step}"
        sf, idf = fast.bins()
        ss, ids = slow.bins()
        assert np.array_equal(sf, ss) and np.array_equal(idf, ids)
        assert np.array_equal(fast.deposit(), slow.deposit())
        assert fast.stats().movers == slow.stats().movers
        assert fast.stats().max_bucket == slow.stats().max_bucket
        assert fast.stats().error == 0


# ---------------------------------------------------------------------------
# a9 re-refinement by the ppc criterion
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
@pytest.mark.parametrize("d,base,ppc,dmin,dmax,n", [(2, 2, 40, 2, 5, 60_001), (3, 1, 30, 1, 3, 40_001)])
def test_adapt_matches_oracle(d, base, ppc, dmin, dmax, n, scheme, precision):
    rng = np.random.default_rng(d * 100 + ppc)
    x = np.mod(0.5 + 0.12 * rng.standard_normal((d, n)), 1.0)
    v = rng.uniform(-0.3, 0.3, (d, n))
    flags0 = W.uniform_tree_flags(d, base)
    g = make(d, flags0, x, v, scheme, precision, q=-1.0 / n, sweeps=5)
    g.step(0.05)                       # move once on the base tree
    g.adapt(ppc, dmin, dmax)
    ot0 = oracle.Tree(d, flags0)
    prm = oracle.Params(scheme=scheme, q=-1.0 / n, sweeps=5, omega=0.8)
    if precision == pic.FP64:
        st = oracle.State64(ot0, x, v, prm)
        st.step(0.05)
        expect = oracle.retree64(d, st.x, ppc, dmin, dmax)
        assert np.array_equal(g.tree_flags(), expect)
        ot1 = oracle.Tree(d, expect)
        st1 = oracle.State64(ot1, st.x, st.v, prm, ids=st.ids)
        xs, vs = g.particles()
        assert rel_err(xs, st1.x) <= REL64 and rel_err(vs, st1.v) <= REL64
    else:
        st = oracle.State32(ot0, x, v, prm)
        st.step(0.05)
        expect = oracle.retree32(ot0, st.leaf, st.o, ppc, dmin, dmax)
        assert np.array_equal(g.tree_flags(), expect)
        ot1 = oracle.Tree(d, expect)
        leaf, o = st.leaf.copy(), st.o.copy()
        ot0.rebin32_into(ot1, leaf, o)
        key = ot1.keys32(scheme, leaf, o)
        start, perm = oracle.stable_bucket(key, ot1.n_keys(scheme))
        gl, go, gv = g.get_state()
        assert np.array_equal(gl, leaf[perm]) and np.array_equal(go, o[:, perm])
        assert np.array_equal(gv, st.v[:, perm])
        st1_ids = st.ids[perm]
        st1 = type("S", (), {"ids": st1_ids, "key": key[perm], "start": start})
    start, ids = g.bins()
    assert np.array_equal(ids, st1.ids)
    assert np.array_equal(g.keys(), st1.key)
    nb = 1 << d if scheme == pic.PIDT else 1
    assert np.array_equal(start, st1.start[::nb])
    # the adapted handle keeps stepping
    g.step(0.05)
    g.sync()


# ---------------------------------------------------------------------------
# a10 batches of independent instances
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_batch_equals_single_instances(scheme, precision):
    """Uneven instances (particle counts, depths 3-5) in one handle give the
    same keys, buckets, charges and states as separate handles."""
    insts = W.batched_langmuir(n_inst=7, n_min=300, n_max=30_000)
    kw = dict(scheme=scheme, precision=precision, sweeps=20, omega=0.8)
    g = pic.Pic.batch(2, [w.flags for w in insts], [w.x for w in insts], [w.v for w in insts],
                      qs=[w.q for w in insts], **kw)
    assert g.info().n_instances == len(insts)
    singles = [pic.Pic(2, w.flags, w.x, w.v, q=w.q, **kw) for w in insts]
    for _ in range(3):
        g.step(0.1)
        for s1 in singles:
            s1.step(0.1)
    g.sync()
    ps, vs, bs = g.instances()
    gstate = g.get_state()
    gstart, gids = g.bins()
    gkeys = g.keys()
    gQ = g.deposit()
    for i, s1 in enumerate(singles):
        sl = slice(ps[i], ps[i + 1])
        st1 = s1.get_state()
        tol = 0.0 if precision == pic.FP32_SPLIT else 1e-12
        loff = gstate[0][sl][0] - st1[0][0]            # the instance's first leaf in the batch
        assert np.array_equal(gstate[0][sl] - loff, st1[0])
        for a, b in zip(gstate[1:], st1[1:]):
            assert np.allclose(a[:, sl], b, rtol=tol, atol=tol)
        start1, ids1 = s1.bins()
        assert np.array_equal(gstart[bs[i]:bs[i + 1] + 1] - ps[i], start1)
        assert np.array_equal(gids[sl] - ps[i], ids1)
        k1 = s1.keys()
        assert np.array_equal(gkeys[sl] - gkeys[sl].min() + k1.min(), k1)
        assert np.allclose(gQ[vs[i]:vs[i + 1]], s1.deposit(), rtol=1e-6 if tol == 0 else 1e-12, atol=1e-12)


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
def test_crowded_buckets_match_oracle(scheme):
    """Thousands of particles per leaf, most of them moving: long mover
    segments (sorted in shared memory) and one over the in-memory limit keep
    the canonical order bit-exactly."""
    d = 2
    flags = W.uniform_tree_flags(d, 2)           # 81 leaves
    rng = np.random.default_rng(7)
    n = 160_000
    x = rng.random((d, n))
    x[:, :20_000] = 0.5 + 0.01 * rng.random((d, 20_000))   # one crowded corner: > 16384 in a bucket
    v = rng.uniform(-0.3, 0.3, (d, n))
    prm = oracle.Params(scheme=scheme, q=-1.0 / n, sweeps=5, omega=0.8)
    st = oracle.State64(oracle.Tree(d, flags), x, v, prm)
    g = make(d, flags, x, v, scheme, pic.FP64, q=-1.0 / n, sweeps=5, omega=0.8)
    for step in range(2):
        st.step(0.05)
        g.step(0.05)
        g.sync()
        start, ids = g.bins()
        assert np.array_equal(ids, st.ids), f"storage order step {step}"
        assert np.array_equal(g.keys(), st.key)


# ---------------------------------------------------------------------------
# the adaptive configurations, scaled down: steps with periodic re-refinement
# ---------------------------------------------------------------------------

def _retarget(st, tree, split):
    """Oracle state moved onto a new tree as fresh particles (all movers,
    stable by key in storage order), solver warm start reset."""
    if split:
        st.tree.rebin32_into(tree, st.leaf, st.o)
        st.tree = tree
        st.V = np.zeros(tree.n_vertices, np.float32)
    else:
        st.tree = tree
        st.V = np.zeros(tree.n_vertices)
    if hasattr(st, "key"):
        del st.key
    st.rebin()


def _run_adaptive(w, scheme, precision, ppc, dmin, dmax, every, steps):
    d = w.d
    prm = oracle.Params(scheme=scheme, q=w.q, qm=w.qm, ion=w.ion, sweeps=10, omega=0.8)
    tree = oracle.Tree(d, w.flags)
    split = precision == pic.FP32_SPLIT
    st = (oracle.State32 if split else oracle.State64)(tree, w.x, w.v, prm)
    g = make(d, w.flags, w.x, w.v, scheme, precision, q=w.q, qm=w.qm, ion=w.ion, sweeps=10, omega=0.8)
    for s in range(steps):
        if s % every == 0:
            g.adapt(ppc, dmin, dmax)
            flags = (oracle.retree32(st.tree, st.leaf, st.o, ppc, dmin, dmax) if split
                     else oracle.retree64(d, st.x, ppc, dmin, dmax))
            assert np.array_equal(g.tree_flags(), flags), f"tree at step {s}"
            _retarget(st, oracle.Tree(d, flags), split)
        st.step(w.dt)
        g.step(w.dt)
        g.sync()
        start, ids = g.bins()
        assert np.array_equal(ids, st.ids), f"storage order step {s}"
        assert np.array_equal(g.keys(), st.key), f"keys step {s}"
        if split:
            leaf, o, v = g.get_state()
            assert np.array_equal(leaf, st.leaf) and np.array_equal(o, st.o) and np.array_equal(v, st.v)
        else:
            x, v = g.particles()
            xs = st.x[:, np.argsort(st.ids)]
            xg = x[:, np.argsort(ids)]
            assert rel_err(xg, xs) <= REL64


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_gaussian_bump_with_rerefinement(scheme, precision):
    """2D Gaussian bump with a clipped Cauchy tail (tunnelling several cells),
    refined where a cell holds more than 64 particles, re-refined every 3
    steps: trees, keys, buckets and states match the oracle."""
    w = W.gaussian_bump(n=60_000, d=2, base_depth=3, finest_depth=5)
    _run_adaptive(w, scheme, precision, ppc=64, dmin=3, dmax=5, every=3, steps=7)


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_two_stream_pidt_with_rerefinement(precision):
    """3D two-stream (beams at +-8 cells per step), PIDT, refined above 32
    particles per cell, re-refined every 2 steps."""
    w = W.two_stream(n=60_000, d=3, base_depth=2)
    _run_adaptive(w, pic.PIDT, precision, ppc=32, dmin=2, dmax=3, every=2, steps=5)
