"""Pins of the CPU oracle against things other than itself: brute force,
lifts and drops applied as rewrite rules to a fixed point, closed forms of the d-linear finite
elements, conservation laws and the Vlasov-Poisson dispersion relation.

No GPU is needed.
"""
from __future__ import annotations

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import workloads as W
from tests import lift_drop_rules as LA

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
QS = 2 * 3 ** 18


def quantise_np(x):
    y = x - np.floor(x)
    y = np.where(y >= 1.0, 0.0, y)
    q = np.floor(y * float(QS)).astype(np.int64)
    return np.clip(q, 0, QS - 1)


def random_tree(d, depth, p, seed, min_depth=1):
    return W.random_tree_flags(d, depth, p, seed, min_depth=min_depth)


def leaves_brute(d, flags):
    """All leaves (level, coords) by a plain breadth-first walk of the flags."""
    root = LA.parse_tree(d, flags)
    out, stack = [], [root]
    while stack:
        c = stack.pop()
        if c.children:
            stack.extend(c.children)
        else:
            out.append((c.level, c.coords))
    return out


# ---------------------------------------------------------------------------
# a1 PIT owner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,depth,p,seed", [(2, 4, 0.35, 1), (2, 5, 0.25, 2), (3, 3, 0.3, 3)])
def test_pit_owner_brute_force(d, depth, p, seed):
    """Every particle's leaf is the unique leaf box containing its quantised
    position (exhaustive scan over all leaves)."""
    flags = random_tree(d, depth, p, seed)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    rng = np.random.default_rng(seed)
    x = rng.random((d, 400))
    Q = quantise_np(x)
    leaf = t.pit_owner(x)
    boxes = leaves_brute(d, flags)
    assert len(boxes) == t.n_leaves
    for pi in range(x.shape[1]):
        hits = [b for b in boxes
                if all(c * 2 * 3 ** (18 - b[0]) <= Q[a, pi] < (c + 1) * 2 * 3 ** (18 - b[0])
                       for a, c in enumerate(b[1]))]
        assert len(hits) == 1
        assert (lev[leaf[pi]], tuple(co[leaf[pi]])) == (hits[0][0], hits[0][1])


def test_quantisation_matches_exact_geometry():
    """Quantised containment equals exact rational containment except within
    one quantum of a face."""
    d, depth = 2, 5
    flags = random_tree(d, depth, 0.4, 7)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    rng = np.random.default_rng(7)
    x = rng.random((d, 300))
    leaf = t.pit_owner(x)
    for pi in range(x.shape[1]):
        l = int(lev[leaf[pi]])
        for a in range(d):
            xa = Fraction(float(x[a, pi]))
            lo = Fraction(int(co[leaf[pi], a]), 3 ** l)
            hi = Fraction(int(co[leaf[pi], a]) + 1, 3 ** l)
            if not lo <= xa < hi:
                assert min(abs(xa - lo), abs(xa - hi)) < Fraction(1, QS)


def test_pit_uniform_is_textbook_binning():
    """On a uniform tree the leaf is floor(x 3^D) (away from rounding at faces)."""
    d, D = 2, 4
    t = oracle.Tree(d, W.uniform_tree_flags(d, D))
    lev, co = t.leaf_info()
    x = np.random.default_rng(0).random((d, 5000))
    leaf = t.pit_owner(x)
    expect = np.floor(x * 3 ** D).astype(np.int64).T
    assert np.all(lev[leaf] == D)
    assert np.array_equal(co[leaf], expect)


@pytest.mark.parametrize("d,depth,p,seed,vmax", [(2, 4, 0.4, 11, 0.3), (2, 5, 0.3, 12, 0.05),
                                                 (3, 3, 0.35, 13, 0.4)])
def test_pit_owner_equals_lift_drop_fixed_point(d, depth, p, seed, vmax):
    """The PIT lift and drop rules, applied until neither fires, end in the
    oracle's owner (Theorem 1), with particles tunnelling several cells."""
    flags = random_tree(d, depth, p, seed)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    x0, v = W.random_particles(d, 300, seed, vmax=vmax)
    x1 = np.mod(x0 + v, 1.0)
    Q0, Q1 = quantise_np(x0).T.tolist(), quantise_np(x1).T.tolist()
    lit = LA.pit_by_rules(d, flags, Q0, Q1)
    leaf = t.pit_owner(x1)
    for pi in range(x1.shape[1]):
        assert lit[pi] == (lev[leaf[pi]], tuple(int(c) for c in co[leaf[pi]]))


@pytest.mark.parametrize("d,depth,p,seed,vmax", [(2, 4, 0.4, 11, 0.3), (2, 5, 0.3, 12, 0.05),
                                                 (3, 3, 0.35, 13, 0.4), (2, 5, 0.5, 14, 0.8)])
def test_pit_lift_counts_equal_rule_firings(d, depth, p, seed, vmax):
    """The oracle's lift and drop counts per particle (old leaf up to the
    deepest common ancestor, down to the new leaf) equal the number of times
    the lift and drop rules fire for it."""
    flags = random_tree(d, depth, p, seed)
    t = oracle.Tree(d, flags)
    x0, v = W.random_particles(d, 300, seed, vmax=vmax)
    x1 = np.mod(x0 + v, 1.0)
    Q0, Q1 = quantise_np(x0).T.tolist(), quantise_np(x1).T.tolist()
    counts = {}
    LA.pit_by_rules(d, flags, Q0, Q1, counts=counts)
    lifts, drops = t.pit_lifts(t.pit_owner(x0), t.pit_owner(x1))
    assert np.array_equal(lifts, counts["lifts"])
    assert np.array_equal(drops, counts["drops"])
    assert lifts.sum() > 0 and (lifts == 0).any()


def test_pit_lift_counts_closed_form_on_a_uniform_tree():
    """2D, depth 3 (27 x 27 leaves, leaf id = depth-first): a move to the
    neighbour inside the same parent is one lift and one drop; across a
    level-2 face two of each; across a level-1 face (or the periodic seam)
    three; a stayer none."""
    d, D = 2, 3
    t = oracle.Tree(d, W.uniform_tree_flags(d, D))
    lev, co = t.leaf_info()
    leaf_of = {tuple(int(c) for c in co[i]): i for i in range(len(lev))}
    pairs = [((4, 4), (4, 4), 0), ((0, 0), (1, 0), 1), ((2, 0), (3, 0), 2), ((8, 5), (9, 5), 3),
             ((26, 3), (0, 3), 3), ((4, 4), (5, 5), 1), ((4, 4), (13, 22), 3), ((1, 1), (0, 2), 1)]
    old = [leaf_of[a] for a, _, _ in pairs]
    new = [leaf_of[b] for _, b, _ in pairs]
    lifts, drops = t.pit_lifts(np.array(old), np.array(new))
    expect = np.array([k for _, _, k in pairs])
    assert np.array_equal(lifts, expect) and np.array_equal(drops, expect)


def test_pit_lift_counts_across_levels():
    """From a leaf on level 3 to a leaf on level 1 in another level-1 cell:
    three lifts to the root, one drop; and the reverse."""
    d = 2
    flags = np.zeros(1 + 9 + 9 + 9, np.uint8)
    flags[0] = 1          # root
    flags[1] = 1          # level-1 cell (0, 0)
    flags[10] = 1         # its first child, level-2 cell (0, 0)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    deep = int(np.flatnonzero(lev == 3)[0])
    coarse = [i for i in range(len(lev)) if lev[i] == 1 and tuple(co[i]) == (2, 2)][0]
    lifts, drops = t.pit_lifts(np.array([deep, coarse]), np.array([coarse, deep]))
    assert list(lifts) == [3, 1] and list(drops) == [1, 3]


def _unit_speed_particles(d, n, seed):
    """Uniform positions; velocities of uniform random direction and speed in
    [0, 1] (the particle workload of the paper's Section 6)."""
    rng = np.random.default_rng(seed)
    x = rng.random((d, n))
    g = rng.standard_normal((d, n))
    v = g / np.linalg.norm(g, axis=0) * rng.random(n)
    return x, v


def _mean_lifts(t, x, v, dt):
    li, dr = t.pit_lifts(t.pit_owner(x), t.pit_owner(np.mod(x + v * dt, 1.0)))
    return li.mean(), dr.mean()


@pytest.mark.parametrize("d,n", [(2, 20_000), (3, 30_000)])
def test_lifts_grow_with_the_time_step(d, n):
    """On a tree refined to a particles-per-cell bound, lifts per particle
    grow with the time step and, for small steps, in proportion to it (a
    particle leaves its cell with probability ~ |v| dt / h)."""
    x, v = _unit_speed_particles(d, n, 5)
    t = oracle.Tree(d, oracle.retree64(d, x, 30, 1, 8 if d == 2 else 5))
    lifts = [_mean_lifts(t, x, v, dt)[0] for dt in (1e-4, 1e-3, 1e-2, 1e-1)]
    assert all(a < b for a, b in zip(lifts, lifts[1:])), lifts
    assert 0.04 < lifts[1] / lifts[2] < 0.2, lifts


@pytest.mark.parametrize("d,n,ppcs", [(2, 20_000, (10, 30, 100, 300)), (3, 30_000, (4, 12, 40))])
def test_more_particles_per_cell_fewer_lifts(d, n, ppcs):
    """Section 6: the more particles a cell may hold before it is refined, the
    coarser the tree and the fewer lifts per particle at a fixed time step."""
    x, v = _unit_speed_particles(d, n, 6)
    lifts = []
    for ppc in ppcs:
        t = oracle.Tree(d, oracle.retree64(d, x, ppc, 1, 8 if d == 2 else 5))
        lifts.append(_mean_lifts(t, x, v, 1e-2)[0])
    assert all(a > b for a, b in zip(lifts, lifts[1:])), lifts


def test_lifts_of_stayers_movers_and_uniform_trees():
    """Stayers are neither lifted nor dropped, every particle that changes
    leaf is lifted at least once, and on a uniform tree every lift is matched
    by a drop."""
    d = 2
    x, v = _unit_speed_particles(d, 5000, 7)
    for flags, uniform in ((W.uniform_tree_flags(d, 4), True), (random_tree(d, 5, 0.35, 8), False)):
        t = oracle.Tree(d, flags)
        old, new = t.pit_owner(x), t.pit_owner(np.mod(x + 0.02 * v, 1.0))
        li, dr = t.pit_lifts(old, new)
        assert np.all((li == 0) == (old == new)) and np.all((dr == 0) == (old == new))
        assert (li > 0).any()
        if uniform:
            assert np.array_equal(li, dr)
        else:
            assert not np.array_equal(li, dr)  # moves between levels


# ---------------------------------------------------------------------------
# a2 PIDT owner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,depth,p,seed,vmax", [(2, 4, 0.4, 21, 0.2), (2, 5, 0.3, 22, 0.03),
                                                 (3, 3, 0.35, 23, 0.3)])
def test_pidt_owner_equals_lift_drop_fixed_point(d, depth, p, seed, vmax):
    """The PIDT lift (to the dual parent) and drop (to the child-level vertex)
    rules, applied until neither fires, end in the oracle's owner vertex
    (Theorem 2)."""
    flags = random_tree(d, depth, p, seed)
    t = oracle.Tree(d, flags)
    x0, v = W.random_particles(d, 250, seed, vmax=vmax)
    x1 = np.mod(x0 + v, 1.0)
    Q0, Q1 = quantise_np(x0).T.tolist(), quantise_np(x1).T.tolist()
    lit = LA.pidt_by_rules(d, flags, Q0, Q1)
    vl, vj = t.pidt_owner(x1)
    for pi in range(x1.shape[1]):
        assert lit[pi] == (int(vl[pi]), tuple(int(j) for j in vj[:, pi]))


@pytest.mark.parametrize("d,depth,p,seed", [(2, 5, 0.35, 24), (3, 3, 0.35, 25)])
def test_owners_on_faces_equal_fixed_point(d, depth, p, seed):
    """Positions exactly on cell faces and on dual-cell faces (the centre
    planes of the leaves): the half-open rules (a face belongs to the upper
    cell or dual cell) decide both owners, PIT and PIDT, as the lift and drop
    rules do."""
    flags = random_tree(d, depth, p, seed)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    rng = np.random.default_rng(seed)
    n = 400
    L = rng.integers(0, len(lev), n)
    s = 3 ** (18 - lev[L].astype(np.int64))
    kind = rng.integers(0, 3, (d, n))          # 0: lower face, 1: centre plane, 2: inside
    inside = (rng.random((d, n)) * (2 * s)).astype(np.int64)
    Q = 2 * co[L].T * s + np.where(kind == 0, 0, np.where(kind == 1, s, inside))
    x = (Q + 0.5) / QS                         # the middle of the quantum whose Q is on the face
    assert np.array_equal(quantise_np(x), Q)
    assert (kind == 1).sum() > n // 3 and (kind == 0).sum() > n // 3
    Ql = Q.T.tolist()
    pit = LA.pit_by_rules(d, flags, Ql, Ql)
    pidt = LA.pidt_by_rules(d, flags, Ql, Ql)
    leaf = t.pit_owner(x)
    vl, vj = t.pidt_owner(x)
    # the PIDT sort key: owner vertex id * 2^d + the quadrant 2^d - 1 - corner,
    # corner = the owner's place among the covering leaf's corners
    key = t.keys64(oracle.PIDT, x)
    pv_lev, pv_j = t.pidt_vertices()
    nc = 1 << d
    for pi in range(n):
        assert pit[pi] == (lev[leaf[pi]], tuple(int(c) for c in co[leaf[pi]]))
        assert pidt[pi] == (int(vl[pi]), tuple(int(j) for j in vj[:, pi]))
        lv, j = pidt[pi]
        vid = key[pi] // nc
        assert (int(pv_lev[vid]), tuple(int(c) for c in pv_j[vid])) == (lv, j)
        per = 3 ** lv
        corner = sum(1 << a for a in range(d) if j[a] != co[leaf[pi], a] % per)
        assert key[pi] % nc == nc - 1 - corner


def test_pidt_owner_brute_force():
    """Owner = vertex on the covering leaf's level whose dual cell contains the
    particle; scan over all leaf corners."""
    d = 2
    flags = random_tree(d, 5, 0.3, 31)
    t = oracle.Tree(d, flags)
    x = np.random.default_rng(31).random((d, 300))
    Q = quantise_np(x)
    vl, vj = t.pidt_owner(x)
    boxes = leaves_brute(d, flags)
    for pi in range(x.shape[1]):
        cands = set()
        for (l, c) in boxes:
            s = 2 * 3 ** (18 - l)
            if all(cc * s <= Q[a, pi] < (cc + 1) * s for a, cc in enumerate(c)):
                per = 3 ** l
                for e in range(1 << d):
                    j = tuple((c[a] + ((e >> a) & 1)) % per for a in range(d))
                    if LA.dual_contains(l, j, Q[:, pi].tolist()):
                        cands.add((l, j))
        assert len(cands) == 1
        assert cands.pop() == (int(vl[pi]), tuple(int(j) for j in vj[:, pi]))


def test_pidt_uniform_is_rounding():
    d, D = 3, 2
    t = oracle.Tree(d, W.uniform_tree_flags(d, D))
    x = np.random.default_rng(1).random((d, 3000))
    vl, vj = t.pidt_owner(x)
    assert np.all(vl == D)
    assert np.array_equal(vj, np.mod(np.floor(x * 3 ** D + 0.5), 3 ** D).astype(np.int64))


# ---------------------------------------------------------------------------
# a6 buckets
# ---------------------------------------------------------------------------

def test_stable_bucket_is_a_stable_sort():
    rng = np.random.default_rng(5)
    key = rng.integers(0, 50, 2000)
    start, perm = oracle.stable_bucket(key, 50)
    assert np.array_equal(np.sort(perm), np.arange(2000))
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(np.diff(start), np.bincount(key, minlength=50))


# ---------------------------------------------------------------------------
# a7 deposit
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,flags_fn", [
    (2, lambda: W.uniform_tree_flags(2, 3)),
    (2, lambda: random_tree(2, 5, 0.3, 41, min_depth=2)),
    (3, lambda: random_tree(3, 3, 0.3, 42, min_depth=1)),
])
@pytest.mark.parametrize("scheme", [oracle.PIT, oracle.PIDT])
def test_charge_conservation(d, flags_fn, scheme):
    """sum_v Q_v = q N + ion |domain| to 1e-12 relative, also with hanging
    vertices (their constraint weights sum to one)."""
    t = oracle.Tree(d, flags_fn())
    x, _ = W.random_particles(d, 3000, 3)
    q = -1.0 / 3000
    Q, tot = t.deposit64(scheme, x, q, 0.0)
    assert abs(Q.sum() - q * 3000) <= 1e-12 * abs(q * 3000)
    Qi, tot_i = t.deposit64(scheme, x, q, 1.0)
    assert abs(tot_i) < 1e-12
    ion, _ = t.vertex_aux()
    assert abs(ion.sum() - 1.0) < 1e-12


def test_single_particle_cic_weights():
    """One particle on a uniform 2D grid: the four corner charges are the
    bilinear (cloud-in-cell) weights times q."""
    D = 2
    t = oracle.Tree(2, W.uniform_tree_flags(2, D))
    pos = t.vertex_pos()
    x = np.array([[0.4], [0.7]])
    Q, _ = t.deposit64(oracle.PIT, x, 2.0, 0.0)
    h = 1.0 / 9
    i0, j0 = int(0.4 // h), int(0.7 // h)
    tx, ty = 0.4 / h - i0, 0.7 / h - j0
    expect = {(i0, j0): (1 - tx) * (1 - ty), (i0 + 1, j0): tx * (1 - ty),
              (i0, j0 + 1): (1 - tx) * ty, (i0 + 1, j0 + 1): tx * ty}
    for v in range(Q.size):
        key = (int(pos[0, v]), int(pos[1, v]))
        assert Q[v] == pytest.approx(2.0 * expect.get(key, 0.0), abs=1e-14)


def test_hanging_vertex_receives_no_charge_directly():
    """A particle in a fine leaf next to a coarse one: the hanging corner's
    weight is passed to the coarse face's vertices; total is conserved and
    every non-hanging vertex charge is non-negative for q > 0."""
    d = 2

    def refine(level, coords):
        if level == 0:
            return np.ones(len(coords), bool)
        return (coords[:, 0] == 1) & (coords[:, 1] == 1)

    flags = W.tree_flags_from_predicate(d, 2, refine)
    t = oracle.Tree(d, flags)
    assert t.n_vertices < sum(1 for _ in range(t.n_leaves * 4))
    x = np.array([[0.35], [0.36]])
    Q, _ = t.deposit64(oracle.PIT, x, 1.0, 0.0)
    assert Q.sum() == pytest.approx(1.0, abs=1e-15)
    assert np.all(Q >= 0)


# ---------------------------------------------------------------------------
# a8 solve and field (auxiliary)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,D", [(2, 3), (3, 2)])
def test_stiffness_fourier_eigenvalue(d, D):
    """On a uniform periodic grid the d-linear stiffness matrix acts on a
    Fourier mode by the closed-form eigenvalue of its 9-/27-point stencil."""
    t = oracle.Tree(d, W.uniform_tree_flags(d, D))
    pos = t.vertex_pos().astype(float)
    M = 3 ** D
    kv = [1, 2, 0][:d]
    th = [2 * math.pi * k / M for k in kv]
    V = np.cos(sum(th[a] * pos[a] for a in range(d)))
    y = t.apply64(V)
    c = [math.cos(x) for x in th]
    if d == 2:
        lam = 8 / 3 - (2 / 3) * (c[0] + c[1]) - (4 / 3) * c[0] * c[1]
    else:
        h = 1.0 / M
        lam = h * (8 / 3 - (4 / 6) * (c[0] * c[1] + c[1] * c[2] + c[0] * c[2])
                   - (8 / 12) * c[0] * c[1] * c[2])
    assert np.allclose(y, lam * V, atol=1e-12)


def test_stiffness_symmetric_semidefinite_adaptive():
    d = 2
    t = oracle.Tree(d, random_tree(d, 4, 0.35, 51, min_depth=2))
    rng = np.random.default_rng(0)
    u, w = rng.standard_normal((2, t.n_vertices))
    assert abs(u @ t.apply64(w) - w @ t.apply64(u)) < 1e-10
    assert np.allclose(t.apply64(np.ones(t.n_vertices)), 0.0, atol=1e-12)
    assert u @ t.apply64(u) > 0


def test_stiffness_energy_converges_on_adaptive_grid():
    """V^T A V of the interpolant of cos(2 pi x) approaches the exact energy
    2 pi^2 with second order on an adaptive grid with hanging vertices."""
    errs = []
    for D in (3, 4):
        def refine(level, coords, D=D):
            if level < D - 1:
                return np.ones(len(coords), bool)
            per = 3 ** level
            return coords[:, 0] < per // 2
        t = oracle.Tree(2, W.tree_flags_from_predicate(2, D, refine))
        pos = t.vertex_pos() / 3 ** t.depth
        V = np.cos(2 * math.pi * pos[0]) * np.cos(2 * math.pi * pos[1])
        errs.append(abs(V @ t.apply64(V) - 2 * math.pi ** 2))
    assert errs[1] < errs[0] / 5


def test_jacobi_reaches_discrete_solution():
    """Enough Jacobi sweeps solve A V = b for a single Fourier mode b:
    V = b / lambda (closed form on the uniform periodic grid)."""
    D = 2
    t = oracle.Tree(2, W.uniform_tree_flags(2, D))
    pos = t.vertex_pos().astype(float)
    th = 2 * math.pi / 9
    b = np.cos(th * pos[0])
    lam = 2 - 2 * math.cos(th)
    V = np.zeros(t.n_vertices)
    res = t.solve64(b, V, 3000, 0.8)
    assert res < 1e-10
    assert np.allclose(V, b / lam, atol=1e-9)


def test_efield_central_difference_closed_form():
    D = 3
    t = oracle.Tree(2, W.uniform_tree_flags(2, D))
    pos = t.vertex_pos().astype(float)
    M = 3 ** D
    h = 1.0 / M
    th = 2 * math.pi / M
    V = np.cos(th * pos[0])
    E = t.efield64(V)
    assert np.allclose(E[0], math.sin(th) / h * np.sin(th * pos[0]), atol=1e-12)
    assert np.allclose(E[1], 0.0, atol=1e-12)


# ---------------------------------------------------------------------------
# a3 + a4 gather and leapfrog push
# ---------------------------------------------------------------------------

def test_gather_partition_of_unity_and_constant_field_trajectory():
    """A constant vertex field gathers exactly (shape functions sum to one,
    hanging corners interpolate constants); leapfrog then follows the closed
    form v_n = v_0 + n a dt, x_n = x_0 + n v_0 dt + n(n+1)/2 a dt^2."""
    d = 2
    t = oracle.Tree(d, random_tree(d, 4, 0.35, 61, min_depth=2))
    x, v = W.random_particles(d, 200, 61, vmax=0.01)
    E = np.zeros((d, t.n_vertices))
    E[0], E[1] = 0.25, -0.5
    Ep = t.gather64(x, E)
    assert np.allclose(Ep[0], 0.25, atol=1e-14) and np.allclose(Ep[1], -0.5, atol=1e-14)
    qm, dt, n = -2.0, 0.01, 7
    xs, vs = x.copy(), v.copy()
    for _ in range(n):
        t.push64(xs, vs, E, qm, dt)
    a = qm * np.array([[0.25], [-0.5]])
    assert np.allclose(vs, v + n * a * dt, atol=1e-14)
    xe = np.mod(x + n * v * dt + n * (n + 1) / 2 * a * dt * dt, 1.0)
    dx = np.abs(xs - xe)
    assert np.all(np.minimum(dx, 1 - dx) < 1e-13)


# ---------------------------------------------------------------------------
# FP32 split mirror
# ---------------------------------------------------------------------------

def test_split_move_stays_in_covering_leaf():
    """After a split push the stored leaf covers the reconstructed position
    and equals the FP64 owner of it (away from a face by 2^-20 cells)."""
    d = 2
    flags = random_tree(d, 5, 0.3, 71, min_depth=2)
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 3000, 71, vmax=0.3)
    leaf, o, vf = t.split_from64(x, v)
    E = np.zeros((d, t.n_vertices), np.float32)
    t.push32(leaf, o, vf, E, -1.0, 0.5)
    assert np.all((o >= 0) & (o < 1))
    xr = t.split_to64(leaf, o)
    owner = t.pit_owner(xr)
    near = np.any((o < 2 ** -20) | (o > 1 - 2 ** -20), axis=0)
    assert np.all((owner == leaf) | near)
    # and it matches the FP64 move up to FP32 rounding of the displacement
    x64 = np.mod(x + v.astype(np.float32).astype(np.float64) * 0.5, 1.0)
    dx = np.abs(xr - x64)
    assert np.all(np.minimum(dx, 1 - dx) < 1e-5)


def test_split_lift_and_drop_between_trees():
    """Re-locating split particles into a coarser then a finer tree keeps them
    in covering leaves and returns to the same leaf."""
    d = 2
    fine = oracle.Tree(d, W.uniform_tree_flags(d, 4))
    coarse = oracle.Tree(d, W.uniform_tree_flags(d, 2))
    x, v = W.random_particles(d, 2000, 72)
    leaf, o, _ = fine.split_from64(x, v)
    l2, o2 = leaf.copy(), o.copy()
    fine.rebin32_into(coarse, l2, o2)
    assert np.array_equal(l2, coarse.pit_owner(coarse.split_to64(l2, o2)))
    coarse.rebin32_into(fine, l2, o2)
    near = np.any((o < 2 ** -18) | (o > 1 - 2 ** -18), axis=0)
    assert np.all((l2 == leaf) | near)
    assert np.max(np.abs(o2 - o)) < 1e-5


# ---------------------------------------------------------------------------
# a9 re-refinement
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ppc", [8, 40])
def test_retree_ppc_criterion(ppc):
    d, dmin, dmax = 2, 2, 5
    rng = np.random.default_rng(ppc)
    x = np.mod(0.5 + 0.08 * rng.standard_normal((d, 4000)), 1.0)
    flags = oracle.retree64(d, x, ppc, dmin, dmax)
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    counts = np.bincount(t.pit_owner(x), minlength=t.n_leaves)
    assert lev.min() >= dmin and lev.max() <= dmax
    assert np.all((counts <= ppc) | (lev == dmax))
    # every refined cell on level >= dmin holds more than ppc particles
    root = LA.parse_tree(d, flags)
    Q = quantise_np(x)
    stack = [root]
    while stack:
        c = stack.pop()
        if c.children:
            stack.extend(c.children)
            if c.level >= dmin:
                s = 2 * 3 ** (18 - c.level)
                inside = np.all([(Q[a] >= c.coords[a] * s) & (Q[a] < (c.coords[a] + 1) * s)
                                 for a in range(d)], axis=0)
                assert inside.sum() > ppc


# ---------------------------------------------------------------------------
# Physics: Langmuir dispersion (Appendix A)
# ---------------------------------------------------------------------------

def kinetic_root(klam):
    """Least-damped root of the Vlasov-Poisson Langmuir dispersion relation
    1 + (1 + zeta Z(zeta)) / (k lambda_D)^2 = 0, zeta = omega / (sqrt 2 k v_th),
    with the plasma dispersion function from scipy's Faddeeva routine."""
    sp = pytest.importorskip("scipy.special")
    opt = pytest.importorskip("scipy.optimize")

    def F(vv):
        w = vv[0] + 1j * vv[1]
        z = w / (math.sqrt(2) * klam)
        r = 1 + (1 + z * 1j * math.sqrt(math.pi) * sp.wofz(z)) / klam ** 2
        return [r.real, r.imag]

    return opt.fsolve(F, [math.sqrt(1 + 3 * klam ** 2), -0.01])[0]


def bohm_gross(klam):
    return math.sqrt(1 + 3 * klam ** 2)


def test_golden_appendix_a_cut():
    """The paper's (k1, k2) cut at omega = 1.14 lies on the Bohm-Gross curve at
    k lambda_D ~ 0.316 (Appendix A), the same k lambda_D as the 27x27 run."""
    g = json.load(open(os.path.join(GOLDEN, "appendix_a.json")))
    klam = math.sqrt((g["omega_cut"] ** 2 - 1) / 3)
    assert abs(klam - 2 * math.pi * g["langmuir_27x27"]["vth"]) < 0.01
    assert bohm_gross(klam) == pytest.approx(g["omega_cut"], rel=1e-12)


def measure_omega(st, w, tree, steps, t0):
    from scipy.optimize import curve_fit
    pos = tree.vertex_pos()
    M = 3 ** tree.depth
    ph = np.exp(-2j * np.pi * w.k_mode * pos[0] / M)
    amps = []
    for _ in range(steps):
        Q, *_ = st.step(w.dt)
        amps.append(float((np.asarray(Q, np.float64) * ph).sum().real))
    tt = np.arange(steps) * w.dt
    m = tt >= t0
    f = lambda t, a, om, p, g: a * np.cos(om * t + p) * np.exp(g * t)
    popt, _ = curve_fit(f, tt[m], np.array(amps)[m], p0=[amps[0], 1.15, 0.0, 0.0])
    return abs(popt[1])


@pytest.mark.parametrize("vth,t0,ref", [(0.05, 6.0, "kinetic"), (0.02, 3.0, "bohm_gross")])
def test_langmuir_frequency(vth, t0, ref):
    """27x27 periodic grid, omega_p dt = 0.1, k = 2 pi, quiet start with 64
    particles per cell: the measured frequency is within 2% of the
    Vlasov-Poisson root; at k lambda_D = 0.126 also within 2% of Bohm-Gross."""
    pytest.importorskip("scipy")
    w = W.langmuir(2, 3, 64, vth=vth)
    tree = oracle.Tree(2, w.flags)
    st = oracle.State64(tree, w.x, w.v, oracle.Params(q=w.q, qm=w.qm, ion=w.ion, sweeps=400,
                                                      omega=1.0))
    st.init_leapfrog(w.dt)
    om = measure_omega(st, w, tree, 200, t0)
    klam = 2 * math.pi * vth
    target = kinetic_root(klam) if ref == "kinetic" else bohm_gross(klam)
    assert abs(om / target - 1) < 0.02, (om, target)
