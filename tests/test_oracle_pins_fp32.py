"""Pins of the oracle's FP32 split-precision mirror and of its FP64 deposit on
trees with hanging vertices, against things other than the oracle itself:

* the d-linear finite-element basis evaluated from the tree's geometry alone
  (leaf boxes, hanging points interpolated on the coarsest leaf whose closure
  holds them), never from the oracle's own corner-expansion tables;
* exact rational geometry for the owner vertex of a split particle;
* closed forms on uniform periodic grids (a Fourier mode under damped
  Jacobi, the central difference of a cosine, linear fields reproduced by
  d-linear interpolation, the cold Langmuir oscillation at t = -dt/2);
* the FP64 oracle, itself pinned, within a worst-case FP32 rounding bound
  derived from the number of operations (u = 2^-24 per operation).

No GPU is needed.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import workloads as W
from tests import lift_drop_rules as LA

U32 = 2.0 ** -24       # unit roundoff of FP32 (round to nearest)
QS = 2 * 3 ** 18


def quantise_np(x):
    y = x - np.floor(x)
    y = np.where(y >= 1.0, 0.0, y)
    q = np.floor(y * float(QS)).astype(np.int64)
    return np.clip(q, 0, QS - 1)


def leaves_of(d, flags):
    """Every leaf as (level, coords), by a plain walk of the refinement flags."""
    root = LA.parse_tree(d, flags)
    out, stack = [], [root]
    while stack:
        c = stack.pop()
        if c.children:
            stack.extend(c.children)
        else:
            out.append((c.level, c.coords))
    return out


class FEGeometry:
    """The d-linear finite-element space of a spacetree from geometry alone.

    Points are integer coordinates in units of 3^-D (D the deepest level),
    periodic modulo M = 3^D.  A point P is a vertex (non-hanging) iff it is a
    corner of the coarsest leaf whose closed box contains it; otherwise its
    nodal value is the d-linear interpolation, on that leaf, of the nodal values
    at the leaf's corners (applied recursively: a corner may hang too).  This is
    the conforming space with hanging vertices constrained to the coarse face,
    built without any of the oracle's tables."""

    def __init__(self, d, flags):
        self.d = d
        self.leaves = leaves_of(d, flags)
        self.D = max(l for l, _ in self.leaves)
        self.M = 3 ** self.D
        self.lo = np.array([[c * 3 ** (self.D - l) for c in co] for l, co in self.leaves], np.int64)
        self.size = np.array([3 ** (self.D - l) for l, _ in self.leaves], np.int64)
        self.level = np.array([l for l, _ in self.leaves], np.int64)
        self._memo = {}
        self.corners = list(itertools.product((0, 1), repeat=d))  # (e_x, e_y[, e_z])

    def nodal(self, P):
        """{vertex point: weight} such that the basis function of vertex v has
        value weight at point P."""
        P = tuple(int(p) % self.M for p in P)
        if P in self._memo:
            return self._memo[P]
        off = (np.array(P)[None, :] - self.lo) % self.M
        inside = np.all(off <= self.size[:, None], axis=1)
        cand = np.nonzero(inside)[0]
        L = cand[np.argmax(self.size[cand])]
        s = int(self.size[L])
        o = [int(v) for v in off[L]]
        if all(v in (0, s) for v in o):
            res = {P: 1.0}
        else:
            res = {}
            t = [Fraction(v, s) for v in o]
            for e in self.corners:
                w = Fraction(1)
                for a in range(self.d):
                    w *= t[a] if e[a] else 1 - t[a]
                if w == 0:
                    continue
                C = tuple(int(self.lo[L, a]) + e[a] * s for a in range(self.d))
                for v, wv in self.nodal(C).items():
                    res[v] = res.get(v, 0.0) + float(w) * wv
        self._memo[P] = res
        return res

    def leaf_corner_nodal(self, L):
        s = int(self.size[L])
        return [self.nodal(tuple(int(self.lo[L, a]) + e[a] * s for a in range(self.d))) for e in self.corners]

    def leaf_of(self, x):
        """Index into self.leaves of the leaf covering each position (exact
        containment of the quantised position, half-open boxes)."""
        Q = quantise_np(x)                              # (d, n)
        unit = 2 * 3 ** (18 - self.D)
        lo = self.lo * unit
        hi = (self.lo + self.size[:, None]) * unit
        out = np.full(x.shape[1], -1, np.int64)
        for L in range(len(self.leaves)):
            inside = np.all((Q >= lo[L][:, None]) & (Q < hi[L][:, None]), axis=0)
            assert np.all(out[inside] == -1)
            out[inside] = L
        assert np.all(out >= 0)
        return out

    def deposit(self, x, q, ion):
        """{vertex point: q sum_p phi_v(x_p) + ion integral(phi_v)} in FP64."""
        Qv = {}
        owner = self.leaf_of(x)
        for L in np.unique(owner):
            nod = self.leaf_corner_nodal(L)
            idx = np.nonzero(owner == L)[0]
            l = int(self.level[L])
            c = self.leaves[L][1]
            tl = np.stack([np.clip(x[a, idx] * 3.0 ** l - c[a], 0.0, 1.0) for a in range(self.d)])
            for e, ne in zip(self.corners, nod):
                phi = np.ones(len(idx))
                for a in range(self.d):
                    phi = phi * (tl[a] if e[a] else 1.0 - tl[a])
                s = float(phi.sum())
                for v, w in ne.items():
                    Qv[v] = Qv.get(v, 0.0) + q * w * s
        for L in range(len(self.leaves)):
            vol = (float(self.size[L]) / self.M) ** self.d
            for ne in self.leaf_corner_nodal(L):
                for v, w in ne.items():
                    Qv[v] = Qv.get(v, 0.0) + ion * vol / len(self.corners) * w
        return Qv


def vertex_index(tree):
    pos = tree.vertex_pos()
    return {tuple(int(p) for p in pos[:, v]): v for v in range(pos.shape[1])}


def deep_jump_tree(d):
    """A tree without 2:1 balance: one corner cell refined three levels below
    its coarse neighbours, so hanging points resolve through hanging points."""
    def refine(level, coords):
        if level == 0:
            return np.ones(len(coords), bool)
        return np.all(coords == 3 ** level - 1, axis=1) | np.all(coords == 0, axis=1) & (level == 1)
    return W.tree_flags_from_predicate(d, 4 if d == 2 else 3, refine)


TREES = [
    (2, lambda: W.random_tree_flags(2, 4, 0.35, 101, min_depth=1)),
    (2, lambda: deep_jump_tree(2)),
    (3, lambda: W.random_tree_flags(3, 3, 0.25, 102, min_depth=1)),
]


# ---------------------------------------------------------------------------
# FP64 deposit, vertex by vertex, on trees with hanging vertices
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,flags_fn", TREES)
@pytest.mark.parametrize("scheme", [oracle.PIT, oracle.PIDT])
def test_deposit64_per_vertex_brute_force(d, flags_fn, scheme):
    """Q_v = q sum_p phi_v(x_p) + ion integral(phi_v) (Section 3 item 1 with
    d-linear R; hanging vertices constrained) at every vertex, with phi_v
    evaluated from the tree's geometry alone; the vertex set itself is the set
    of non-hanging points of that geometry."""
    flags = flags_fn()
    t = oracle.Tree(d, flags)
    geo = FEGeometry(d, flags)
    assert geo.D == t.depth
    x, _ = W.random_particles(d, 1500 if d == 2 else 2500, 7)
    q, ion = -0.37 / x.shape[1], 0.8
    Qb = geo.deposit(x, q, ion)
    vid = vertex_index(t)
    assert set(Qb) == set(vid), "vertex sets differ"
    Q, _ = t.deposit64(scheme, x, q, ion)
    ref = np.zeros(len(vid))
    for P, v in vid.items():
        ref[v] = Qb[P]
    scale = np.abs(ref).max()
    assert np.max(np.abs(Q - ref)) <= 1e-12 * scale
    # the tree really has hanging points (a nodal expansion with >1 entry)
    assert any(len(nd) > 1 for nd in geo._memo.values())


# ---------------------------------------------------------------------------
# FP32 deposit against the exact load within the FP32 rounding bound
# ---------------------------------------------------------------------------

def incidences_per_vertex(t):
    ptr, vid, w = t.corner_expansion()
    return np.bincount(vid, minlength=t.n_vertices)


@pytest.mark.parametrize("d,flags_fn", TREES + [(2, lambda: W.uniform_tree_flags(2, 3)),
                                                (3, lambda: W.uniform_tree_flags(3, 2))])
@pytest.mark.parametrize("scheme", [oracle.PIT, oracle.PIDT])
def test_deposit32_within_rounding_bound(d, flags_fn, scheme):
    """The FP32 deposit of split particles equals the FP64 deposit of the same
    (exactly reconstructed) positions to within its worst-case rounding error:
    per vertex, every weight carries <= 2d roundings, the per-leaf partial sums
    <= m_max - 1, the vertex sum <= k_v, the scaling and the ion term two more,
    each at most u times the sum of the (non-negative) terms."""
    flags = flags_fn()
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 4000, 8)
    leaf, o, _ = t.split_from64(x, v)
    xr = t.split_to64(leaf, o)
    q, ion = np.float32(-1.0 / 4000), np.float32(1.0)
    Q32, tot32 = t.deposit32(scheme, leaf, o, q, ion)
    S, _ = t.deposit64(scheme, xr, 1.0, 0.0)         # sum_p phi_v(x_p), non-negative terms
    I, _ = t.vertex_aux()                              # integral(phi_v)
    Q64 = float(q) * S + float(ion) * I
    m_max = int(np.bincount(leaf, minlength=t.n_leaves).max())
    k = incidences_per_vertex(t)
    bound = (m_max + k + 2 * d + 6) * U32 * 1.01 * (abs(float(q)) * S + abs(float(ion)) * I)
    err = np.abs(Q32.astype(np.float64) - Q64)
    assert np.all(err <= bound), float((err / bound).max())
    # and the charge balance: every vertex bound summed
    assert abs(tot32 - Q64.sum()) <= bound.sum() + t.n_vertices * U32 * np.abs(Q64).max()


def test_deposit32_single_particle_cic_weights():
    """One split particle on a uniform 2D grid: the four vertex charges are q
    times the bilinear weights of its offset (each one product of two FP32
    factors, so exact to 2 u)."""
    t = oracle.Tree(2, W.uniform_tree_flags(2, 2))
    x = np.array([[0.4], [0.7]])
    leaf, o, _ = t.split_from64(x, np.zeros((2, 1)))
    Q, _ = t.deposit32(oracle.PIT, leaf, o, np.float32(2.0), np.float32(0.0))
    pos = t.vertex_pos()
    h = 1.0 / 9
    i0, j0 = int(0.4 // h), int(0.7 // h)
    tx, ty = float(o[0, 0]), float(o[1, 0])
    expect = {(i0, j0): (1 - tx) * (1 - ty), (i0 + 1, j0): tx * (1 - ty),
              (i0, j0 + 1): (1 - tx) * ty, (i0 + 1, j0 + 1): tx * ty}
    for vv in range(Q.size):
        e = 2.0 * expect.get((int(pos[0, vv]), int(pos[1, vv])), 0.0)
        assert abs(float(Q[vv]) - e) <= 4 * U32 * 2.0


# ---------------------------------------------------------------------------
# FP32 solve and field
# ---------------------------------------------------------------------------

def stencil_eigenvalue(d, th, M):
    c = [math.cos(x) for x in th]
    if d == 2:
        return 8 / 3 - (2 / 3) * (c[0] + c[1]) - (4 / 3) * c[0] * c[1]
    h = 1.0 / M
    return h * (8 / 3 - (4 / 6) * (c[0] * c[1] + c[1] * c[2] + c[0] * c[2]) - (8 / 12) * c[0] * c[1] * c[2])


@pytest.mark.parametrize("d,D,sweeps", [(2, 3, 7), (2, 2, 60), (3, 2, 9)])
def test_solve32_single_mode_closed_form(d, D, sweeps):
    """Damped Jacobi from V = 0 on a single Fourier mode b of a uniform periodic
    grid: V_s = (1 - r^s) b / lambda with r = 1 - omega lambda / diag, and the
    residual norm ||b - A V_s|| = |r|^s ||b|| (closed form of the iteration on
    an eigenvector).  FP32: every sweep adds at most (3^d + 4) roundings of
    terms bounded by |b| / lambda."""
    t = oracle.Tree(d, W.uniform_tree_flags(d, D))
    M = 3 ** D
    pos = t.vertex_pos().astype(float)
    kv = [1, 2, 1][:d]
    th = [2 * math.pi * k / M for k in kv]
    b = np.cos(sum(th[a] * pos[a] for a in range(d)))
    lam = stencil_eigenvalue(d, th, M)
    diag = 8 / 3 if d == 2 else 8 / 3 / M
    om = 0.8
    r = 1 - om * lam / diag
    V = np.zeros(t.n_vertices, np.float32)
    res = t.solve32(b.astype(np.float32), V, sweeps, np.float32(om))
    Vx = (1 - r ** sweeps) * b / lam
    tol = (sweeps * (3 ** d + 4) + 8) * U32 * (np.abs(b).max() / lam) * 2
    assert np.max(np.abs(V - Vx)) <= tol
    rx = abs(r) ** sweeps * np.linalg.norm(b)
    assert abs(res - rx) <= 1e-4 * np.linalg.norm(b) + rx * 1e-4


def test_solve32_tracks_solve64_on_adaptive_tree():
    """On an adaptive tree with hanging vertices the FP32 sweeps stay within
    the accumulated FP32 rounding of the FP64 sweeps: per sweep at most
    (k_max 2^d + 6) roundings of terms bounded by the iterate's scale (the
    damped iteration does not amplify an error in the energy norm)."""
    d = 2
    t = oracle.Tree(d, W.random_tree_flags(d, 4, 0.35, 103, min_depth=2))
    rng = np.random.default_rng(3)
    Q = rng.standard_normal(t.n_vertices)
    Q -= Q.mean()
    sweeps = 25
    V64 = np.zeros(t.n_vertices)
    r64 = t.solve64(Q.astype(np.float32).astype(np.float64), V64, sweeps, 0.8)
    V32 = np.zeros(t.n_vertices, np.float32)
    r32 = t.solve32(Q.astype(np.float32), V32, sweeps, np.float32(0.8))
    k = incidences_per_vertex(t).max()
    _, diag = t.vertex_aux()
    scale = np.abs(V64).max() + np.abs(Q).max() / diag.min()
    tol = sweeps * (k * 2 ** d + 6) * U32 * scale * 4
    assert np.max(np.abs(V32 - V64)) <= tol
    assert abs(r32 - r64) <= 1e-3 * r64


def test_efield32_central_difference_closed_form():
    """E = -grad V of V = cos(theta i) on a uniform grid is sin(theta)/h
    sin(theta i) in x and 0 in y (central differences), to FP32 rounding."""
    D = 3
    t = oracle.Tree(2, W.uniform_tree_flags(2, D))
    pos = t.vertex_pos().astype(float)
    M = 3 ** D
    h = 1.0 / M
    th = 2 * math.pi / M
    V = np.cos(th * pos[0]).astype(np.float32)
    E = t.efield32(V)
    ex = math.sin(th) / h * np.sin(th * pos[0])
    tol = 16 * U32 / h
    assert np.max(np.abs(E[0] - ex)) <= tol
    assert np.max(np.abs(E[1])) <= tol


@pytest.mark.parametrize("d,flags_fn", TREES)
def test_efield32_tracks_efield64(d, flags_fn):
    """On adaptive trees the FP32 field of the same potential is the FP64 one
    to within the rounding of its differences: |V| / h_min times a few u per
    incident leaf."""
    t = oracle.Tree(d, flags_fn())
    rng = np.random.default_rng(5)
    V = rng.standard_normal(t.n_vertices).astype(np.float32)
    E32 = t.efield32(V)
    E64 = t.efield64(V.astype(np.float64))
    k = incidences_per_vertex(t).max()
    tol = (k * 2 ** d + 8) * U32 * 2 * np.abs(V).max() * 3 ** t.depth * 4
    assert np.max(np.abs(E32 - E64)) <= tol


# ---------------------------------------------------------------------------
# FP32 gather and push
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,flags_fn", TREES)
def test_gather32_reproduces_constant_and_linear_fields(d, flags_fn):
    """d-linear interpolation with hanging corners constrained to the coarse
    face reproduces constants everywhere and linear functions inside the
    periodic cell (leaves that do not touch the wrap-around face): the FP32
    gather does so to a few u."""
    flags = flags_fn()
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 3000, 9)
    leaf, o, _ = t.split_from64(x, v)
    pos = t.vertex_pos() / 3 ** t.depth
    alpha = np.array([0.3, -0.2, 0.7][:d])
    beta = np.array([[0.5, -1.0, 0.25], [0.75, 0.5, -0.5], [-0.25, 1.0, 0.125]])[:d, :d]
    E = (alpha[:, None] + beta @ pos).astype(np.float32)
    Ep = t.gather32(leaf, o, E)
    # leaves whose corner values resolve without crossing the periodic seam
    geo = FEGeometry(d, flags)
    lev, co = t.leaf_info()
    gl = {(int(l), tuple(int(c) for c in cc)): i for i, (l, cc) in enumerate(geo.leaves)}
    clean = np.zeros(t.n_leaves, bool)
    for L in range(t.n_leaves):
        G = gl[(int(lev[L]), tuple(int(c) for c in co[L]))]
        s = int(geo.size[G])
        ok = True
        for e, nd in zip(geo.corners, geo.leaf_corner_nodal(G)):
            C = [int(geo.lo[G, a]) + e[a] * s for a in range(d)]
            for P in nd:
                ok &= all(C[a] < geo.M and abs(C[a] - P[a]) < geo.M // 2 for a in range(d))
        clean[L] = ok
    away = clean[leaf]
    assert away.sum() > 500
    xr = t.split_to64(leaf, o)
    expect = alpha[:, None] + beta @ xr
    mag = np.abs(alpha)[:, None] + np.abs(beta) @ np.ones_like(xr)
    assert np.all(np.abs(Ep - expect)[:, away] <= 32 * U32 * mag[:, away])
    Ec = np.broadcast_to(alpha[:, None], E.shape).astype(np.float32).copy()
    Ep = t.gather32(leaf, o, Ec)
    assert np.all(np.abs(Ep - alpha[:, None]) <= 16 * U32 * np.abs(alpha)[:, None])


@pytest.mark.parametrize("d,flags_fn", TREES)
def test_gather32_tracks_gather64(d, flags_fn):
    """A random vertex field gathered in FP32 at split particles equals the FP64
    gather at the reconstructed positions to within 2^d (k_max + 2d + 2)
    roundings of the field's magnitude."""
    t = oracle.Tree(d, flags_fn())
    x, v = W.random_particles(d, 3000, 10)
    leaf, o, _ = t.split_from64(x, v)
    E = W.random_field(d, t.n_vertices, 10, 1.0)
    E32 = t.gather32(leaf, o, E)
    E64 = t.gather64(t.split_to64(leaf, o), E.astype(np.float64))
    k = incidences_per_vertex(t).max()
    assert np.max(np.abs(E32 - E64)) <= 2 ** d * (k + 2 * d + 2) * U32 * 2


def test_push32_constant_field_kick_and_drift():
    """In a constant field the split push kicks every particle by q/m dt E (the
    gathered field equals E up to the rounding of the FP32 weights), and the
    new position is the FP64 drift by v' dt to FP32 rounding of the cell-unit
    displacement."""
    d = 2
    t = oracle.Tree(d, W.random_tree_flags(d, 4, 0.35, 104, min_depth=2))
    x, v = W.random_particles(d, 2000, 11, vmax=0.02)
    leaf, o, vf = t.split_from64(x, v)
    E = np.zeros((d, t.n_vertices), np.float32)
    E[0], E[1] = 0.5, -0.25
    qm, dt = -1.0, 0.1
    v0 = vf.copy()
    x0 = t.split_to64(leaf, o)
    t.push32(leaf, o, vf, E, qm, dt)
    qmdt = float(np.float32(qm * dt))
    for a, Ea in ((0, 0.5), (1, -0.25)):
        # the gathered field is E (1 + delta), |delta| <= (2^d + 2d) u (weights of
        # d roundings each, summed over 2^d corners); then one product, one sum
        expect = v0[a].astype(np.float64) + qmdt * Ea
        tol = abs(qmdt * Ea) * (2 ** d + 2 * d + 1) * U32 + np.abs(expect) * U32
        assert np.all(np.abs(vf[a] - expect) <= tol)
    xr = t.split_to64(leaf, o)
    dx = np.abs(xr - np.mod(x0 + vf.astype(np.float64) * dt, 1.0))
    assert np.all(np.minimum(dx, 1 - dx) < 1e-6)


# ---------------------------------------------------------------------------
# split PIDT owner (quadrant rule) against exact rational geometry
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("d,flags_fn", TREES)
def test_keys32_pidt_owner_exact_geometry(d, flags_fn):
    """The PIDT key of a split particle names the vertex, on its leaf's level,
    whose half-open dual cell [(j - 1/2) h, (j + 1/2) h) holds the exact
    rational position (c + o) / 3^l (Theorem 2 end state; a point on a dual
    face belongs to the upper cell), found by scanning every vertex of that
    level.  Offsets exactly 1/2 and one ulp either side are included."""
    flags = flags_fn()
    t = oracle.Tree(d, flags)
    lev, co = t.leaf_info()
    rng = np.random.default_rng(12)
    n = 600
    leaf = rng.integers(0, t.n_leaves, n).astype(np.int32)
    specials = np.array([0.5, np.nextafter(np.float32(0.5), np.float32(0)),
                         np.nextafter(np.float32(0.5), np.float32(1)), 0.0], np.float32)
    o = rng.random((d, n)).astype(np.float32)
    pick = rng.random((d, n)) < 0.5
    o = np.where(pick, specials[rng.integers(0, 4, (d, n))], o).astype(np.float32)
    key = t.keys32(oracle.PIDT, leaf, o)
    nc = 1 << d
    pv_lev, pv_j = t.pidt_vertices()
    for p in range(n):
        L = leaf[p]
        l = int(lev[L])
        per = 3 ** l
        X = [Fraction(int(co[L, a])) + Fraction(float(o[a, p])) for a in range(d)]   # cell units
        # dual cells are boxes: scan every vertex index of the level per axis
        axis_hits = []
        for Xa in X:
            axis_hits.append([jj for jj in range(per) if any(
                Fraction(2 * jj - 1, 2) <= Xa + s * per < Fraction(2 * jj + 1, 2) for s in (-1, 0, 1))])
        hits = list(itertools.product(*axis_hits))
        assert len(hits) == 1
        pv = int(key[p]) // nc
        assert int(pv_lev[pv]) == l
        assert tuple(int(v) for v in pv_j[pv]) == hits[0], (p, o[:, p])
        # the quadrant: the corner of the leaf at that vertex, seen from it
        corner = sum(1 << a for a in range(d) if (int(co[L, a]) + 1) % per == hits[0][a] and per > 1
                     or (per == 1 and X[a] - co[L, a] >= Fraction(1, 2)))
        assert int(key[p]) % nc == nc - 1 - corner


# ---------------------------------------------------------------------------
# split re-refinement: ppc criterion on exact fine cells
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("ppc", [8, 40])
def test_retree32_ppc_criterion_on_exact_cells(ppc):
    """The split re-refinement applies the particles-per-cell criterion (refine
    on overrun between dmin and dmax) to the cells that hold the exact rational
    positions (c + o) / 3^l: every leaf holds at most ppc particles or sits on
    dmax, every refined cell from dmin on holds more than ppc, and no leaf lies
    above dmin.  Particles within 2^-20 of a level-dmax face are left out of
    the sample (the FP32 drop rule decides those by rounding)."""
    d, dmin, dmax = 2, 2, 5
    t = oracle.Tree(d, W.random_tree_flags(d, 4, 0.3, 105, min_depth=2))
    rng = np.random.default_rng(ppc)
    x = np.mod(0.5 + 0.08 * rng.standard_normal((d, 5000)), 1.0)
    leaf, o, _ = t.split_from64(x, np.zeros_like(x))
    lev, co = t.leaf_info()
    L = lev[leaf].astype(np.int64)
    sc = 3.0 ** (dmax - L)
    fine_f = (co[leaf].T.astype(np.float64) + o.astype(np.float64)) * sc   # exact in FP64 (o has 24 bits)
    frac = fine_f - np.floor(fine_f)
    keep = np.all((frac > 2 ** -20) & (frac < 1 - 2 ** -20), axis=0)
    leaf, o, fine = leaf[keep], np.ascontiguousarray(o[:, keep]), np.floor(fine_f[:, keep]).astype(np.int64)
    flags = oracle.retree32(t, leaf, o, ppc, dmin, dmax)
    nt = oracle.Tree(d, flags)
    nlev, nco = nt.leaf_info()
    assert nlev.min() >= dmin and nlev.max() <= dmax
    cnt = {}
    for m in range(dmax + 1):
        cm = fine // 3 ** (dmax - m)
        keys, c = np.unique(cm[0] + 3 ** m * cm[1], return_counts=True)
        cnt[m] = dict(zip(keys.tolist(), c.tolist()))
    for l, c in zip(nlev, nco):
        n_in = cnt[int(l)].get(int(c[0] + 3 ** int(l) * c[1]), 0)
        assert n_in <= ppc or l == dmax
    root = LA.parse_tree(d, flags)
    stack = [root]
    while stack:
        c = stack.pop()
        if c.children:
            stack.extend(c.children)
            if c.level >= dmin:
                assert cnt[c.level].get(c.coords[0] + 3 ** c.level * c.coords[1], 0) > ppc


# ---------------------------------------------------------------------------
# leapfrog start: the cold Langmuir oscillation at t = -dt/2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_init_leapfrog_cold_langmuir_half_kick(precision):
    """A cold plasma (v = 0) with density 1 + eps cos(2 pi x) against a unit
    ion background has E(x) = -eps sin(2 pi x) / (2 pi) (Poisson, -V'' = rho);
    with q/m = -1 every particle starts accelerating by a = eps sin(2 pi x0) /
    (2 pi), so the leapfrog start velocity is v_{-1/2} = -a dt / 2.  The
    discrete value (CIC, d-linear elements, 27 x 27 grid) agrees within the
    O((k h)^2) discretisation error; a wrong sign, a missing half or a missing
    kick is off by 100%."""
    eps, dt = 0.01, 0.1
    w = W.langmuir(2, 3, 16, vth=0.0, amp=eps, dt=dt)
    tree = oracle.Tree(2, w.flags)
    prm = oracle.Params(q=w.q, qm=w.qm, ion=w.ion, sweeps=2000, omega=1.0)
    st = (oracle.State64 if precision == "fp64" else oracle.State32)(tree, w.x, w.v, prm)
    x0 = st.x[0].copy() if precision == "fp64" else st.positions()[0]
    st.init_leapfrog(dt)
    a = eps * np.sin(2 * np.pi * x0) / (2 * np.pi)
    vx = np.asarray(st.v[0], np.float64)
    expect = -a * dt / 2
    rel = np.linalg.norm(vx - expect) / np.linalg.norm(expect)
    assert rel < 0.03, rel
    assert np.max(np.abs(np.asarray(st.v[1], np.float64))) < 0.03 * np.abs(expect).max()


# ---------------------------------------------------------------------------
# lift and drop counts of PIDT, tunnellers
# ---------------------------------------------------------------------------

def _dual_cell(level, j):
    """Half-open dual cell of vertex (level, j) on one axis, in units of
    1 / (2 3^18): [(2j - 1) 3^(18 - l), (2j + 1) 3^(18 - l))."""
    s = 3 ** (18 - level)
    return (2 * j - 1) * s, 2 * s


def _contains(outer, inner, P):
    (a, wa), (b, wb) = outer, inner
    return (b - a) % P + wb <= wa


@pytest.mark.parametrize("d,depth,p,seed", [(2, 4, 0.35, 201), (3, 3, 0.3, 202)])
def test_pidt_lifts_against_dual_cell_geometry(d, depth, p, seed):
    """PIDT lifts and drops: zero when the new owner is a vertex of the old
    leaf on its level (hand-over inside the cell), else up to the deepest
    vertex whose dual cell contains both owners' dual cells (found here by
    scanning every vertex of every level, exact integer intervals) and down
    to the new owner."""
    flags = W.random_tree_flags(d, depth, p, seed, min_depth=1)
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 1500, seed, vmax=0.3)
    x2 = np.mod(x + v * 0.5, 1.0)
    old_leaf = t.pit_owner(x)
    k1, k2 = t.keys64(oracle.PIDT, x), t.keys64(oracle.PIDT, x2)
    lifts, drops = t.pidt_lifts(old_leaf, k1, k2)
    lev, co = t.leaf_info()
    pv_lev, pv_j = t.pidt_vertices()
    nc = 1 << d
    P = 2 * 3 ** 18
    expect_l, expect_d = np.zeros(len(k1), np.int64), np.zeros(len(k1), np.int64)
    for i in range(len(k1)):
        a, b = int(k1[i]) // nc, int(k2[i]) // nc
        l1, l2 = int(pv_lev[a]), int(pv_lev[b])
        j1, j2 = [int(c) for c in pv_j[a]], [int(c) for c in pv_j[b]]
        L = int(old_leaf[i])
        ll = int(lev[L])
        corners = {tuple((int(co[L, ax]) + e[ax]) % 3 ** ll for ax in range(d))
                   for e in itertools.product((0, 1), repeat=d)}
        if a == b or (l2 == ll and tuple(j2) in corners):
            continue
        m_found = None
        for m in range(min(l1, l2), -1, -1):
            ok = True
            for ax in range(d):
                c1, c2 = _dual_cell(l1, j1[ax]), _dual_cell(l2, j2[ax])
                if not any(_contains(_dual_cell(m, J), c1, P) and _contains(_dual_cell(m, J), c2, P)
                           for J in range(3 ** m)):
                    ok = False
                    break
            if ok:
                m_found = m
                break
        assert m_found is not None
        expect_l[i], expect_d[i] = l1 - m_found, l2 - m_found
    assert np.array_equal(lifts, expect_l) and np.array_equal(drops, expect_d)
    assert lifts.sum() > 0 and (lifts == 0).sum() > 0


@pytest.mark.parametrize("d,depth,p,seed", [(2, 4, 0.35, 203), (3, 3, 0.3, 204)])
def test_tunnellers_exact_geometry(d, depth, p, seed):
    """A particle tunnels when its new leaf's closed box shares no point with
    its old leaf's (periodic): checked with exact interval arithmetic over the
    three periodic images."""
    flags = W.random_tree_flags(d, depth, p, seed, min_depth=1)
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 2000, seed, vmax=0.2)
    L1, L2 = t.pit_owner(x), t.pit_owner(np.mod(x + v * 0.5, 1.0))
    tun = t.tunnellers(L1, L2)
    lev, co = t.leaf_info()
    for i in range(len(L1)):
        a, b = int(L1[i]), int(L2[i])
        touch = True
        for ax in range(d):
            lo1, hi1 = Fraction(int(co[a, ax]), 3 ** int(lev[a])), Fraction(int(co[a, ax]) + 1, 3 ** int(lev[a]))
            lo2, hi2 = Fraction(int(co[b, ax]), 3 ** int(lev[b])), Fraction(int(co[b, ax]) + 1, 3 ** int(lev[b]))
            touch &= any(lo1 <= hi2 + s and lo2 + s <= hi1 for s in (-1, 0, 1))
        assert bool(tun[i]) == (not touch), i
    assert tun.sum() > 0 and (~tun).sum() > 0


@pytest.mark.parametrize("scheme", [oracle.PIT, oracle.PIDT])
def test_vmax_is_the_subtree_maximum(scheme):
    """raPIDT v_max per node equals, by brute force over the subtree's leaf
    boxes, the largest velocity component of the particles inside it (PIT) or
    inside any dual cell that meets a leaf below it (PIDT: the dual cell of
    vertex (l, j) of a leaf on level l, found by scanning the particles'
    owners)."""
    d = 2
    flags = W.random_tree_flags(d, 4, 0.35, 301, min_depth=1)
    t = oracle.Tree(d, flags)
    x, v = W.random_particles(d, 3000, 301, vmax=1.0)
    leaf = t.pit_owner(x)
    key = t.keys64(oracle.PIDT, x)
    out = t.vmax(scheme, leaf, key, v)
    vabs = np.abs(v).max(axis=0)
    root = LA.parse_tree(d, flags)
    nodes, queue = [], [root]          # level order
    while queue:
        c = queue.pop(0)
        nodes.append(c)
        if c.children:
            queue.extend(c.children)
    assert len(nodes) == len(out)
    pv_lev, pv_j = t.pidt_vertices()
    own_l = pv_lev[key // 4]
    own_j = pv_j[key // 4]
    Q = quantise_np(x)
    for i, c in enumerate(nodes):
        s = 2 * 3 ** (18 - c.level)
        if scheme == oracle.PIT:
            inside = np.all([(Q[a] >= c.coords[a] * s) & (Q[a] < (c.coords[a] + 1) * s) for a in range(d)], axis=0)
        else:
            # particles whose owner vertex is a corner of a leaf inside c
            inside = np.zeros(x.shape[1], bool)
            stack = [c]
            while stack:
                cc = stack.pop()
                if cc.children:
                    stack.extend(cc.children)
                    continue
                per = 3 ** cc.level
                for e in itertools.product((0, 1), repeat=d):
                    j = [(cc.coords[a] + e[a]) % per for a in range(d)]
                    inside |= (own_l == cc.level) & np.all(own_j == np.array(j)[None, :], axis=1)
        expect = vabs[inside].max() if inside.any() else 0.0
        assert out[i] == expect, (i, c.level, c.coords)


# ---------------------------------------------------------------------------
# the particle-handling step of Section 6 (no field, reflecting walls)
# ---------------------------------------------------------------------------

def _triangle(y: Fraction) -> tuple[Fraction, int]:
    """Exact position after reflections at 0 and 1 of the free motion to y,
    and the number of wall hits."""
    k = y // 1                                  # floor
    r = y - k
    hits = int(k) if k >= 0 else -int(k)
    if int(k) % 2 == 0:
        return r, hits
    return 1 - r, hits


def test_move64_reflection_closed_form():
    """A free particle between reflecting walls follows the triangle wave of
    x0 + v t: after every FP64 step the position equals the exact fold of
    the (rounded) free path to within the roundings of that path, and the
    velocity's sign is (-1)^(wall hits)."""
    d = 2
    t = oracle.Tree(d, W.uniform_tree_flags(d, 2))
    x0 = np.array([[0.1, 0.95, 0.5, 0.0], [0.3, 0.02, 0.999, 0.7]])
    v0 = np.array([[0.9, -3.3, 12.25, 0.0], [-0.45, 1.0, 7.0, -2.5]])
    x, v = x0.copy(), v0.copy()
    dt = 0.125
    for step in range(1, 9):
        t.move64(x, v, dt, 1)
        for a in range(d):
            for p in range(x.shape[1]):
                y = Fraction(float(x0[a, p])) + Fraction(float(v0[a, p])) * step * Fraction(dt)
                r, hits = _triangle(y)
                assert abs(float(r) - x[a, p]) <= 1e-14 * step, (a, p, step)
                assert np.sign(v[a, p]) == np.sign(v0[a, p]) * (-1) ** hits or v0[a, p] == 0.0
                assert 0.0 <= x[a, p] < 1.0
    assert np.array_equal(np.abs(v), np.abs(v0))


def test_move64_far_wall_tie_and_periodic_mode():
    d = 2
    t = oracle.Tree(d, W.uniform_tree_flags(d, 1))
    x = np.array([[0.5], [0.25]])
    v = np.array([[0.5], [-0.25]])
    t.move64(x, v, 1.0, 1)          # 0.5 + 0.5 = 1 exactly: the far wall
    assert x[0, 0] == np.nextafter(1.0, 0.0) and v[0, 0] == -0.5
    assert x[1, 0] == 0.0 and v[1, 0] == -0.25   # 0.25 - 0.25 = 0: no reflection
    x = np.array([[0.75], [0.1]])
    v = np.array([[0.5], [-0.3]])
    t.move64(x, v, 1.0, 0)          # periodic: wrap, velocity kept
    assert x[0, 0] == 0.25 and v[0, 0] == 0.5
    assert abs(x[1, 0] - 0.8) < 1e-15 and v[1, 0] == -0.3


@pytest.mark.parametrize("d,flags_fn", TREES)
def test_move32_tracks_move64(d, flags_fn):
    """The split move lands every particle in the leaf that covers the FP64
    move of the same particle (away from faces by 2^-18 of a cell), at the
    same position to FP32 rounding of the cell-unit displacement, with the
    same velocity signs."""
    flags = flags_fn()
    t = oracle.Tree(d, flags)
    w = W.particle_handling(d, 4000, seed=31)
    leaf, o, vf = t.split_from64(w.x, w.v)
    x64, v64 = t.split_to64(leaf, o), vf.astype(np.float64)
    dt = 0.3
    t.move32(leaf, o, vf, dt, 1)
    t.move64(x64, v64, dt, 1)
    xr = t.split_to64(leaf, o)
    assert np.all((o >= 0) & (o < 1))
    assert np.max(np.abs(xr - x64)) < 1e-5
    assert np.array_equal(np.sign(vf), np.sign(v64)) or np.all((np.sign(vf) == np.sign(v64)) | (v64 == 0))
    near = np.any((o < 2 ** -18) | (o > 1 - 2 ** -18), axis=0)
    assert np.all((t.pit_owner(x64) == leaf) | near)
