"""CPU oracle for the PIT / PIDT particle step (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library product never touches it.

The arithmetic lives in ``oracle.c`` (plain serial C, FP64 plus an FP32 mirror
of the split-precision mode, compiled with floating-point contraction off).
This module compiles it on first use and composes its phases into one time
step in the order of the paper's PIC cycle (Section 3): deposit
rho = sum_i R(x_i), solve L(V) = rho, E = -grad V, gather E_i = R^T(x_i) E,
push, then re-bin every particle into the leaf (PIT, Algorithm 1) or dual cell
(PIDT, Algorithms 2-3) that covers it.

Parity pins (tests/test_oracle_*.py) check this oracle against brute force,
the lift and drop rules applied to a fixed point, closed forms and
conservation laws.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PIT, PIDT = 0, 1


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (no fast-math, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-fvisibility=hidden", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, f64, f32 = C.c_int64, C.c_int, C.c_double, C.c_float
        sig = {
            "or_tree_new": (P, [i32, i64, P, C.POINTER(C.c_int)]),
            "or_tree_free": (None, [P]),
            "or_n_leaves": (i64, [P]),
            "or_depth": (i32, [P]),
            "or_leaf_info": (None, [P, P, P]),
            "or_pit_owner": (None, [P, i64, P, P]),
            "or_pidt_owner": (None, [P, i64, P, P, P]),
            "or_grid_build": (i32, [P]),
            "or_n_vertices": (i64, [P]),
            "or_vertex_pos": (None, [P, P]),
            "or_vertex_aux": (None, [P, P, P]),
            "or_corner_expansion": (i64, [P, P, P, P]),
            "or_pidt_build": (i32, [P]),
            "or_n_pidt_vertices": (i64, [P]),
            "or_pidt_vertex_info": (None, [P, P, P]),
            "or_n_keys": (i64, [P, i32]),
            "or_keys64": (None, [P, i32, i64, P, P]),
            "or_stable_bucket": (None, [i64, P, i64, P, P]),
            "or_deposit64": (f64, [P, i32, i64, P, f64, f64, P]),
            "or_apply64": (None, [P, P, P]),
            "or_solve64": (f64, [P, P, P, i32, f64]),
            "or_efield64": (None, [P, P, P]),
            "or_push64": (None, [P, i64, P, P, P, f64, f64]),
            "or_gather64": (None, [P, i64, P, P, P]),
            "or_move64": (None, [P, i64, P, P, f64, i32]),
            "or_move32": (None, [P, i64, P, P, P, f64, i32]),
            "or_split_from64": (None, [P, i64, P, P, P, P, P]),
            "or_split_to64": (None, [P, i64, P, P, P]),
            "or_keys32": (None, [P, i32, i64, P, P, P]),
            "or_deposit32": (f64, [P, i32, i64, P, P, f32, f32, P]),
            "or_solve32": (f64, [P, P, P, i32, f32]),
            "or_efield32": (None, [P, P, P]),
            "or_push32": (None, [P, i64, P, P, P, P, f64, f64]),
            "or_gather32": (None, [P, i64, P, P, P, P]),
            "or_retree64": (i64, [i32, i64, P, i64, i32, i32]),
            "or_retree32": (i64, [P, i64, P, P, i64, i32, i32]),
            "or_retree_fetch": (None, [P]),
            "or_rebin32": (None, [P, P, i64, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


class Tree:
    """A k = 3 spacetree built from level-order refinement flags."""

    def __init__(self, d: int, flags: np.ndarray):
        lib = _load()
        self.d = d
        self.flags = _c(flags, np.uint8)
        err = C.c_int(0)
        h = lib.or_tree_new(d, len(self.flags), _p(self.flags), C.byref(err))
        if not h:
            raise ValueError(f"malformed tree flags (oracle error {err.value})")
        self._h = C.c_void_p(h)
        self._lib = lib

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self._lib.or_tree_free(h)
            self._h = None

    @property
    def n_leaves(self) -> int:
        return int(self._lib.or_n_leaves(self._h))

    @property
    def depth(self) -> int:
        return int(self._lib.or_depth(self._h))

    def leaf_info(self):
        """(level[n_leaves], coords[n_leaves, d]) in depth-first leaf order."""
        n = self.n_leaves
        lev = np.zeros(n, np.int32)
        co = np.zeros((n, self.d), np.int64)
        self._lib.or_leaf_info(self._h, _p(lev), _p(co))
        return lev, co

    def pit_lifts(self, old_leaf: np.ndarray, new_leaf: np.ndarray):
        """Lifts and drops of Algorithm 1 for particles that go from leaf
        old_leaf[i] to leaf new_leaf[i]: a particle is lifted out of every cell
        from its old leaf up to the deepest ancestor that also contains its new
        leaf, then dropped cell by cell down to the new leaf; lifting (or
        dropping) n levels counts as n lifts (drops), as the paper counts them
        (Section 6).  Returns (lifts, drops), int64 per particle."""
        lev, co = self.leaf_info()
        old_leaf = np.asarray(old_leaf, np.int64)
        new_leaf = np.asarray(new_leaf, np.int64)
        l1, l2 = lev[old_leaf].astype(np.int64), lev[new_leaf].astype(np.int64)
        c1, c2 = co[old_leaf], co[new_leaf]
        low = np.minimum(l1, l2)
        common = np.zeros(len(old_leaf), np.int64)  # level of the deepest common ancestor
        for m in range(1, int(low.max(initial=0)) + 1):
            on = low >= m
            a1 = c1 // (3 ** np.where(on, l1 - m, 0))[:, None]
            a2 = c2 // (3 ** np.where(on, l2 - m, 0))[:, None]
            same = on & np.all(a1 == a2, axis=1)
            common = np.where(same, m, common)
        return l1 - common, l2 - common

    def pidt_lifts(self, old_leaf, old_key, new_key):
        """Lifts and drops of a PIDT particle whose owner went from the vertex
        of old_key to the vertex of new_key (key = vertex 2^d + quadrant) while
        its leaf before the move was old_leaf.  Reading of Algorithms 2-3 as a
        count: a particle that ends at a vertex of its old leaf on that leaf's
        level is handed over between the cell's vertices (no lift, no drop);
        any other particle is lifted from its old vertex to the deepest
        vertex of the dual tree whose dual cell holds both owners' dual cells
        and dropped from there to the new owner -- the dual parent of vertex
        (l, j) being the vertex (l - 1, (j + 1) div 3) whose dual cell contains
        its dual cell (k = 3).  Returns (lifts, drops), int64 per particle."""
        d = self.d
        nc = 1 << d
        lev, co = self.leaf_info()
        pv_lev, pv_j = self.pidt_vertices()
        old_leaf = np.asarray(old_leaf, np.int64)
        k1 = np.asarray(old_key, np.int64) // nc
        k2 = np.asarray(new_key, np.int64) // nc
        l1, l2 = pv_lev[k1].astype(np.int64), pv_lev[k2].astype(np.int64)
        j1, j2 = pv_j[k1].astype(np.int64), pv_j[k2].astype(np.int64)
        ll, cl = lev[old_leaf].astype(np.int64), co[old_leaf]
        per = 3 ** ll
        rel = np.mod(j2 - cl, per[:, None])
        handed = (l2 == ll) & np.all(rel <= 1, axis=1)
        m = np.minimum(l1, l2)

        def up(j, lfrom, lto):
            j = j.copy()
            lcur = lfrom.copy()
            while np.any(lcur > lto):
                go = lcur > lto
                j[go] = np.mod((j[go] + 1) // 3, (3 ** (lcur[go] - 1))[:, None])
                lcur[go] -= 1
            return j

        a1, a2 = up(j1, l1, m), up(j2, l2, m)
        while True:
            differ = (m > 0) & np.any(a1 != a2, axis=1)
            if not np.any(differ):
                break
            a1[differ] = np.mod((a1[differ] + 1) // 3, (3 ** (m[differ] - 1))[:, None])
            a2[differ] = np.mod((a2[differ] + 1) // 3, (3 ** (m[differ] - 1))[:, None])
            m = np.where(differ, m - 1, m)
        same = k1 == k2
        zero = handed | same
        return np.where(zero, 0, l1 - m), np.where(zero, 0, l2 - m)

    def tunnellers(self, old_leaf, new_leaf):
        """True for a particle whose new leaf does not touch its old leaf (the
        closed boxes, periodic, share no point): it moved two cells or more,
        counted on the finer of the two levels."""
        lev, co = self.leaf_info()
        old_leaf = np.asarray(old_leaf, np.int64)
        new_leaf = np.asarray(new_leaf, np.int64)
        l1, l2 = lev[old_leaf].astype(np.int64), lev[new_leaf].astype(np.int64)
        lm = np.maximum(l1, l2)
        s1, s2 = (3 ** (lm - l1))[:, None], (3 ** (lm - l2))[:, None]
        P = (3 ** lm)[:, None]
        lo1, lo2 = co[old_leaf] * s1, co[new_leaf] * s2
        touch = (np.mod(lo2 - lo1, P) <= s1) | (np.mod(lo1 - lo2, P) <= s2)
        return ~np.all(touch, axis=1)

    def vmax(self, scheme: int, leaf, key, v) -> np.ndarray:
        """The raPIDT tree attribute v_max (Section 5.4) per tree node in the
        level order of the refinement flags: on a leaf the largest velocity
        component magnitude of its particles (PIT) or of the particles of its
        2^d vertices, every dual cell intersecting it (PIDT); on a refined
        cell the largest of its children's values (the v_max equation)."""
        d = self.d
        nc, nch = 1 << d, 3 ** d
        v = np.abs(np.asarray(v, np.float64)).max(axis=0)
        lev, co = self.leaf_info()
        leaf_v = np.zeros(self.n_leaves)
        if scheme == PIT:
            np.maximum.at(leaf_v, np.asarray(leaf, np.int64), v)
        else:
            pv_lev, pv_j = self.pidt_vertices()
            vert_v = np.zeros(len(pv_lev))
            np.maximum.at(vert_v, np.asarray(key, np.int64) // nc, v)
            index = {(int(l), tuple(int(c) for c in j)): i for i, (l, j) in enumerate(zip(pv_lev, pv_j))}
            for L in range(self.n_leaves):
                per = 3 ** int(lev[L])
                for e in range(nc):
                    j = tuple((int(co[L, a]) + ((e >> a) & 1)) % per for a in range(d))
                    leaf_v[L] = max(leaf_v[L], vert_v[index[(int(lev[L]), j)]])
        # level-order nodes: children of the k-th refined node are 1 + nch k ...
        flags = self.flags
        n_nodes = len(flags)
        child0 = np.full(n_nodes, -1, np.int64)
        refined = np.flatnonzero(flags)
        child0[refined] = 1 + nch * np.arange(len(refined))
        # depth-first leaf numbering (children in digit order)
        leaf_of_node = np.full(n_nodes, -1, np.int64)
        stack, next_leaf = [0], 0
        while stack:
            i = stack.pop()
            if child0[i] < 0:
                leaf_of_node[i] = next_leaf
                next_leaf += 1
            else:
                stack.extend(range(child0[i] + nch - 1, child0[i] - 1, -1))
        out = np.zeros(n_nodes)
        for i in range(n_nodes - 1, -1, -1):  # children follow their parents in level order
            out[i] = leaf_v[leaf_of_node[i]] if child0[i] < 0 else out[child0[i]:child0[i] + nch].max()
        return out

    # ---- keys -----------------------------------------------------------
    def pit_owner(self, x: np.ndarray) -> np.ndarray:
        x = _c(x, np.float64)
        n = x.shape[1]
        out = np.zeros(n, np.int32)
        self._lib.or_pit_owner(self._h, n, _p(x), _p(out))
        return out

    def pidt_owner(self, x: np.ndarray):
        """(level[n], j[d, n]) of the owner vertex of every particle."""
        x = _c(x, np.float64)
        n = x.shape[1]
        lev = np.zeros(n, np.int32)
        j = np.zeros((self.d, n), np.int64)
        self._lib.or_pidt_owner(self._h, n, _p(x), _p(lev), _p(j))
        return lev, j

    def n_keys(self, scheme: int) -> int:
        return int(self._lib.or_n_keys(self._h, scheme))

    def keys64(self, scheme: int, x: np.ndarray) -> np.ndarray:
        x = _c(x, np.float64)
        out = np.zeros(x.shape[1], np.int64)
        self._lib.or_keys64(self._h, scheme, x.shape[1], _p(x), _p(out))
        return out

    def keys32(self, scheme: int, leaf: np.ndarray, o: np.ndarray) -> np.ndarray:
        leaf = _c(leaf, np.int32)
        o = _c(o, np.float32)
        out = np.zeros(len(leaf), np.int64)
        self._lib.or_keys32(self._h, scheme, len(leaf), _p(leaf), _p(o), _p(out))
        return out

    # ---- grid -----------------------------------------------------------
    @property
    def n_vertices(self) -> int:
        n = int(self._lib.or_n_vertices(self._h))
        if n < 0:
            raise ValueError("grid too deep for the oracle (depth > 12)")
        return n

    def vertex_pos(self) -> np.ndarray:
        """Positions of the non-hanging vertices, units 3^-depth, shape (d, nv)."""
        nv = self.n_vertices
        pos = np.zeros((self.d, nv), np.int64)
        self._lib.or_vertex_pos(self._h, _p(pos))
        return pos

    def vertex_aux(self):
        nv = self.n_vertices
        ion = np.zeros(nv)
        diag = np.zeros(nv)
        self._lib.or_vertex_aux(self._h, _p(ion), _p(diag))
        return ion, diag

    def corner_expansion(self):
        """CSR (ptr, vid, w) of every leaf corner onto non-hanging vertices."""
        nnz = int(self._lib.or_corner_expansion(self._h, None, None, None))
        nlc = self.n_leaves * (1 << self.d)
        ptr = np.zeros(nlc + 1, np.int64)
        vid = np.zeros(nnz, np.int32)
        w = np.zeros(nnz)
        self._lib.or_corner_expansion(self._h, _p(ptr), _p(vid), _p(w))
        return ptr, vid, w

    def pidt_vertices(self):
        nv = int(self._lib.or_n_pidt_vertices(self._h))
        lev = np.zeros(nv, np.int32)
        j = np.zeros((nv, self.d), np.int64)
        self._lib.or_pidt_vertex_info(self._h, _p(lev), _p(j))
        return lev, j

    # ---- FP64 phases ----------------------------------------------------
    def deposit64(self, scheme, x, q, ion):
        x = _c(x, np.float64)
        Q = np.zeros(self.n_vertices)
        tot = self._lib.or_deposit64(self._h, scheme, x.shape[1], _p(x), q, ion, _p(Q))
        return Q, float(tot)

    def apply64(self, V):
        V = _c(V, np.float64)
        y = np.zeros_like(V)
        self._lib.or_apply64(self._h, _p(V), _p(y))
        return y

    def solve64(self, Q, V, sweeps, omega):
        """In-place damped Jacobi on V; returns the residual norm."""
        Q = _c(Q, np.float64)
        assert V.dtype == np.float64 and V.flags.c_contiguous
        return float(self._lib.or_solve64(self._h, _p(Q), _p(V), sweeps, omega))

    def efield64(self, V):
        V = _c(V, np.float64)
        E = np.zeros((self.d, self.n_vertices))
        self._lib.or_efield64(self._h, _p(V), _p(E))
        return E

    def gather64(self, x, Ev):
        x = _c(x, np.float64)
        Ev = _c(Ev, np.float64)
        Ep = np.zeros_like(x)
        self._lib.or_gather64(self._h, x.shape[1], _p(x), _p(Ev), _p(Ep))
        return Ep

    def push64(self, x, v, Ev, qm, dt):
        """In place: gather + leapfrog kick/drift + wrap."""
        assert x.dtype == np.float64 and x.flags.c_contiguous and v.flags.c_contiguous
        Ev = _c(Ev, np.float64)
        self._lib.or_push64(self._h, x.shape[1], _p(x), _p(v), _p(Ev), qm, dt)

    # ---- FP32 split mirror ---------------------------------------------
    def split_from64(self, x, v):
        x = _c(x, np.float64)
        v = _c(v, np.float64)
        n = x.shape[1]
        leaf = np.zeros(n, np.int32)
        o = np.zeros((self.d, n), np.float32)
        vf = np.zeros((self.d, n), np.float32)
        self._lib.or_split_from64(self._h, n, _p(x), _p(v), _p(leaf), _p(o), _p(vf))
        return leaf, o, vf

    def split_to64(self, leaf, o):
        leaf = _c(leaf, np.int32)
        o = _c(o, np.float32)
        x = np.zeros((self.d, len(leaf)))
        self._lib.or_split_to64(self._h, len(leaf), _p(leaf), _p(o), _p(x))
        return x

    def deposit32(self, scheme, leaf, o, q, ion):
        leaf = _c(leaf, np.int32)
        o = _c(o, np.float32)
        Q = np.zeros(self.n_vertices, np.float32)
        tot = self._lib.or_deposit32(self._h, scheme, len(leaf), _p(leaf), _p(o), q, ion, _p(Q))
        return Q, float(tot)

    def solve32(self, Q, V, sweeps, omega):
        Q = _c(Q, np.float32)
        assert V.dtype == np.float32 and V.flags.c_contiguous
        return float(self._lib.or_solve32(self._h, _p(Q), _p(V), sweeps, omega))

    def efield32(self, V):
        V = _c(V, np.float32)
        E = np.zeros((self.d, self.n_vertices), np.float32)
        self._lib.or_efield32(self._h, _p(V), _p(E))
        return E

    def gather32(self, leaf, o, Ev):
        leaf = _c(leaf, np.int32)
        o = _c(o, np.float32)
        Ev = _c(Ev, np.float32)
        Ep = np.zeros((self.d, len(leaf)), np.float32)
        self._lib.or_gather32(self._h, len(leaf), _p(leaf), _p(o), _p(Ev), _p(Ep))
        return Ep

    def push32(self, leaf, o, v, Ev, qm, dt):
        """In place: FP32 gather + kick + drift in cell units + integer re-location."""
        assert leaf.dtype == np.int32 and o.dtype == np.float32 and v.dtype == np.float32
        Ev = _c(Ev, np.float32)
        self._lib.or_push32(self._h, len(leaf), _p(leaf), _p(o), _p(v), _p(Ev), qm, dt)

    def move64(self, x, v, dt, reflect):
        """In place: the particle-handling move of Section 6 (no field),
        periodic (reflect = 0) or reflecting walls (reflect = 1)."""
        assert x.dtype == np.float64 and x.flags.c_contiguous and v.flags.c_contiguous
        self._lib.or_move64(self._h, x.shape[1], _p(x), _p(v), dt, int(reflect))

    def move32(self, leaf, o, v, dt, reflect):
        """In place: the same move in the split representation."""
        assert leaf.dtype == np.int32 and o.dtype == np.float32 and v.dtype == np.float32
        self._lib.or_move32(self._h, len(leaf), _p(leaf), _p(o), _p(v), dt, int(reflect))

    def rebin32_into(self, new_tree: "Tree", leaf, o):
        """In place: same split positions, re-located in ``new_tree``."""
        self._lib.or_rebin32(self._h, new_tree._h, len(leaf), _p(leaf), _p(o))


def stable_bucket(key: np.ndarray, n_keys: int):
    """(start[n_keys+1], perm[n]): stable counting sort by key."""
    key = _c(key, np.int64)
    lib = _load()
    start = np.zeros(n_keys + 1, np.int64)
    perm = np.zeros(len(key), np.int64)
    lib.or_stable_bucket(len(key), _p(key), n_keys, _p(start), _p(perm))
    return start, perm


def _canonical_bucket(key, old_key, n_keys):
    """Counting sort by (key, moved, storage index); returns (start over keys,
    perm)."""
    moved = np.ones(len(key), np.int64) if old_key is None else (key != old_key).astype(np.int64)
    start2, perm = stable_bucket(2 * key + moved, 2 * n_keys)
    return start2[::2].copy(), perm


def retree64(d, x, ppc, dmin, dmax) -> np.ndarray:
    lib = _load()
    x = _c(x, np.float64)
    nf = lib.or_retree64(d, x.shape[1], _p(x), ppc, dmin, dmax)
    out = np.zeros(nf, np.uint8)
    lib.or_retree_fetch(_p(out))
    return out


def retree32(tree: Tree, leaf, o, ppc, dmin, dmax) -> np.ndarray:
    lib = _load()
    leaf = _c(leaf, np.int32)
    o = _c(o, np.float32)
    nf = lib.or_retree32(tree._h, len(leaf), _p(leaf), _p(o), ppc, dmin, dmax)
    out = np.zeros(nf, np.uint8)
    lib.or_retree_fetch(_p(out))
    return out


# --------------------------------------------------------------------------
# Composed time step
# --------------------------------------------------------------------------

@dataclass
class Params:
    scheme: int = PIT
    q: float = -1.0
    qm: float = -1.0
    ion: float = 1.0
    sweeps: int = 100
    omega: float = 0.8


class State64:
    """FP64 particles in storage order (bucket-sorted), plus warm-start V."""

    def __init__(self, tree: Tree, x, v, params: Params, ids=None):
        self.tree = tree
        self.p = params
        x = _c(x, np.float64)
        y = x - np.floor(x)                      # periodic wrap into [0, 1)
        self.x = np.where(y >= 1.0, 0.0, y)
        self.v = _c(v, np.float64).copy()
        n = self.x.shape[1]
        self.ids = np.arange(n, dtype=np.int64) if ids is None else _c(ids, np.int64).copy()
        self.V = np.zeros(tree.n_vertices)
        self.start = None
        self.rebin()

    def rebin(self):
        """Stable re-bin: by (key, moved, storage index), i.e. the particles
        that stay keep their order at the head of their bucket and the movers
        follow in storage order.  At creation every particle counts as moved."""
        key = self.tree.keys64(self.p.scheme, self.x)
        start, perm = _canonical_bucket(key, getattr(self, "key", None), self.tree.n_keys(self.p.scheme))
        self.x = np.ascontiguousarray(self.x[:, perm])
        self.v = np.ascontiguousarray(self.v[:, perm])
        self.ids = self.ids[perm]
        self.key = key[perm]
        self.start = start

    def field(self):
        """Deposit, solve and vertex field for the current positions."""
        Q, tot = self.tree.deposit64(self.p.scheme, self.x, self.p.q, self.p.ion)
        res = self.tree.solve64(Q, self.V, self.p.sweeps, self.p.omega)
        E = self.tree.efield64(self.V)
        return Q, tot, res, E

    def init_leapfrog(self, dt):
        """v_{-1/2} = v_0 - (q/m) E(x_0) dt / 2 (gather at the start positions)."""
        Q, tot, res, E = self.field()
        Ep = self.tree.gather64(self.x, E)
        self.v = self.v - (self.p.qm * (0.5 * dt)) * Ep
        return Q

    def move(self, dt, reflect):
        """The particle-handling step of Section 6: move (no field) and re-bin."""
        self.tree.move64(self.x, self.v, dt, reflect)
        self.rebin()

    def step(self, dt):
        """One PIC step: deposit, solve, field, gather + push, re-bin.
        Returns (Q, total charge, residual, vertex field) of x_n."""
        Q, tot, res, E = self.field()
        self.tree.push64(self.x, self.v, E, self.p.qm, dt)
        self.rebin()
        return Q, tot, res, E


class State32:
    """FP32 split-precision particles in storage order."""

    def __init__(self, tree: Tree, x, v, params: Params, ids=None):
        self.tree = tree
        self.p = params
        self.leaf, self.o, self.v = tree.split_from64(x, v)
        n = len(self.leaf)
        self.ids = np.arange(n, dtype=np.int64) if ids is None else _c(ids, np.int64).copy()
        self.V = np.zeros(tree.n_vertices, np.float32)
        self.rebin()

    def rebin(self):
        key = self.tree.keys32(self.p.scheme, self.leaf, self.o)
        start, perm = _canonical_bucket(key, getattr(self, "key", None), self.tree.n_keys(self.p.scheme))
        self.leaf = np.ascontiguousarray(self.leaf[perm])
        self.o = np.ascontiguousarray(self.o[:, perm])
        self.v = np.ascontiguousarray(self.v[:, perm])
        self.ids = self.ids[perm]
        self.key = key[perm]
        self.start = start

    def field(self):
        Q, tot = self.tree.deposit32(self.p.scheme, self.leaf, self.o, np.float32(self.p.q),
                                     np.float32(self.p.ion))
        res = self.tree.solve32(Q, self.V, self.p.sweeps, np.float32(self.p.omega))
        E = self.tree.efield32(self.V)
        return Q, tot, res, E

    def init_leapfrog(self, dt):
        Q, tot, res, E = self.field()
        Ep = self.tree.gather32(self.leaf, self.o, E)
        half = np.float32(self.p.qm * (0.5 * dt))
        self.v = (self.v - half * Ep).astype(np.float32)
        return Q

    def move(self, dt, reflect):
        self.tree.move32(self.leaf, self.o, self.v, dt, reflect)
        self.rebin()

    def step(self, dt):
        Q, tot, res, E = self.field()
        self.tree.push32(self.leaf, self.o, self.v, E, self.p.qm, dt)
        self.rebin()
        return Q, tot, res, E

    def positions(self):
        return self.tree.split_to64(self.leaf, self.o)
