"""Literal executions of the paper's Algorithm 1 (PIT) and Algorithms 2-3
(PIDT) on a recursive depth-first traversal, in pure Python.

These are pins for the oracle: the oracle computes the owner of a particle
directly from its definition (covering leaf; covering dual cell on the leaf
level), while the code below reaches the assignment the way the paper does,
event by event, with lifts, drops and (PIDT) linked-list hand-overs.  It shares
no code with the oracle.

Geometry is evaluated on the quantised positions (integers Q in
[0, 2*3^18) per axis) so that containment is exact: a cell (l, c) holds
[c*2*3^(18-l), (c+1)*2*3^(18-l)), the dual cell of vertex (l, j) holds
[(2j-1)*3^(18-l), (2j+1)*3^(18-l)) modulo the period.
"""
from __future__ import annotations

import itertools

QSTEPS = 2 * 3 ** 18


def quantise(x: float) -> int:
    y = x - __import__("math").floor(x)
    if y >= 1.0:
        y = 0.0
    q = int(__import__("math").floor(y * float(QSTEPS)))
    return min(max(q, 0), QSTEPS - 1)


class Cell:
    __slots__ = ("level", "coords", "children", "parent")

    def __init__(self, level, coords, parent):
        self.level = level
        self.coords = coords
        self.children = None
        self.parent = parent


def parse_tree(d: int, flags) -> Cell:
    """Level-order flags -> linked cells (children in digit order, x fastest)."""
    root = Cell(0, (0,) * d, None)
    queue = [root]
    qi = 0
    for f in flags:
        cell = queue[qi]
        qi += 1
        if f:
            cell.children = []
            for digit in range(3 ** d):
                off = tuple((digit // 3 ** a) % 3 for a in range(d))
                ch = Cell(cell.level + 1, tuple(3 * c + o for c, o in zip(cell.coords, off)), cell)
                cell.children.append(ch)
                queue.append(ch)
    assert qi == len(queue), "flags do not match the tree"
    return root


def cell_contains(cell: Cell, Q) -> bool:
    s = 2 * 3 ** (18 - cell.level)
    return all(c * s <= q < (c + 1) * s for c, q in zip(cell.coords, Q))


def dual_contains(level: int, j, Q) -> bool:
    s = 3 ** (18 - level)
    for jj, q in zip(j, Q):
        lo = ((2 * jj - 1) * s) % QSTEPS
        off = (q - lo) % QSTEPS
        if not off < 2 * s:
            return False
    return True


# --------------------------------------------------------------------------
# Algorithm 1: particle in tree
# --------------------------------------------------------------------------

def pit_literal(d, flags, Q_old, Q_new, max_traversals=8, counts=None):
    """Particles start in the leaf covering Q_old; the move replaces the
    position by Q_new in the first traversal.  Traversals repeat until no
    particle is lifted or dropped.  Returns {particle: (level, coords)}.
    With a dict `counts`, counts["lifts"][m] and counts["drops"][m] receive
    the lift and drop events of particle m during the traversals (the initial
    placement is not counted)."""
    lifts = [0] * len(Q_old)
    drops = [0] * len(Q_old)
    if counts is not None:
        counts["lifts"] = lifts
        counts["drops"] = drops
    root = parse_tree(d, flags)
    assoc = {id(root): list(range(len(Q_old)))}
    cells = {id(root): root}
    pos = [tuple(q) for q in Q_old]

    # initial sort: place every particle in its leaf by drops alone
    def drop_all(cell):
        mine = assoc.get(id(cell), [])
        if cell.children:
            for m in mine:
                for ch in cell.children:
                    if cell_contains(ch, pos[m]):
                        assoc.setdefault(id(ch), []).append(m)
                        cells[id(ch)] = ch
                        break
            assoc[id(cell)] = []
            for ch in cell.children:
                drop_all(ch)

    drop_all(root)
    state = {"moving": True, "changes": 0}

    def traverse(cell):
        cells[id(cell)] = cell
        mine = assoc.setdefault(id(cell), [])
        # enterCell
        if cell.children:                       # preamble: drop
            for m in list(mine):
                for ch in cell.children:
                    if cell_contains(ch, pos[m]):
                        assoc.setdefault(id(ch), []).append(m)
                        mine.remove(m)
                        state["changes"] += 1
                        drops[m] += 1
                        break
        else:                                   # move
            if state["moving"]:
                for m in mine:
                    pos[m] = tuple(Q_new[m])
        if cell.children:
            for ch in cell.children:
                traverse(ch)
        # leaveCell: lift what the cell no longer covers
        if cell.parent is not None:
            for m in list(mine):
                if not cell_contains(cell, pos[m]):
                    assoc.setdefault(id(cell.parent), []).append(m)
                    mine.remove(m)
                    state["changes"] += 1
                    lifts[m] += 1

    for t in range(max_traversals):
        state["changes"] = 0
        traverse(root)
        state["moving"] = False
        if t > 0 and state["changes"] == 0:
            break
    out = {}
    for cid, lst in assoc.items():
        c = cells[cid]
        for m in lst:
            assert c.children is None, "particle left on a refined cell"
            out[m] = (c.level, c.coords)
    return out


# --------------------------------------------------------------------------
# Algorithms 2-3: particle in dual tree
# --------------------------------------------------------------------------

def pidt_literal(d, flags, Q_old, Q_new, max_traversals=8):
    """Particles start at the owner vertex of Q_old; the move replaces the
    position by Q_new in the first traversal; traversals repeat until nothing
    changes.  Returns {particle: (level, j)}.

    Event order of a depth-first traversal: touchVertexFirstTime(v) right
    before the first enterCell of a cell adjacent to v on v's level,
    touchVertexLastTime(v) right after the last leaveCell of such a cell.

    Readings (see the design notes): the preamble of touchVertexFirstTime
    resets `moved` for every vertex (with the printed guard `v refined` the
    particles of leaf-level vertices would never move again); the lift of
    touchVertexLastTime also applies to particles that left every cell adjacent
    to v on v's level (hanging vertices, "PIDT has to lift them there").
    """
    root = parse_tree(d, flags)
    levels = {}
    allcells = []

    def collect(c):
        allcells.append(c)
        levels.setdefault(c.level, set()).add(c.coords)
        if c.children:
            for ch in c.children:
                collect(ch)

    collect(root)
    corners = list(itertools.product((0, 1), repeat=d))

    def vertices_of(cell):
        per = 3 ** cell.level
        return [(cell.level, tuple((c + e) % per for c, e in zip(cell.coords, es))) for es in corners]

    adjacent = {}
    for c in allcells:
        for v in vertices_of(c):
            adjacent.setdefault(v, []).append(c)

    pos = [tuple(q) for q in Q_old]
    n = len(pos)

    def cell_at(level, Q):
        s = 2 * 3 ** (18 - level)
        co = tuple(q // s for q in Q)
        return co if co in levels.get(level, ()) else None

    def leaf_level(Q):
        node = root
        while node.children:
            for ch in node.children:
                if cell_contains(ch, Q):
                    node = ch
                    break
        return node.level

    def nearest_vertex(level, Q):
        s = 3 ** (18 - level)
        per = 3 ** level
        return (level, tuple(((q + s) // (2 * s)) % per for q in Q))

    assoc = {}
    for m in range(n):  # initial state: drop through refined cells from the root vertex
        assoc.setdefault(nearest_vertex(leaf_level(pos[m]), pos[m]), []).append(m)
    moved = [False] * n
    st = {"moving": True, "changes": 0}

    def parent_vertex(v):
        level, j = v
        per = 3 ** (level - 1)
        return (level - 1, tuple(((jj + 1) // 3) % per for jj in j))

    def child_vertex_for(cell, Q):
        return nearest_vertex(cell.level + 1, Q)

    def covered_by_adjacent(v, Q):
        return any(cell_contains(c, Q) for c in adjacent[v])

    touched_first = set()
    remaining = {}

    def touch_first(v):
        for m in assoc.get(v, []):
            moved[m] = False

    def touch_last(v):
        if v[0] == 0:
            return
        lst = assoc.get(v, [])
        for m in list(lst):
            if moved[m] and (not dual_contains(v[0], v[1], pos[m]) or not covered_by_adjacent(v, pos[m])):
                lst.remove(m)
                assoc.setdefault(parent_vertex(v), []).append(m)
                st["changes"] += 1

    def enter(cell):
        for v in vertices_of(cell):
            if v not in touched_first:
                touched_first.add(v)
                touch_first(v)
        if cell.children:
            for v in vertices_of(cell):
                lst = assoc.get(v, [])
                for m in list(lst):
                    if not moved[m] and cell_contains(cell, pos[m]):
                        lst.remove(m)
                        assoc.setdefault(child_vertex_for(cell, pos[m]), []).append(m)
                        st["changes"] += 1
        else:
            for v in vertices_of(cell):
                for m in assoc.get(v, []):
                    if not moved[m] and cell_contains(cell, pos[m]):
                        if st["moving"]:
                            pos[m] = tuple(Q_new[m])
                        moved[m] = True

    def leave(cell):
        vs = vertices_of(cell)
        for v in vs:
            lst = assoc.get(v, [])
            for m in list(lst):
                if not moved[m]:
                    continue
                for v2 in vs:
                    if v2 != v and dual_contains(v2[0], v2[1], pos[m]):
                        lst.remove(m)
                        assoc.setdefault(v2, []).append(m)
                        st["changes"] += 1
                        break
        for v in vs:
            remaining[v] -= 1
            if remaining[v] == 0:
                touch_last(v)

    def traverse(cell):
        enter(cell)
        if cell.children:
            for ch in cell.children:
                traverse(ch)
        leave(cell)

    for t in range(max_traversals):
        touched_first.clear()
        remaining.clear()
        for v, cs in adjacent.items():
            remaining[v] = len(cs)
        st["changes"] = 0
        traverse(root)
        st["moving"] = False
        if t > 0 and st["changes"] == 0:
            break
    out = {}
    for v, lst in assoc.items():
        for m in lst:
            out[m] = v
    return out
