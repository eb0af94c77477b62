"""Lifts and drops as rewrite rules on a linked spacetree, applied until none
fires, in pure Python: pins for the oracle's particle owners and its PIT lift
and drop counts that share no code with the oracle.

Particles are stored on the tree (Section 4.2): PIT associates a particle
with a cell, PIDT with a vertex, whose dual cell (Section 4.1) is the cube of
the vertex's level centred on it.  A lift hands a particle to the next coarser
level, a drop to the next finer one (Sections 5.1 and 5.2).  The rules fire
in any order; where none applies, every particle sits where Theorems 1 and 2
put it, which the oracle computes directly from the positions.

PIT rules (a particle on cell c):
  lift - c does not contain the particle: it goes to c's parent;
  drop - c is refined and contains the particle: it goes to the child of c
         that contains it.
PIDT rules (a particle on vertex (l, j)):
  lift - the dual cell of (l, j) does not hold the particle, or no cell of
         the tree on level l contains it: it goes to the dual parent
         (l - 1, (j + 1) div 3), the vertex whose dual cell contains that of
         (l, j) (k = 3: dual grid consistency, Section 4.1);
  drop - the level-l cell of the tree that contains the particle is refined:
         it goes to the level-(l + 1) vertex whose dual cell holds it.

A particle's lift and drop counts are the number of times each rule moved
it.  Geometry is evaluated on quantised positions (integers Q in
[0, 2*3^18) per axis) so that containment is exact: the cell (l, c) holds
[c*2*3^(18-l), (c+1)*2*3^(18-l)) per axis, the dual cell of vertex (l, j)
holds [(2j-1)*3^(18-l), (2j+1)*3^(18-l)) modulo the period.
"""
from __future__ import annotations

import math

QSTEPS = 2 * 3 ** 18


def quantise(x: float) -> int:
    y = x - math.floor(x)
    if y >= 1.0:
        y = 0.0
    q = int(math.floor(y * float(QSTEPS)))
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


def _pit_settle(cell: Cell, Q, counts):
    """Applies the PIT rules to one particle until neither fires."""
    while True:
        if cell.parent is not None and not cell_contains(cell, Q):
            cell = cell.parent
            counts[0] += 1
            continue
        if cell.children:
            nxt = [ch for ch in cell.children if cell_contains(ch, Q)]
            assert len(nxt) == 1, "children must tile their parent"
            cell = nxt[0]
            counts[1] += 1
            continue
        return cell


def pit_by_rules(d, flags, Q_old, Q_new, counts=None):
    """Every particle starts on the root cell at Q_old and settles (its
    initial placement, not counted); its position becomes Q_new and it
    settles again.  Returns {particle: (level, coords)}; with a dict
    `counts`, counts["lifts"][m] and counts["drops"][m] receive the rule
    firings of particle m after the move."""
    root = parse_tree(d, flags)
    lifts, drops = [0] * len(Q_old), [0] * len(Q_old)
    out = {}
    for m, (q0, q1) in enumerate(zip(Q_old, Q_new)):
        cell = _pit_settle(root, tuple(q0), [0, 0])
        c = [0, 0]
        cell = _pit_settle(cell, tuple(q1), c)
        lifts[m], drops[m] = c
        out[m] = (cell.level, cell.coords)
    if counts is not None:
        counts["lifts"] = lifts
        counts["drops"] = drops
    return out


def pidt_by_rules(d, flags, Q_old, Q_new):
    """Every particle starts on the root vertex (0, 0...) at Q_old and
    settles; its position becomes Q_new and it settles again.  Returns
    {particle: (level, j)}."""
    root = parse_tree(d, flags)
    cells = {}

    def collect(c):
        cells[(c.level, c.coords)] = c
        if c.children:
            for ch in c.children:
                collect(ch)

    collect(root)

    def cell_at(level, Q):
        s = 2 * 3 ** (18 - level)
        return cells.get((level, tuple(q // s for q in Q)))

    def settle(v, Q):
        while True:
            level, j = v
            here = cell_at(level, Q)
            if level > 0 and (not dual_contains(level, j, Q) or here is None):
                per = 3 ** (level - 1)
                v = (level - 1, tuple(((jj + 1) // 3) % per for jj in j))
                continue
            if here is not None and here.children:
                s = 3 ** (18 - level - 1)
                per = 3 ** (level + 1)
                nv = (level + 1, tuple(((q + s) // (2 * s)) % per for q in Q))
                assert dual_contains(nv[0], nv[1], Q)
                v = nv
                continue
            return v

    out = {}
    for m, (q0, q1) in enumerate(zip(Q_old, Q_new)):
        v = settle((0, (0,) * d), tuple(q0))
        out[m] = settle(v, tuple(q1))
    return out
