"""The partitioned single plasma (paper_1508_02435_gb300/partition.py) on
gloo CPU ranks, world size 2 and 4, with the CPU oracle doing each rank's
local work, against the single-rank oracle:

* every rank ends with exactly the particles whose new leaf it owns, with
  the single-rank keys, positions and velocities bit for bit, in the
  single-rank canonical order (PIT: each rank holds a contiguous slice of the
  single-rank array) or, for PIDT, in the single-rank order restricted to the
  rank's particles (bucket by bucket the same sets; the rank-local order
  breaks ties between source ranks by rank);
* the deposit halo sum gives every rank the single-rank vertex charges at
  its replicated vertices (within 1e-13, the summation order differs);
* the FP64 charge total is the same on every rank and equals the single-rank
  total;
* raPIDT: with every rank's v_max dt below the finest leaf width the
  migration runs between neighbouring ranks only (no global all-to-all);
  with tunnelling particles it takes the all-to-all.

Failure paths are made on the host (no GPU): a rank that promised
neighbour-only migration but holds a farther mover raises before anything is
sent.
"""
from __future__ import annotations

import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1508_02435_gb300 import partition as PT  # noqa: E402
from paper_1508_02435_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _setup(d, flags_kind, n, vmax, seed):
    if flags_kind == "uniform":
        flags = W.uniform_tree_flags(d, 3 if d == 2 else 2)
    else:
        flags = W.random_tree_flags(d, 4 if d == 2 else 3, 0.3, seed, min_depth=1)
    x, v = W.random_particles(d, n, seed, vmax=vmax)
    E = np.random.default_rng(seed).uniform(-0.5, 0.5, (d, oracle.Tree(d, flags).n_vertices))
    return flags, x, v, E


def _cexp(tree):
    ptr, vid, _ = tree.corner_expansion()
    return ptr, vid


def _rank(rank, world, port, cases, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        for ci, case in enumerate(cases):
            _one_case(rank, world, ci, case, out)
    finally:
        dist.destroy_process_group()


def _one_case(rank, world, ci, case, out):
    d, kind, n, vmax, seed, scheme, dt = case
    flags, x, v, E = _setup(d, kind, n, vmax, seed)
    tree = oracle.Tree(d, flags)
    part = PT.Partition(d, flags, world, _cexp(tree), level=1)
    ex = PT.Exchange(part, rank, dist)
    q, qm = -1.0 / n, -1.0
    # the canonical start, this rank's particles (its leaves), in order
    st = oracle.State64(tree, x, v, oracle.Params(scheme=scheme, q=q, qm=qm, sweeps=0))
    leaf0 = tree.pit_owner(st.x)
    mine = part.rank_of_leaf(leaf0) == rank
    lx, lv = np.ascontiguousarray(st.x[:, mine]), np.ascontiguousarray(st.v[:, mine])
    lid, lkey = st.ids[mine], st.key[mine]
    # 1. deposit halo of the rank's own particles (ion background apart)
    Qall, _ = tree.deposit64(scheme, lx, q, 0.0)
    Qh = ex.halo_sum(Qall[part.vertices[rank]])
    # 2. FP64 total: own charge + the ion load of the vertices this rank owns
    ion, _ = tree.vertex_aux()
    owner = np.full(tree.n_vertices, world)
    for r in range(world - 1, -1, -1):
        owner[part.vertices[r]] = r
    total = ex.total(q * lx.shape[1] + float(ion[owner == rank].sum()))
    # 3. push with the (replicated) field, new keys, migration
    tree.push64(lx, lv, E, qm, dt)
    nkey = tree.keys64(scheme, lx)
    dest = part.rank_of_leaf(tree.pit_owner(lx))
    vloc = float(np.abs(lv).max()) if lv.size else 0.0
    h_min = 3.0 ** -int(part.level.max())
    rapidt = not ex.flag_any(vloc * dt >= h_min)
    moved = (nkey != lkey).astype(np.int64)
    src = np.arange(lx.shape[1], dtype=np.int64)
    got = ex.migrate(dest, [lx, lv, lid, nkey, src], neighbour_only=rapidt)
    stay = dest == rank
    cols = [[lx[:, stay], lv[:, stay], lid[stay], nkey[stay], moved[stay], np.full(stay.sum(), rank),
             src[stay]]]
    for s, (rx, rv, rid, rkey, rsrc) in got:
        cols.append([rx, rv, rid, rkey, np.ones(len(rid), np.int64), np.full(len(rid), s), rsrc])
    X = np.concatenate([c[0] for c in cols], axis=1)
    V = np.concatenate([c[1] for c in cols], axis=1)
    ID, KEY, MOV, SR, SI = (np.concatenate([c[k] for c in cols]) for k in range(2, 7))
    # 4. re-bin: stable by (key, moved, source rank, source index)
    order = np.lexsort((SI, SR, MOV, KEY))
    out.put(((ci, rank), dict(ids=ID[order], key=KEY[order], x=X[:, order], v=V[:, order],
                              Q=Qh, verts=part.vertices[rank], total=total, rapidt=rapidt,
                              stats=dict(ex.stats))))
    dist.barrier()


_RESULTS = {}


def _run(world, cases):
    """All cases of one world size in one set of spawned gloo ranks."""
    if world in _RESULTS:
        return _RESULTS[world]
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, cases, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=600) for _ in range(world * len(cases)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    _RESULTS[world] = res
    return res


# d, tree, n, vmax, seed, scheme, dt
CASES = {
    2: [(2, "adaptive", 6000, 0.4, 11, oracle.PIT, 0.5),
        (3, "adaptive", 8000, 0.3, 14, oracle.PIDT, 0.4),
        (3, "uniform", 8000, 0.05, 15, oracle.PIT, 0.05)],
    4: [(2, "adaptive", 6000, 0.4, 11, oracle.PIT, 0.5),
        (2, "adaptive", 6000, 0.4, 12, oracle.PIDT, 0.5),
        (2, "uniform", 6000, 0.05, 13, oracle.PIT, 0.05)],
}
PARAMS = [pytest.param(w, i, id=f"w{w}-{c[0]}d-{c[1]}-{'pit' if c[5] == oracle.PIT else 'pidt'}")
          for w, cs in CASES.items() for i, c in enumerate(cs)]


@pytest.mark.parametrize("world,ci", PARAMS)
def test_partitioned_step_matches_single_rank(world, ci):
    case = CASES[world][ci]
    d, kind, n, vmax, seed, scheme, dt = case
    flags, x, v, E = _setup(d, kind, n, vmax, seed)
    tree = oracle.Tree(d, flags)
    q = -1.0 / n
    st = oracle.State64(tree, x, v, oracle.Params(scheme=scheme, q=q, qm=-1.0, sweeps=0))
    Q0, _ = tree.deposit64(scheme, st.x, q, 0.0)
    _, total0 = tree.deposit64(scheme, st.x, q, 1.0)
    tree.push64(st.x, st.v, E, -1.0, dt)
    st.rebin()
    part = PT.Partition(d, flags, world, _cexp(tree), level=1)
    allres = _run(world, CASES[world])
    res = {r: allres[(ci, r)] for r in range(world)}
    leaf = tree.pit_owner(st.x)
    rank_of = part.rank_of_leaf(leaf)
    assert sum(len(res[r]["ids"]) for r in res) == n
    for r in range(world):
        o = res[r]
        sel = rank_of == r
        if scheme == oracle.PIT:          # a contiguous slice of the single-rank array
            idx = np.flatnonzero(sel)
            assert len(idx) == 0 or np.array_equal(idx, np.arange(idx[0], idx[-1] + 1))
        assert np.array_equal(o["key"], st.key[sel]), r
        if scheme == oracle.PIT:
            assert np.array_equal(o["ids"], st.ids[sel]) and np.array_equal(o["x"], st.x[:, sel])
            assert np.array_equal(o["v"], st.v[:, sel])
        else:                             # same sets per bucket, same state per particle
            by_id = np.argsort(st.ids)
            for k in np.unique(o["key"]):
                a = o["ids"][o["key"] == k]
                b = st.ids[sel][st.key[sel] == k]
                assert np.array_equal(np.sort(a), np.sort(b))
            pos = by_id[o["ids"]]
            assert np.array_equal(o["x"], st.x[:, pos]) and np.array_equal(o["v"], st.v[:, pos])
        Qr = Q0[o["verts"]]
        assert np.max(np.abs(o["Q"] - Qr)) <= 1e-13 * np.abs(Q0).max()
        assert o["total"] == res[0]["total"]
        assert abs(o["total"] - total0) <= 1e-12 * max(1.0, abs(total0))
    rapidt = res[0]["rapidt"]
    assert all(res[r]["rapidt"] == rapidt for r in res)
    if vmax * dt < 3.0 ** -int(part.level.max()):
        assert rapidt and all(res[r]["stats"]["neighbour"] == 1 for r in res)
        assert all(res[r]["stats"]["all_to_all"] == 1 for r in res)   # the deposit halo only
    else:
        assert not rapidt and all(res[r]["stats"]["all_to_all"] == 2 for r in res)


def test_partition_cuts_at_subtree_boundaries_and_balances():
    d = 2
    flags = W.random_tree_flags(d, 4, 0.35, 21, min_depth=1)
    tree = oracle.Tree(d, flags)
    lev, co = PT.leaf_table(d, flags)
    olev, oco = tree.leaf_info()
    assert np.array_equal(lev, olev) and np.array_equal(co, oco)   # the same depth-first order
    for world in (2, 3, 4):
        part = PT.Partition(d, flags, world, _cexp(tree), level=1)
        st = part.leaf_start
        assert st[0] == 0 and st[-1] == tree.n_leaves and np.all(np.diff(st) >= 0)
        for c in st[1:-1]:   # a cut never splits a level-1 subtree
            a = co[c - 1] // 3 ** np.maximum(lev[c - 1] - 1, 0)
            b = co[c] // 3 ** np.maximum(lev[c] - 1, 0)
            assert not (min(lev[c - 1], lev[c]) >= 1 and np.array_equal(a, b))
        for r in range(world):
            for s in part.neighbours[r]:
                assert r in part.neighbours[s]


def test_rapidt_refuses_a_far_mover_before_sending():
    """A rank whose particle would go beyond its neighbours under a raPIDT
    promise raises on the host before any message is sent."""
    d = 2
    flags = W.uniform_tree_flags(d, 4)
    tree = oracle.Tree(d, flags)
    part = PT.Partition(d, flags, 16, _cexp(tree), level=2)
    far = [s for s in range(16) if s != 0 and s not in part.neighbours[0]]
    assert far

    class NoDist:
        def __getattr__(self, name):
            raise AssertionError("no collective may run")

    ex = PT.Exchange(part, 0, NoDist())
    with pytest.raises(RuntimeError, match="raPIDT"):
        ex.migrate(np.array([0, far[0]]), [np.zeros((2, 2))], neighbour_only=True)
