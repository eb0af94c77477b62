"""Partitioned single plasma over several ranks (one GPU each): the exchange
layer of the particle step.

The paper cuts the spacetree into non-overlapping subtrees along the
space-filling (depth-first) order and replicates the vertices on partition
faces (Section 4.3); lifts and drops across a partition face become
master-worker communication (Sections 5.1-5.3), and raPIDT (Section 5.4)
avoids that communication when the tree attribute v_max shows that no
particle can leave.  Here the same decomposition serves data-parallel ranks:

* Partition: the leaves in depth-first order are cut into `world` contiguous
  ranges, at boundaries of level-`level` subtrees, balanced by a weight per
  leaf.  Rank r owns the particles whose leaf lies in its range, so the
  concatenation of the ranks' bucket-sorted arrays is the single-rank array.
  A vertex is replicated on every rank whose leaves' corners expand onto it.
* Per step, with the local compute done by each rank's backend (the GPU
  library; the tests use the CPU oracle):
    1. deposit halo: a rank deposits its own particles onto its vertices;
       the partial charges of replicated vertices are exchanged and every
       rank sums the contributions of all ranks in rank order;
    2. FP64 totals (charge neutrality, residual norms): partials gathered and
       summed in rank order, the same bits on every rank;
    3. migration: pushed particles whose new leaf belongs to another rank go
       there, in storage order -- a count exchange, then the payload
       (all-to-all-v).  With raPIDT (every rank's v_max dt is below the width
       of its finest leaf, so no particle moves past a leaf touching its own)
       only neighbouring ranks can receive, and the exchange runs between
       neighbours (point-to-point) instead of the global all-to-all;
    4. re-bin: each rank orders its particles stably by (new key, moved, old
       global storage index) -- its slice of the single-rank canonical order.

Only torch.distributed collectives are used (NCCL on GPUs, gloo on CPU);
no TMA or multicast touches another rank's memory.  The field solve's halo
(one exchange of replicated vertex values per sweep) is the same primitive
as the deposit halo (`halo_sum` of the per-rank partial products A V).
"""
from __future__ import annotations

import numpy as np

__all__ = ["leaf_table", "uniform_corner_expansion", "Partition", "Exchange"]


def leaf_table(d: int, flags) -> tuple[np.ndarray, np.ndarray]:
    """(level[n_leaves], coords[n_leaves, d]) of the tree given by level-order
    refinement flags, leaves in depth-first order (children in digit order
    l = i0 + 3 i1 + 9 i2)."""
    flags = np.asarray(flags, np.uint8)
    nch = 3 ** d
    n = len(flags)
    child0 = np.full(n, -1, np.int64)
    refined = np.flatnonzero(flags)
    child0[refined] = 1 + nch * np.arange(len(refined))
    level = np.zeros(n, np.int64)
    coords = np.zeros((n, d), np.int64)
    digit = np.arange(nch)
    offs = np.stack([(digit // 3 ** a) % 3 for a in range(d)], axis=1)
    for i in refined:                       # parents precede children in level order
        c = child0[i]
        level[c:c + nch] = level[i] + 1
        coords[c:c + nch] = 3 * coords[i][None, :] + offs
    out_l, out_c, stack = [], [], [0]
    while stack:
        i = stack.pop()
        if child0[i] < 0:
            out_l.append(level[i])
            out_c.append(coords[i])
        else:
            stack.extend(range(child0[i] + nch - 1, child0[i] - 1, -1))
    return np.array(out_l, np.int64), np.array(out_c, np.int64).reshape(-1, d)


def uniform_corner_expansion(d: int, depth: int):
    """(ptr, vid) of every leaf corner of the uniform tree of `depth` onto
    its vertex (row-major on that level, periodic): one entry per corner."""
    lev, co = leaf_table(d, np.concatenate([np.ones(sum(3 ** (l * d) for l in range(depth)), np.uint8),
                                            np.zeros(3 ** (depth * d), np.uint8)]))
    M = 3 ** depth
    nc = 1 << d
    vid = np.zeros((len(lev), nc), np.int64)
    for e in range(nc):
        v = np.zeros(len(lev), np.int64)
        mul = 1
        for a in range(d):
            v += ((co[:, a] + ((e >> a) & 1)) % M) * mul
            mul *= M
        vid[:, e] = v
    return np.arange(len(lev) * nc + 1, dtype=np.int64), vid.reshape(-1)


class Partition:
    """Contiguous depth-first leaf ranges per rank, cut at subtree boundaries
    of `level`, balanced by `weight` (one value per leaf; default 1).

    `cexp` = (ptr, vid): the vertices every leaf corner expands onto
    (hanging corners onto their coarse face's vertices), leaf corner
    i = leaf 2^d + corner -- from the host tabulation of the tree."""

    def __init__(self, d: int, flags, world: int, cexp, level: int = 1, weight=None):
        self.d, self.world = d, world
        self.level, self.coords = leaf_table(d, flags)
        nl = len(self.level)
        w = np.ones(nl) if weight is None else np.asarray(weight, np.float64)
        # admissible cut points: leaves that start a level-`level` subtree
        anc = self.coords // (3 ** np.maximum(self.level - level, 0))[:, None]
        anc_l = np.minimum(self.level, level)
        key = anc_l * (3 ** (level * d)) + sum(anc[:, a] * (3 ** level) ** a for a in range(d))
        cut_ok = np.ones(nl + 1, bool)
        cut_ok[1:nl] = key[1:] != key[:-1]
        cw = np.concatenate([[0.0], np.cumsum(w)])
        start = [0]
        for r in range(1, world):
            target = cw[-1] * r / world
            cand = np.flatnonzero(cut_ok & (np.arange(nl + 1) > start[-1]))
            i = cand[np.argmin(np.abs(cw[cand] - target))] if len(cand) else nl
            start.append(int(i))
        start.append(nl)
        self.leaf_start = np.maximum.accumulate(np.array(start, np.int64))
        self.rank_of = np.repeat(np.arange(world), np.diff(self.leaf_start))
        # vertices per rank (replicated on every rank whose corners expand onto them)
        ptr, vid = (np.asarray(a, np.int64) for a in cexp)
        nc = 1 << d
        corner_rank = np.repeat(self.rank_of, nc)
        entry_rank = np.repeat(corner_rank, np.diff(ptr))
        self.vertices = [np.unique(vid[entry_rank == r]) for r in range(world)]
        self.shared = {(r, s): np.intersect1d(self.vertices[r], self.vertices[s])
                       for r in range(world) for s in range(world) if r != s}
        self.neighbours = [sorted(s for s in range(world) if s != r and len(self.shared[(r, s)]) > 0)
                           for r in range(world)]
        self.finest = [int(self.level[self.rank_of == r].max()) if np.any(self.rank_of == r) else 0
                       for r in range(world)]

    def rank_of_leaf(self, leaf) -> np.ndarray:
        return self.rank_of[np.asarray(leaf, np.int64)]

    def leaves(self, r: int) -> tuple[int, int]:
        return int(self.leaf_start[r]), int(self.leaf_start[r + 1])


class Exchange:
    """The collectives of one rank over a torch.distributed process group."""

    def __init__(self, part: Partition, rank: int, dist, group=None):
        self.part, self.rank, self.dist, self.group = part, rank, dist, group
        self.stats = {"all_to_all": 0, "neighbour": 0}

    # ---- FP64 totals ------------------------------------------------------
    def total(self, x: float) -> float:
        """Sum over ranks of x in rank order (the same bits everywhere)."""
        import torch
        mine = torch.tensor([x], dtype=torch.float64)
        parts = [torch.zeros(1, dtype=torch.float64) for _ in range(self.part.world)]
        self.dist.all_gather(parts, mine, group=self.group)
        s = 0.0
        for p in parts:
            s += float(p[0])
        return s

    def flag_any(self, flag: bool) -> bool:
        import torch
        t = torch.tensor([1 if flag else 0], dtype=torch.int32)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX, group=self.group)
        return bool(t[0])

    # ---- halo of replicated vertices ------------------------------------
    def halo_sum(self, values: np.ndarray) -> np.ndarray:
        """values[k] = this rank's partial at vertex part.vertices[rank][k];
        returns the sum over all ranks holding each vertex, added in rank
        order.  One all-to-all-v of the shared vertices' partials."""
        import torch
        P, r = self.part, self.rank
        mine = P.vertices[r]
        values = np.asarray(values, np.float64)
        send, sizes = [], []
        for s in range(P.world):
            if s == r:
                sizes.append(0)
                continue
            idx = np.searchsorted(mine, P.shared[(r, s)])
            send.append(values[idx])
            sizes.append(len(idx))
        recv_sizes = [0 if s == r else len(P.shared[(s, r)]) for s in range(P.world)]
        sbuf = torch.from_numpy(np.concatenate(send) if send else np.zeros(0))
        rbuf = torch.zeros(sum(recv_sizes), dtype=torch.float64)
        self.dist.all_to_all_single(rbuf, sbuf, recv_sizes, sizes, group=self.group)
        self.stats["all_to_all"] += 1
        got = rbuf.numpy()
        contrib = {r: values}
        off = 0
        for s in range(P.world):
            n = recv_sizes[s]
            if s != r and n:
                full = np.zeros(len(mine))
                full[np.searchsorted(mine, P.shared[(s, r)])] = got[off:off + n]
                contrib[s] = full
            off += n
        out = np.zeros(len(mine))
        for s in sorted(contrib):
            out = out + contrib[s]
        return out

    # ---- particle migration ----------------------------------------------
    def migrate(self, dest: np.ndarray, rows: list, neighbour_only: bool):
        """Send every particle i with dest[i] != rank (in storage order) to
        rank dest[i]; rows are per-particle arrays ([..., n], any dtype,
        sent as float64 or int64).  Returns, per source rank in rank order,
        the received rows.  neighbour_only: the destinations are known to be
        neighbour ranks, so counts and payload go point-to-point between
        neighbours (raPIDT) instead of through the global all-to-all."""
        import torch
        P, r = self.part, self.rank
        dest = np.asarray(dest, np.int64)
        peers = P.neighbours[r] if neighbour_only else [s for s in range(P.world) if s != r]
        if neighbour_only and np.any((dest != r) & ~np.isin(dest, peers)):
            raise RuntimeError("raPIDT promised neighbour-only migration, but a particle leaves farther")
        sel = {s: np.flatnonzero(dest == s) for s in peers}
        flat_rows = [np.asarray(a).reshape(-1, np.asarray(a).shape[-1]) for a in rows]   # [width_a, n]
        width = sum(fr.shape[0] for fr in flat_rows)

        def pack(s):
            # one record of `width` float64 values per particle, particles in storage order
            if not len(sel[s]):
                return np.zeros(0)
            return np.concatenate([fr[:, sel[s]].astype(np.float64) for fr in flat_rows], axis=0).T.reshape(-1)

        counts_out = {s: len(sel[s]) for s in peers}
        if neighbour_only:
            self.stats["neighbour"] += 1
            cin = {s: torch.zeros(1, dtype=torch.int64) for s in peers}
            keep = [torch.tensor([counts_out[s]], dtype=torch.int64) for s in peers]
            reqs = [self.dist.isend(keep[i], s, group=self.group) for i, s in enumerate(peers)]
            reqs += [self.dist.irecv(cin[s], s, group=self.group) for s in peers]
            for q in reqs:
                q.wait()
            counts_in = {s: int(cin[s][0]) for s in peers}
            bufs_out = {s: torch.from_numpy(pack(s)) for s in peers}
            bufs_in = {s: torch.zeros(counts_in[s] * width, dtype=torch.float64) for s in peers}
            reqs = [self.dist.isend(bufs_out[s], s, group=self.group) for s in peers if counts_out[s]]
            reqs += [self.dist.irecv(bufs_in[s], s, group=self.group) for s in peers if counts_in[s]]
            for q in reqs:
                q.wait()
            recv = {s: bufs_in[s].numpy() for s in peers}
        else:
            self.stats["all_to_all"] += 1
            cout = torch.tensor([counts_out.get(s, 0) for s in range(P.world)], dtype=torch.int64)
            cin = torch.zeros(P.world, dtype=torch.int64)
            self.dist.all_to_all_single(cin, cout, group=self.group)
            counts_in = {s: int(cin[s]) for s in range(P.world) if s != r}
            sbuf = torch.from_numpy(np.concatenate([pack(s) for s in range(P.world) if s != r] or [np.zeros(0)]))
            ssz = [0 if s == r else counts_out[s] * width for s in range(P.world)]
            rsz = [0 if s == r else counts_in[s] * width for s in range(P.world)]
            rbuf = torch.zeros(sum(rsz), dtype=torch.float64)
            self.dist.all_to_all_single(rbuf, sbuf, rsz, ssz, group=self.group)
            got = rbuf.numpy()
            recv, off = {}, 0
            for s in range(P.world):
                recv[s] = got[off:off + rsz[s]]
                off += rsz[s]
        out = []
        for s in sorted(recv):
            if s == r:
                continue
            m = len(recv[s]) // width if width else 0
            rec = recv[s].reshape(m, width).T          # [width, m]
            cols, k = [], 0
            for a, fr in zip(rows, flat_rows):
                w = fr.shape[0]
                shp = np.asarray(a).shape[:-1]
                cols.append(rec[k:k + w].reshape(shp + (m,)).astype(np.asarray(a).dtype))
                k += w
            out.append((s, cols))
        return out
