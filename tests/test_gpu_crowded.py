"""Crowded buckets: a leaf or key that collects a large share of all particles
must sort in O(m log^2 m), not in a per-thread insertion sort, and keep the
canonical order (stayers, then movers in storage order; for fresh keys: input
order) bit for bit.

* the generic re-bin with half a million arrivals in one bucket;
* the brick path with a leaf of tens of thousands of arrivals (its unit
  overflows the staging area: global-memory pull) and a leaf of several
  hundred (shared-memory pull, warp network);
* pic_bucket_noalloc with few keys and many elements, and its argument checks.
"""
from __future__ import annotations

import time

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)


def test_generic_rebin_half_a_million_in_one_bucket():
    """1e6 fresh particles, every other one in leaf 0 (keys not ascending, so
    the full re-bin runs): bucket 0 receives 5e5 movers and must list them in
    input order, like numpy's stable argsort; then one step in which every
    particle moves keeps matching the oracle."""
    d, n = 2, 1_000_000
    flags = W.uniform_tree_flags(d, 2)             # 81 leaves of width 1/9
    rng = np.random.default_rng(21)
    x = rng.random((d, n))
    x[:, 0::2] = 0.01 + 0.09 * rng.random((d, n // 2))   # leaf 0
    v = rng.uniform(-0.05, 0.05, (d, n))
    t0 = time.perf_counter()
    g = pic.Pic(d, flags, x, v, scheme=pic.PIT, precision=pic.FP64, q=-1.0 / n, sweeps=3, omega=0.8,
                path=pic.PATH_GENERIC)
    g.sync()
    took = time.perf_counter() - t0
    t = oracle.Tree(d, flags)
    key = t.keys64(oracle.PIT, x)
    order = np.argsort(key, kind="stable")
    start, ids = g.bins()
    assert np.array_equal(ids, order)
    assert int(start[1] - start[0]) >= n // 2
    assert took < 30.0, took
    st = oracle.State64(t, x, v, oracle.Params(scheme=oracle.PIT, q=-1.0 / n, sweeps=3, omega=0.8))
    st.step(0.1)
    g.step(0.1)
    g.sync()
    start, ids = g.bins()
    assert np.array_equal(ids, st.ids)
    assert g.stats().max_bucket >= n // 4


def test_brick_path_crowded_leaves():
    """A brick-path plasma (27^3 leaves, FP32 split, PIT) with 25,000
    particles in one leaf (its destination unit overflows the staging area)
    and 600 in another leaf of a different brick (sorted in shared memory):
    two steps bit-identical to the generic path and to the oracle's mirror."""
    d, n = 3, 150_000
    flags = W.uniform_tree_flags(d, 3)
    rng = np.random.default_rng(22)
    x = rng.random((d, n))
    v = rng.uniform(-0.01, 0.01, (d, n))
    x[:, :25_000] = (13 + rng.random((d, 25_000))) / 27          # leaf (13, 13, 13)
    x[:, 25_000:25_600] = (2 + rng.random((d, 600))) / 27         # leaf (2, 2, 2)
    v[:, :25_600] *= 0.2
    # q/m = 0: the crowd's own field would blow it apart in one step; the
    # drift alone keeps it in place while the background moves through
    kw = dict(q=-1.0 / n, qm=0.0, ion=1.0, sweeps=3, omega=0.8)
    fast = pic.Pic(d, flags, x, v, scheme=pic.PIT, precision=pic.FP32_SPLIT, path=pic.PATH_AUTO, **kw)
    slow = pic.Pic(d, flags, x, v, scheme=pic.PIT, precision=pic.FP32_SPLIT, path=pic.PATH_GENERIC, **kw)
    assert fast.info().brick == 1
    st = oracle.State32(oracle.Tree(d, flags), x, v, oracle.Params(scheme=oracle.PIT, **kw))
    for step in range(2):
        fast.step(0.1)
        slow.step(0.1)
        st.step(0.1)
        fast.sync()
        slow.sync()
        for a, b in zip(fast.get_state(), slow.get_state()):
            assert np.array_equal(a, b), f"brick and generic states differ at step {step}"
        sf, idf = fast.bins()
        assert np.array_equal(idf, st.ids), f"order differs from the oracle at step {step}"
        leaf, o, vv = fast.get_state()
        assert np.array_equal(leaf, st.leaf) and np.array_equal(o, st.o) and np.array_equal(vv, st.v)
        assert fast.stats().max_bucket >= 20_000


@pytest.mark.parametrize("n,n_keys,hot", [(200_000, 3, None), (1_000_003, 17, 5)])
def test_noalloc_few_keys_many_elements(n, n_keys, hot):
    """2e5 keys into 3 buckets, and 1e6 keys with one bucket holding 90% of
    them: the same offsets and order as a stable argsort, in milliseconds."""
    rng = np.random.default_rng(n)
    keys_in = rng.integers(0, n_keys, n).astype(np.int32)
    if hot is not None:
        keys_in[rng.random(n) < 0.9] = hot
    keys = torch.from_numpy(keys_in).cuda()
    start = torch.empty(n_keys + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    pic.bucket_noalloc(keys, n_keys, start, perm)     # first call: set-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    pic.bucket_noalloc(keys, n_keys, start, perm)
    e1.record()
    torch.cuda.synchronize()
    order = np.argsort(keys_in, kind="stable")
    assert np.array_equal(perm.cpu().numpy(), order)
    assert np.array_equal(start.cpu().numpy(), np.searchsorted(keys_in[order], np.arange(n_keys + 1)))
    assert e0.elapsed_time(e1) < 200.0, e0.elapsed_time(e1)


def test_noalloc_rejects_bad_tensors_before_launch():
    """Wrong dtype, host memory, non-contiguous views and short outputs raise
    before any kernel runs (the outputs stay untouched)."""
    keys = torch.zeros(64, dtype=torch.int32, device="cuda")
    start = torch.full((9,), -5, dtype=torch.int32, device="cuda")
    perm = torch.full((64,), -5, dtype=torch.int32, device="cuda")
    bad = [
        (keys.to(torch.int64), 8, start, perm),
        (keys.cpu(), 8, start, perm),
        (keys, 8, start.to(torch.int64), perm),
        (keys, 8, start[:5], perm),
        (keys, 8, start, perm[:63]),
        (keys, 8, start, torch.full((128,), -5, dtype=torch.int32, device="cuda")[::2]),
    ]
    for k, nk, s, p in bad:
        with pytest.raises(pic.PicError):
            pic.bucket_noalloc(k, nk, s, p)
    torch.cuda.synchronize()
    assert int((start != -5).sum()) == 0 and int((perm != -5).sum()) == 0
