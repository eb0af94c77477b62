"""pic_bucket_noalloc (stable bucket sort on file-scope device scratch)
against the handle's own re-bin: the buckets of fresh particles from
pic_bins.  Two different calls in a row check that the scratch left by one
call does not leak into the next."""
from __future__ import annotations

import ctypes as C

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)


def fresh_bins(d, flags, n, seed, scheme):
    """Keys in input order and the handle's bucket offsets / order."""
    x, v = W.random_particles(d, n, seed)
    g = pic.Pic(d, flags, x, v, scheme=scheme, precision=pic.FP64)
    keys_sorted = g.keys()
    start, ids = g.bins()
    keys_in = np.empty(n, np.int32)
    keys_in[ids] = keys_sorted
    n_keys = int(g.info().n_keys)
    return keys_in, n_keys, start, ids


def run(keys_in, n_keys, stream):
    keys = torch.from_numpy(keys_in).cuda()
    start = torch.full((n_keys + 1,), -7, dtype=torch.int32, device="cuda")
    perm = torch.full((keys_in.size,), -7, dtype=torch.int32, device="cuda")
    pic.bucket_noalloc(keys, n_keys, start, perm, stream=stream)
    return start, perm


def test_noalloc_matches_bins_two_calls():
    s = torch.cuda.Stream()
    a = fresh_bins(3, W.uniform_tree_flags(3, 3), 200_003, 1, pic.PIT)
    b = fresh_bins(2, W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), 90_001, 2, pic.PIT)
    outs = []
    with torch.cuda.stream(s):
        for keys_in, n_keys, _, _ in (a, b, a):
            outs.append(run(keys_in, n_keys, s))
    s.synchronize()
    for (keys_in, n_keys, start, ids), (gs, gp) in zip((a, b, a), outs):
        assert np.array_equal(gs.cpu().numpy().astype(np.int64), start)
        assert np.array_equal(gp.cpu().numpy(), ids)


def test_noalloc_pidt_keys_match_stable_sort():
    keys_in, n_keys, _, _ = fresh_bins(2, W.uniform_tree_flags(2, 4), 50_001, 3, pic.PIDT)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gs, gp = run(keys_in, n_keys, s)
    s.synchronize()
    order = np.argsort(keys_in, kind="stable")
    assert np.array_equal(gp.cpu().numpy(), order)
    assert np.array_equal(gs.cpu().numpy(), np.searchsorted(keys_in[order], np.arange(n_keys + 1)))


def test_noalloc_skips_out_of_range_and_empty():
    rng = np.random.default_rng(4)
    keys_in = rng.integers(-3, 40, 5000).astype(np.int32)
    gs, gp = run(keys_in, 37, None)
    torch.cuda.synchronize()
    valid = np.flatnonzero((keys_in >= 0) & (keys_in < 37))
    order = valid[np.argsort(keys_in[valid], kind="stable")]
    gs, gp = gs.cpu().numpy(), gp.cpu().numpy()
    assert gs[-1] == valid.size
    assert np.array_equal(gp[:valid.size], order)
    assert np.all(gp[valid.size:] == -7)   # left untouched
    gs0, _ = run(np.zeros(0, np.int32), 5, None)
    torch.cuda.synchronize()
    assert np.array_equal(gs0.cpu().numpy(), np.zeros(6, np.int32))


def test_noalloc_rejects_oversize():
    lib = pic.load()
    keys = torch.zeros(10, dtype=torch.int32, device="cuda")
    start = torch.zeros(16, dtype=torch.int32, device="cuda")
    perm = torch.zeros(10, dtype=torch.int32, device="cuda")
    rc = lib.pic_bucket_noalloc(C.c_void_p(keys.data_ptr()), 10, pic.NOALLOC_MAX_KEYS + 1,
                                C.c_void_p(start.data_ptr()), C.c_void_p(perm.data_ptr()), None)
    assert rc == -1
    with pytest.raises(pic.PicError, match="fixed scratch"):
        pic.bucket_noalloc(keys, pic.NOALLOC_MAX_KEYS + 1, start, perm)
    torch.cuda.synchronize()
    assert int(start.abs().sum()) == 0 and int(perm.abs().sum()) == 0   # nothing launched
