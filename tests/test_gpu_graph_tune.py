"""CUDA-graph replay of the fixed-field step and the autotuner, through the
C ABI: a replayed step is the same step (bit for bit), and tuning changes
timing only, never results or the particle state."""
from __future__ import annotations

import json

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

CASES = [
    pytest.param(3, "uniform", pic.PIT, pic.FP32_SPLIT, id="3d-brick-split-pit"),
    pytest.param(2, "uniform", pic.PIT, pic.FP32_SPLIT, id="2d-brick-split-pit"),
    pytest.param(3, "uniform", pic.PIDT, pic.FP64, id="3d-uniform-fp64-pidt"),
    pytest.param(2, "adaptive", pic.PIT, pic.FP64, id="2d-adaptive-fp64-pit"),
    pytest.param(2, "adaptive", pic.PIDT, pic.FP32_SPLIT, id="2d-adaptive-split-pidt"),
]


def case(d, kind, n=60_001, seed=3):
    flags = W.uniform_tree_flags(d, 4 if d == 2 else 3) if kind == "uniform" else \
        W.random_tree_flags(d, 5, 0.3, seed, min_depth=2)
    x, v = W.random_particles(d, n, seed, vmax=0.5)
    return flags, x, v


def handles(d, kind, scheme, precision, n=60_001):
    flags, x, v = case(d, kind, n)
    kw = dict(scheme=scheme, precision=precision, q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=5, omega=0.8)
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = pic.Pic(d, flags, x, v, stream=sa, **kw)
    b = pic.Pic(d, flags, x, v, stream=sb, **kw)
    for g in (a, b):
        g.step(0.05)  # a solved field, then fixed-field steps
    return a, b, (sa, sb)


def same(a, b):
    a.sync()
    b.sync()
    for u, w in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, w)
    sa, ia = a.bins()
    sb, ib = b.bins()
    assert np.array_equal(sa, sb) and np.array_equal(ia, ib)
    assert np.array_equal(a.keys(), b.keys())
    assert np.array_equal(a.deposit(), b.deposit())


@pytest.mark.parametrize("d,kind,scheme,precision", CASES)
def test_graph_replay_equals_steps(d, kind, scheme, precision):
    a, b, _streams = handles(d, kind, scheme, precision)
    dt = 0.07
    a.graph_capture(dt)          # one ordinary step, then capture
    a.graph_launch(3)
    a.step_fixed_field(dt)       # ordinary and replayed steps mix
    a.graph_launch(2)
    for _ in range(7):
        b.step_fixed_field(dt)
    same(a, b)
    assert a.stats().error == 0


@pytest.mark.parametrize("d,kind,scheme,precision", CASES[:1] + CASES[3:4])
def test_graph_dropped_by_state_change(d, kind, scheme, precision):
    a, b, _streams = handles(d, kind, scheme, precision)
    a.graph_capture(0.05)
    a.graph_launch(1)
    b.step_fixed_field(0.05)
    b.step_fixed_field(0.05)
    st = a.get_state()
    a.set_state(*st)
    with pytest.raises(pic.PicError):
        a.graph_launch(1)
    a.graph_capture(0.05)
    a.graph_launch(1)
    b.step_fixed_field(0.05)
    b.step_fixed_field(0.05)
    same(a, b)


def test_graph_needs_own_stream():
    flags, x, v = case(2, "uniform", 5000)
    g = pic.Pic(2, flags, x, v, precision=pic.FP32_SPLIT)
    with pytest.raises(pic.PicError):
        g.graph_capture(0.05)


@pytest.mark.parametrize("d,kind,scheme,precision", CASES)
def test_autotune_keeps_state_and_results(d, kind, scheme, precision, tmp_path):
    a, b, _streams = handles(d, kind, scheme, precision)
    before = a.get_state()
    tuned = a.autotune(0.05, trials=2)
    after = a.get_state()
    for u, w in zip(before, after):
        assert np.array_equal(u, w)
    assert tuned == a.tuning()
    info = a.info()
    assert tuned[0] in ((0, 1) if b.info().brick else (0,))
    assert all(t in (128, 256, 512) for t in tuned[1:])
    assert info.brick == tuned[0]
    for _ in range(3):
        a.step_fixed_field(0.05)
        b.step_fixed_field(0.05)
    same(a, b)
    # every candidate gives the same steps
    for t in ([0, 128, 128, 256], [0, 512, 256, 256]):
        a.set_tuning(t)
        b.step_fixed_field(0.05)
        a.step_fixed_field(0.05)
        same(a, b)
    # the cache returns the stored choice without timing again
    cache = tmp_path / "tune.json"
    t1 = a.autotune(0.05, trials=1, cache=str(cache))
    stored = json.loads(cache.read_text())
    assert list(stored.values()) == [t1]
    stored[next(iter(stored))] = [0, 128, 256, 256]
    cache.write_text(json.dumps(stored))
    assert a.autotune(0.05, cache=str(cache)) == [0, 128, 256, 256]
    assert a.tuning() == [0, 128, 256, 256]


def test_tuning_rejects_bad_values():
    flags, x, v = case(2, "adaptive", 5000)
    g = pic.Pic(2, flags, x, v, precision=pic.FP64)
    with pytest.raises(pic.PicError):
        g.set_tuning([1, 256, 256, 256])   # no brick path on an adaptive tree
    with pytest.raises(pic.PicError):
        g.set_tuning([0, 96, 256, 256])


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
def test_set_state_sorted_and_shuffled(scheme):
    """A state read back by get_state (keys ascending) re-enters unchanged and
    without a re-sort; the same particles shuffled go through the full re-bin,
    whose result is the stable sort of the shuffled input by key."""
    flags, x, v = case(3, "uniform", 50_000)
    kw = dict(scheme=scheme, precision=pic.FP32_SPLIT, q=-2e-5, qm=-1.0, ion=1.0, sweeps=5)
    a = pic.Pic(3, flags, x, v, **kw)
    b = pic.Pic(3, flags, x, v, **kw)
    a.step(0.05)
    b.step(0.05)
    leaf, o, vv = a.get_state()
    keys = a.keys()
    start0, _ = a.bins(with_ids=False)
    a.set_state(leaf, o, vv)                       # ascending keys: fast path
    a.sync()
    for u, w in zip(a.get_state(), (leaf, o, vv)):
        assert np.array_equal(u, w)
    assert np.array_equal(a.bins(with_ids=False)[0], start0) and np.array_equal(a.keys(), keys)
    perm = np.random.default_rng(1).permutation(leaf.size)
    b.set_state(np.ascontiguousarray(leaf[perm]), np.ascontiguousarray(o[:, perm]),
                np.ascontiguousarray(vv[:, perm]))  # shuffled: full re-bin
    b.sync()
    order = perm[np.argsort(keys[perm], kind="stable")]
    lb, ob, vb = b.get_state()
    assert np.array_equal(lb, leaf[order]) and np.array_equal(ob, o[:, order]) and np.array_equal(vb, vv[:, order])
    assert np.array_equal(b.bins(with_ids=False)[0], start0)
    # the fast path keeps stepping like an untouched handle
    c = pic.Pic(3, flags, x, v, **kw)
    c.step(0.05)
    for _ in range(2):
        a.step(0.05)
        c.step(0.05)
    for u, w in zip(a.get_state(), c.get_state()):
        assert np.array_equal(u, w)
