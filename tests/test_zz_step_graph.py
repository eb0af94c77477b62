"""The whole time step as a CUDA graph (pic_graph_capture_step): deposit,
built-in solve, gather + push, re-bin.  Replays must give the same bits as
ordinary pic_step calls, and ordinary steps after the replays continue from
the same state."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

DT = 0.05

CASES = [
    pytest.param(3, "uniform", pic.PIT, pic.FP32_SPLIT, id="3d-brick-split-pit"),
    pytest.param(2, "adaptive", pic.PIDT, pic.FP32_SPLIT, id="2d-adaptive-split-pidt"),
    pytest.param(3, "uniform", pic.PIDT, pic.FP64, id="3d-uniform-fp64-pidt"),
    pytest.param(2, "adaptive", pic.PIT, pic.FP64, id="2d-adaptive-fp64-pit"),
]


def same(a, b):
    a.sync()
    b.sync()
    for u, w in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, w)
    for u, w in zip(a.bins(), b.bins()):
        assert np.array_equal(u, w)
    assert np.array_equal(a.potential(), b.potential())
    assert np.array_equal(a.field(), b.field())
    assert a.stats().step == b.stats().step
    assert a.stats().error == 0


@pytest.mark.parametrize("d,kind,scheme,precision", CASES)
def test_whole_step_replay_equals_steps(d, kind, scheme, precision):
    flags = W.uniform_tree_flags(d, 4 if d == 2 else 3) if kind == "uniform" else \
        W.random_tree_flags(d, 5, 0.3, 9, min_depth=2)
    n = 50_001
    x, v = W.random_particles(d, n, 9, vmax=0.5)
    kw = dict(scheme=scheme, precision=precision, q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=5, omega=0.8)
    a = pic.Pic(d, flags, x, v, stream=torch.cuda.Stream(), **kw)
    b = pic.Pic(d, flags, x, v, stream=torch.cuda.Stream(), **kw)
    for g in (a, b):
        g.init_leapfrog(DT)
    a.graph_capture_step(DT)  # one ordinary step, then the capture
    b.step(DT)
    same(a, b)
    a.graph_launch(3)
    for _ in range(3):
        b.step(DT)
    same(a, b)
    a.step(DT)
    b.step(DT)
    same(a, b)


def test_whole_step_replay_of_a_batch():
    ws = W.batched_langmuir(n_inst=6, n_min=300, n_max=8000)
    args = (2, [w.flags for w in ws], [w.x for w in ws], [w.v for w in ws], [w.q for w in ws])
    a = pic.Pic.batch(*args, precision=pic.FP32_SPLIT, sweeps=5, stream=torch.cuda.Stream())
    b = pic.Pic.batch(*args, precision=pic.FP32_SPLIT, sweeps=5, stream=torch.cuda.Stream())
    a.graph_capture_step(0.1)
    b.step(0.1)
    a.graph_launch(4)
    for _ in range(4):
        b.step(0.1)
    same(a, b)
