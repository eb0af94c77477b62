"""Checkpoint and resume through the C ABI (pic_save / pic_load): a handle
loaded from a checkpoint holds the saved state in the saved order, and its
later steps give the same bits as the steps of the handle it was saved from.
Saving both after the same steps writes byte-identical files."""
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


def case(d, kind, n=30_001, seed=5):
    flags = W.uniform_tree_flags(d, 4 if d == 2 else 3) if kind == "uniform" else \
        W.random_tree_flags(d, 5, 0.3, seed, min_depth=2)
    x, v = W.random_particles(d, n, seed, vmax=0.5)
    return flags, x, v


def same(a, b):
    a.sync()
    b.sync()
    for u, w in zip(a.get_state(), b.get_state()):
        assert np.array_equal(u, w)
    sa, ia = a.bins()
    sb, ib = b.bins()
    assert np.array_equal(sa, sb) and np.array_equal(ia, ib)
    assert np.array_equal(a.potential(), b.potential())
    assert np.array_equal(a.field(), b.field())
    assert np.array_equal(a.deposit(), b.deposit())
    assert a.stats().step == b.stats().step


@pytest.mark.parametrize("d,kind,scheme,precision", CASES)
def test_resume_gives_the_same_steps(d, kind, scheme, precision, tmp_path):
    flags, x, v = case(d, kind)
    n = x.shape[1]
    sa, sb = torch.cuda.Stream(), torch.cuda.Stream()
    a = pic.Pic(d, flags, x, v, scheme=scheme, precision=precision, q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=5,
                omega=0.8, stream=sa)
    a.init_leapfrog(DT)
    for _ in range(3):
        a.step(DT)
    a.sync()
    path = tmp_path / "a.ckpt"
    a.save(path)
    b = pic.Pic.load(path, stream=sb)
    ia, ib = a.info(), b.info()
    for k in ("d", "scheme", "precision", "depth", "n_particles", "n_leaves", "n_vertices", "n_buckets",
              "n_keys", "uniform", "brick", "n_instances"):
        assert getattr(ia, k) == getattr(ib, k), k
    assert b.tuning() == a.tuning()
    assert np.array_equal(b.tree_flags(), a.tree_flags())
    same(a, b)
    for _ in range(3):
        a.step(DT)
        b.step(DT)
    same(a, b)
    a.step_fixed_field(DT)
    b.step_fixed_field(DT)
    same(a, b)
    pa, pb = tmp_path / "a2.ckpt", tmp_path / "b2.ckpt"
    a.save(pa)
    b.save(pb)
    assert pa.read_bytes() == pb.read_bytes()


def test_resume_of_a_batch(tmp_path):
    ws = W.batched_langmuir(n_inst=5, n_min=200, n_max=5000)
    s0, s1 = torch.cuda.Stream(), torch.cuda.Stream()
    a = pic.Pic.batch(2, [w.flags for w in ws], [w.x for w in ws], [w.v for w in ws], [w.q for w in ws],
                      precision=pic.FP32_SPLIT, sweeps=5, stream=s0)
    for _ in range(2):
        a.step(0.1)
    a.sync()
    path = tmp_path / "batch.ckpt"
    a.save(path)
    b = pic.Pic.load(path, stream=s1)
    for u, w in zip(a.instances(), b.instances()):
        assert np.array_equal(u, w)
    same(a, b)
    for _ in range(2):
        a.step(0.1)
        b.step(0.1)
    same(a, b)


def test_save_after_a_tuning_change_restores_it(tmp_path):
    flags, x, v = case(3, "uniform")
    a = pic.Pic(3, flags, x, v, precision=pic.FP32_SPLIT, q=-1.0 / x.shape[1], sweeps=5,
                stream=torch.cuda.Stream())
    a.step(DT)
    a.set_tuning([0, 512, 128, 256])
    path = tmp_path / "t.ckpt"
    a.save(path)
    b = pic.Pic.load(path, stream=torch.cuda.Stream())
    assert b.tuning() == [0, 512, 128, 256] and b.info().brick == 0
    a.step_fixed_field(DT)
    b.step_fixed_field(DT)
    same(a, b)


def test_load_rejects_a_corrupted_checkpoint(tmp_path):
    flags, x, v = case(2, "uniform", n=2000)
    a = pic.Pic(2, flags, x, v, precision=pic.FP32_SPLIT, stream=torch.cuda.Stream())
    path = tmp_path / "c.ckpt"
    a.save(path)
    data = bytearray(path.read_bytes())
    data[-1] ^= 1  # last byte of E
    path.write_bytes(bytes(data))
    with pytest.raises(pic.PicError) as e:
        pic.Pic.load(path)
    assert e.value.code == -8
