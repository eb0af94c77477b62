"""The finite-element and owner-vertex tables of adaptive trees tabulated on
the device (csrc/tree_dev.cu) against the host tabulation (pic_tree_tabulate,
itself pinned against the oracle in tests/test_host_tables.py): the same
vertices, leaf-corner expansions, vertex loads, stiffness diagonals and PIDT
owners, value for value; a handle built on host tables steps to the same
bits; re-refinement installs tables equal to the host's of the new tree."""
from __future__ import annotations

import os

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)


def slab_tree(d):
    """Uniform to a base depth (4 in 2D, 3 in 3D), one level more in a slab
    and a corner block, two more in a thinner slab: refinement jumps of one
    and two levels, as ppc trees have."""
    base = 4 if d == 2 else 3

    def refine(level, coords):
        c = coords.astype(np.float64)
        x = (c[:, 0] + 0.5) / 3 ** level
        y = (c[:, 1] + 0.5) / 3 ** level
        if level < base:
            return np.ones(len(c), bool)
        if level == base:
            return (np.abs(x - 0.5) < 0.2) | ((x < 0.15) & (y < 0.15))
        return (np.abs(x - 0.5) < 0.05) | ((x < 0.05) & (y < 0.05))
    return W.tree_flags_from_predicate(d, base + 2, refine)


TREES = [
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 5, min_depth=2), id="2d-random-a"),
    pytest.param(2, lambda: W.random_tree_flags(2, 8, 0.22, 11, min_depth=1), id="2d-random-deep"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 6, min_depth=1), id="3d-random-a"),
    pytest.param(3, lambda: W.random_tree_flags(3, 4, 0.08, 9, min_depth=2), id="3d-random-b"),
    pytest.param(2, lambda: slab_tree(2), id="2d-slabs"),
    pytest.param(3, lambda: slab_tree(3), id="3d-slabs"),
]


def compare_tables(g, d, flags, scheme):
    host = pic.tree_tables(d, flags)
    assert np.array_equal(g.vertex_table(), host["vertex_pos"])
    dev = g.grid_tables()
    for k in ("cexp_ptr", "cexp_vid", "cexp_w", "ion_load", "diag"):
        assert np.array_equal(dev[k], host[k]), k
    if scheme == pic.PIDT:
        lev, j = g.pidt_table()
        assert np.array_equal(lev, host["pidt_level"]) and np.array_equal(j, host["pidt_j"])
    return host


@pytest.mark.parametrize("d,flags_fn", TREES)
@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
def test_device_tables_equal_host_tables(d, flags_fn, scheme):
    flags = flags_fn()
    x, v = W.random_particles(d, 5000, 3, vmax=0.1)
    g = pic.Pic(d, flags, x, v, scheme=scheme, precision=pic.FP64, q=-1.0 / 5000, sweeps=2)
    host = compare_tables(g, d, flags, scheme)
    assert (np.diff(host["cexp_ptr"]) > 1).any()   # hanging vertices present


@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
def test_host_tabulated_handle_steps_to_the_same_bits(scheme, precision):
    d = 3
    flags = slab_tree(d)
    x, v = W.random_particles(d, 60_000, 4, vmax=0.05)
    kw = dict(scheme=scheme, precision=precision, q=-1.0 / 60_000, qm=-1.0, ion=1.0, sweeps=5, omega=0.8)
    dev = pic.Pic(d, flags, x, v, **kw)
    os.environ["PIC_HOST_TABLES"] = "1"
    try:
        host = pic.Pic(d, flags, x, v, **kw)
    finally:
        del os.environ["PIC_HOST_TABLES"]
    for _ in range(2):
        dev.step(0.05)
        host.step(0.05)
    dev.sync()
    host.sync()
    for a, b in zip(dev.get_state(), host.get_state()):
        assert np.array_equal(a, b)
    assert np.array_equal(dev.deposit(), host.deposit())
    assert np.array_equal(dev.field(), host.field())


@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
def test_refinement_installs_device_tables_of_the_new_tree(scheme):
    d = 2
    w = W.particle_handling(d, 40_000, dam=True, seed=8)
    g = pic.Pic(d, w.flags, w.x, w.v, scheme=scheme, precision=pic.FP32_SPLIT, q=0.0, qm=0.0, ion=0.0, sweeps=0)
    for _ in range(3):
        g.adapt(50, 1, 7)
        compare_tables(g, d, g.tree_flags(), scheme)
        g.step_particles(0.05, reflect=True)
