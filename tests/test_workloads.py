"""The seeded input recipes (no GPU): tree-flag layouts, the Langmuir quiet
start, the two-stream beams, the particle-handling starts of Section 6, the
Appendix A thermal plasma and the uneven batch are what their docstrings state,
and every draw is reproducible from its seed."""
from __future__ import annotations

import math

import numpy as np
import pytest

from paper_1508_02435_gb300 import workloads as W


@pytest.mark.parametrize("d,depth", [(2, 0), (2, 3), (3, 2)])
def test_uniform_flags_are_level_order_with_every_leaf_on_one_level(d, depth):
    f = W.uniform_tree_flags(d, depth)
    n_internal = sum(3 ** (l * d) for l in range(depth))
    assert f.dtype == np.uint8 and len(f) == n_internal + 3 ** (depth * d)
    assert f[:n_internal].all() and not f[n_internal:].any()
    # the same tree from the predicate form
    assert np.array_equal(f, W.tree_flags_from_predicate(d, depth, lambda lev, c: np.ones(len(c), bool)))


def test_predicate_flags_follow_the_child_order():
    # refine only the child with local digit 4 (x = 1, y = 1) of the root, in 2D
    f = W.tree_flags_from_predicate(2, 2, lambda lev, c: (c[:, 0] == 1) & (c[:, 1] == 1) if lev == 1
                                    else np.ones(len(c), bool))
    assert f[0] == 1 and list(f[1:10]) == [0, 0, 0, 0, 1, 0, 0, 0, 0] and len(f) == 1 + 9 + 9
    assert np.array_equal(W.tree_flags_from_predicate(3, 4, lambda lev, c: np.zeros(len(c), bool)), [0])


@pytest.mark.parametrize("d,depth,ppc,k", [(2, 3, 16, 1), (3, 2, 8, 2)])
def test_langmuir_quiet_start(d, depth, ppc, k):
    amp, vth = 0.01, 0.05
    w = W.langmuir(d, depth, ppc, vth=vth, amp=amp, k=k, seed=3)
    m = 3 ** depth * round(ppc ** (1 / d))
    assert w.n == ppc * 3 ** (depth * d) == m ** d
    assert w.x.min() >= 0.0 and w.x.max() < 1.0 and w.q == -1.0 / w.n and w.qm == -1.0
    # transverse coordinates: the stratified lattice, x fastest in the particle index
    g = (np.arange(m) + 0.5) / m
    assert np.array_equal(np.unique(w.x[1]), g)
    # the x coordinates carry density 1 + amp cos(2 pi k x): mean of cos(2 pi k x) = amp / 2
    assert abs(np.mean(np.cos(2 * math.pi * k * w.x[0])) - amp / 2) < 1e-6
    assert abs(np.mean(np.cos(2 * math.pi * (k + 1) * w.x[0]))) < 1e-6
    # quiet velocities: every line of equal initial x holds the Maxwellian quantiles
    vx = w.v[0].reshape(-1, m)            # rows: transverse index, columns: x index
    q = np.sort(vx[:, 0])
    assert np.allclose(np.sort(vx[:, m // 2]), q) and abs(np.std(w.v[0]) / vth - 1) < 0.05
    assert abs(np.std(w.v[1]) / vth - 1) < 0.05
    with pytest.raises(ValueError):
        W.langmuir(d, depth, 7)


def test_two_stream_beams():
    n, base = 60_000, 4
    w = W.two_stream(n=n, base_depth=base, seed=5)
    nb = int(round(0.1 * n))
    ub = 8.0 * 3.0 ** -(base + 1) / 0.1
    assert abs(np.mean(w.v[0, :nb]) - ub) < 1e-3 and abs(np.mean(w.v[0, nb:2 * nb]) + ub) < 1e-3
    assert abs(np.std(w.v[1, :2 * nb]) / 0.01 - 1) < 0.05
    assert abs(np.std(w.v[:, 2 * nb:]) / 0.05 - 1) < 0.05 and abs(np.mean(w.v[:, 2 * nb:])) < 1e-3
    assert w.x.min() >= 0 and w.x.max() < 1 and w.extra["max_depth"] == base + 2
    assert np.array_equal(w.flags, W.uniform_tree_flags(3, base))


@pytest.mark.parametrize("dam", [False, True])
def test_particle_handling_starts(dam):
    w = W.particle_handling(3, 50_000, dam=dam, seed=9)
    top = 0.1 if dam else 1.0
    assert w.x.min() >= 0 and w.x.max() < top and abs(np.mean(w.x) - top / 2) < 0.01 * top
    s = np.linalg.norm(w.v, axis=0)
    assert s.max() <= 1.0 and abs(np.mean(s) - 0.5) < 0.01 and abs(np.mean(s * s) - 1 / 3) < 0.01
    assert np.all(np.abs(np.mean(w.v / s, axis=1)) < 0.02)    # isotropic directions
    assert w.q == 0.0 and w.qm == 0.0 and w.ion == 0.0


def test_thermal_plasma_of_appendix_a():
    w = W.thermal_plasma(d=2, depth=3, ppc=20, seed=1)
    assert w.n == 20 * 3 ** 6 and w.dt == 0.01 and w.extra["vth"] == 1 / 27
    assert abs(np.std(w.v) * 27 - 1) < 0.03 and w.x.min() >= 0 and w.x.max() < 1


def test_uneven_batch():
    ws = W.batched_langmuir(n_inst=12, n_min=1000, n_max=20_000)
    for i, w in enumerate(ws):
        assert 1000 <= w.n <= 20_000 and w.extra["depth"] in (3, 4, 5) and w.k_mode in (1, 2, 4)
        assert 0.02 <= w.vth <= 0.1 and w.d == 2 and w.q == -1.0 / w.n
        assert np.array_equal(w.flags, W.uniform_tree_flags(2, w.extra["depth"]))
    again = W.batched_langmuir(n_inst=12, n_min=1000, n_max=20_000)
    assert all(np.array_equal(a.x, b.x) and np.array_equal(a.v, b.v) for a, b in zip(ws, again))
    assert len({w.n for w in ws}) > 6                 # uneven sizes


def test_draws_are_reproducible_from_their_seeds():
    for make in (lambda s: W.random_particles(3, 1000, s, vmax=0.5),
                 lambda s: (W.random_field(3, 500, s, 2.0),),
                 lambda s: (W.particle_handling(2, 1000, seed=s).v,),
                 lambda s: (W.two_stream(n=1000, seed=s).x,)):
        a, b, c = make(4), make(4), make(5)
        assert all(np.array_equal(p, q) for p, q in zip(a, b))
        assert not all(np.array_equal(p, q) for p, q in zip(a, c))
    x, v = W.random_particles(3, 1000, 4, vmax=0.5)
    assert x.min() >= 0 and x.max() < 1 and np.abs(v).max() <= 0.5
    f = W.random_field(3, 500, 4, 2.0)
    assert f.dtype == np.float32 and f.shape == (3, 500) and np.abs(f).max() <= 2.0
    t = W.random_tree_flags(2, 4, 0.3, seed=7, min_depth=2)
    assert np.array_equal(t, W.random_tree_flags(2, 4, 0.3, seed=7, min_depth=2))
    assert t[:1 + 9].all()                              # levels above min_depth all refined
