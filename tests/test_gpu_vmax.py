"""The raPIDT tree attribute v_max (pic_vmax) against the oracle's, after
steps, on adaptive and uniform trees, PIT and PIDT, FP64 and split: node by
node equal (split: the same FP32 velocities, so the same maxima) or within
1e-12 (FP64 velocities, whose last bits follow the field's summation
order), and the count of closed cells (v_max dt < 3^-level) the same."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)

CASES = [
    pytest.param(2, lambda: W.random_tree_flags(2, 5, 0.3, 7, min_depth=2), id="2d-adaptive"),
    pytest.param(3, lambda: W.random_tree_flags(3, 3, 0.3, 8, min_depth=1), id="3d-adaptive"),
    pytest.param(3, lambda: W.uniform_tree_flags(3, 3), id="3d-uniform"),
]


@pytest.mark.parametrize("d,flags_fn", CASES)
@pytest.mark.parametrize("scheme", [pic.PIT, pic.PIDT])
@pytest.mark.parametrize("precision", [pic.FP64, pic.FP32_SPLIT])
def test_vmax_matches_oracle(d, flags_fn, scheme, precision):
    flags = flags_fn()
    n = 30_000
    x, v = W.random_particles(d, n, 23, vmax=0.2)
    q = -1.0 / n
    split = precision == pic.FP32_SPLIT
    prm = oracle.Params(scheme=scheme, q=q, qm=-1.0, ion=1.0, sweeps=10, omega=0.8)
    ot = oracle.Tree(d, flags)
    st = (oracle.State32 if split else oracle.State64)(ot, x, v, prm)
    g = pic.Pic(d, flags, x, v, scheme=scheme, precision=precision, q=q, qm=-1.0, ion=1.0, sweeps=10, omega=0.8)
    for _ in range(2):
        st.step(0.05)
        g.step(0.05)
    g.sync()
    leaf = st.leaf if split else ot.pit_owner(st.x)
    expect = ot.vmax(scheme, leaf, st.key, st.v)
    got, closed = g.vmax(dt=0.5)   # v_max dt ~ 0.1: open on the finest levels, closed above
    if split:   # the same FP32 velocities: the maxima are the same bits
        assert np.array_equal(got, expect)
    else:       # FP64 velocities agree to 1e-12 (the field's summation order differs)
        assert np.allclose(got, expect, rtol=1e-12, atol=0.0)
    lev = np.zeros(len(expect), np.int64)
    # node levels in level order, from the flags
    nch, cur, i = 3 ** d, [0], 0
    level_of = {0: 0}
    refined = np.flatnonzero(ot.flags)
    for k, r in enumerate(refined):
        for c in range(1 + nch * k, 1 + nch * (k + 1)):
            level_of[c] = level_of[int(r)] + 1
    lev = np.array([level_of[i] for i in range(len(expect))])
    assert closed == int(np.sum(expect * 0.5 < 3.0 ** -lev))
    assert 0 < closed < len(expect)
