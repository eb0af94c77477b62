"""The stream-like calibration update (the particle-only benchmark of the
paper's memory-throughput experiment, Section 6): explicit Euler step and
reflection at the unit-box walls, in place, against the same arithmetic in
numpy (FP64 exactly; FP32 with separate roundings of product and sum)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover - CPU hosts
    pytest.skip("needs a CUDA device", allow_module_level=True)


def reference(x, v, dt, steps):
    x = x.copy()
    v = v.copy()
    dt = x.dtype.type(dt)
    for _ in range(steps):
        y = x + v * dt
        lo, hi = y < 0, y > 1
        y[lo] = -y[lo]
        y[hi] = x.dtype.type(2) - y[hi]
        v[lo | hi] = -v[lo | hi]
        x = y
    return x, v


@pytest.mark.parametrize("d", [2, 3])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
@pytest.mark.parametrize("n", [100_003, 100_000])      # scalar and 16-byte vector kernels
def test_stream_step_matches_reference(d, dtype, n):
    rng = np.random.default_rng(3)
    x = rng.random((d, n)).astype(dtype)
    v = rng.uniform(-0.3, 0.3, (d, n)).astype(dtype)   # many particles cross a wall in 5 steps
    xt, vt = torch.from_numpy(x).cuda(), torch.from_numpy(v).cuda()
    pic.stream_step(xt, vt, 0.1, steps=5)
    torch.cuda.synchronize()
    xr, vr = reference(x, v, 0.1, 5)
    assert np.array_equal(xt.cpu().numpy(), xr) and np.array_equal(vt.cpu().numpy(), vr)
    assert (xr >= 0).all() and (xr <= 1).all()


def test_stream_step_rejects_bad_arguments():
    lib = pic.load()
    assert lib.pic_stream_step(4, 0, None, None, 10, 0.1, 1, None) != 0
    assert lib.pic_stream_step(3, 0, None, None, 10, 0.1, 1, None) != 0
    assert lib.pic_stream_step(3, 0, None, None, 0, 0.1, 1, None) == 0
