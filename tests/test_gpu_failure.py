"""Failure paths that need a device, made without faulting, trapping or
hanging it: a field-solve hook that reports an error, and a bounded device
wait that runs out (a barrier armed for bytes that are never sent).  After
each failure the context stays usable."""
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

PIC_ETIMEOUT, PIC_EHOOK = -5, -4


def _plasma(precision=pic.FP64):
    x, v = W.random_particles(2, 5000, 3, vmax=0.05)
    return pic.Pic(2, W.uniform_tree_flags(2, 3), x, v, scheme=pic.PIT, precision=precision, q=-1.0 / 5000,
                   sweeps=5, omega=0.8)


def test_hook_failure_is_reported_and_the_handle_survives():
    calls = []

    @pic.SOLVE_FN
    def failing(user, Q, E, nv, precision, stream):
        calls.append(int(nv))
        return 3

    g = _plasma()
    with pytest.raises(pic.PicError) as e:
        g.step(0.05, C.cast(failing, C.c_void_p), None)
    assert e.value.code == PIC_EHOOK and calls
    assert "returned 3" in g.lib.pic_last_error(g.h).decode()
    g.step(0.05)            # the built-in solve still works on the same handle
    g.sync()
    assert g.stats().error == 0


def test_bounded_wait_gives_up_and_returns():
    """A wait of 1e5 cycles on a barrier that never completes: the kernel
    returns and reports the timeout; a full plasma step runs afterwards."""
    s = torch.cuda.Stream()
    assert pic.wait_selftest(100_000, s) == PIC_ETIMEOUT
    assert pic.wait_selftest(1_000_000) == PIC_ETIMEOUT
    g = _plasma(pic.FP32_SPLIT)
    g.step(0.05)
    g.sync()
    assert g.stats().error == 0


def test_wait_limit_is_validated_and_kept_for_steps():
    x, v = W.random_particles(3, 30_000, 4, vmax=0.05)
    g = pic.Pic(3, W.uniform_tree_flags(3, 3), x, v, scheme=pic.PIT, precision=pic.FP32_SPLIT,
                q=-1.0 / 30_000, sweeps=3, omega=0.8)
    assert g.info().brick == 1
    with pytest.raises(pic.PicError):
        g.set_wait_limit(10)
    g.set_wait_limit(2_000_000_000)      # about a second: the bulk copies land long before
    ref = pic.Pic(3, W.uniform_tree_flags(3, 3), x, v, scheme=pic.PIT, precision=pic.FP32_SPLIT,
                  q=-1.0 / 30_000, sweeps=3, omega=0.8)
    for _ in range(2):
        g.step(0.1)
        ref.step(0.1)
    g.sync()
    ref.sync()
    for a, b in zip(g.get_state(), ref.get_state()):
        assert np.array_equal(a, b)
