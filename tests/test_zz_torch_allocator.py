"""Device memory of a handle from PyTorch's caching allocator
(pic_set_allocator): the handle's buffers show up in torch's allocated bytes
and go back to torch when the handle is destroyed, and the steps are the same
bits as those of a handle on cudaMalloc memory."""
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


@pytest.mark.parametrize("d,depth,scheme,precision", [(3, 3, pic.PIT, pic.FP32_SPLIT),
                                                      (2, 4, pic.PIDT, pic.FP64)])
def test_handle_on_torch_memory(d, depth, scheme, precision):
    flags = W.uniform_tree_flags(d, depth)
    n = 40_001
    x, v = W.random_particles(d, n, 11, vmax=0.5)
    kw = dict(scheme=scheme, precision=precision, q=-1.0 / n, qm=-1.0, ion=1.0, sweeps=5, omega=0.8)
    ref = pic.Pic(d, flags, x, v, stream=torch.cuda.Stream(), **kw)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    pic.use_torch_allocator(True)
    try:
        g = pic.Pic(d, flags, x, v, stream=torch.cuda.Stream(), **kw)
    finally:
        pic.use_torch_allocator(False)
    held = torch.cuda.memory_allocated() - before
    assert held >= g.info().device_bytes > 0
    assert g.info().brick == ref.info().brick
    for _ in range(3):
        ref.step(DT)
        g.step(DT)
    ref.sync()
    g.sync()
    for u, w in zip(ref.get_state(), g.get_state()):
        assert np.array_equal(u, w)
    for u, w in zip(ref.bins(), g.bins()):
        assert np.array_equal(u, w)
    assert np.array_equal(ref.field(), g.field())
    g.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before
