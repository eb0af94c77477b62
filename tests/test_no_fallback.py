"""The product has no CPU fallback: the binding raises when libpic.so cannot
be loaded, nothing in the package imports the oracle, and on a host without a
CUDA device creating a handle fails with a CUDA error instead of computing
anywhere else."""
from __future__ import annotations

import glob
import os

import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

PKG = os.path.dirname(os.path.abspath(pic.__file__))


def test_binding_raises_without_the_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pic, "_lib", None)
    monkeypatch.setattr(pic, "lib_path", lambda: str(tmp_path / "libpic.so"))
    with pytest.raises(RuntimeError):
        pic.load(build_if_missing=False)


def test_package_never_imports_the_oracle():
    for path in glob.glob(os.path.join(PKG, "*.py")):
        text = open(path).read()
        assert "import oracle" not in text and "from oracle" not in text, path


def test_no_handle_without_a_cuda_device():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    x, v = W.random_particles(2, 100, 0)
    with pytest.raises(pic.PicError) as e:
        pic.Pic(2, W.uniform_tree_flags(2, 2), x, v)
    assert e.value.code == -6  # PIC_ECUDA
