"""CPU-only checks of the C-ABI boundary: the library builds, loads and exports
every entry point that include/pic.h declares, and the Python binding binds
each of them.  No compute call is made (no GPU here)."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from paper_1508_02435_gb300 import pic

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "pic.h")).read()
    return sorted(set(re.findall(r"PIC_API[^;]*?\b(pic_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pic_create", "pic_step", "pic_deposit", "pic_bins", "pic_destroy"):
        assert required in names


def test_library_loads_and_exports_every_declared_symbol():
    lib = pic.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
        assert ctypes.cast(getattr(lib, name), ctypes.c_void_p).value


def test_binding_covers_every_declared_symbol():
    bound = {name for name, _, _ in pic.SIGNATURES}
    assert bound == set(declared_symbols())


def test_strerror_is_host_only():
    lib = pic.load()
    assert lib.pic_strerror(0) == b"ok"
    assert b"malformed" in lib.pic_strerror(-1)


def test_set_allocator_takes_both_callbacks_or_neither():
    lib = pic.load()
    alloc, free = pic._TORCH_CALLBACKS
    try:
        assert lib.pic_set_allocator(alloc, pic.FREE_FN(), None) == -1
        assert lib.pic_set_allocator(pic.ALLOC_FN(), free, None) == -1
        pic.use_torch_allocator(True)
    finally:
        pic.use_torch_allocator(False)
    assert lib.pic_set_allocator(pic.ALLOC_FN(), pic.FREE_FN(), None) == 0


def test_bucket_noalloc_checks_tensors_on_the_host():
    """Host tensors, a wrong dtype or short outputs are refused by the binding
    before the library is called (no device needed)."""
    torch = pytest.importorskip("torch")
    keys = torch.zeros(10, dtype=torch.int32)
    start = torch.zeros(5, dtype=torch.int32)
    perm = torch.zeros(10, dtype=torch.int32)
    for k, s, p in ((keys, start, perm), (keys.to(torch.int64), start, perm), (keys, start[:2], perm)):
        with pytest.raises(pic.PicError) as e:
            pic.bucket_noalloc(k, 4, s, p)
        assert e.value.code == -1
