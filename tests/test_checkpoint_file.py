"""CPU-only checks of the checkpoint format read by pic_load.

Files are written here by a writer of the layout documented in include/pic.h,
independent of the library's own writer.  Every file below is rejected on the
host before the first device call, so no GPU is needed: a missing, foreign,
truncated or corrupted file gives PIC_EIO; a well-formed file whose checksum
matches but whose trees or particle values are out of range gives PIC_EINVAL.
Reaching PIC_EINVAL also shows that the library folds the checksum exactly as
documented, since the writer here computes it from that description."""
from __future__ import annotations

import struct

import numpy as np
import pytest

from paper_1508_02435_gb300 import pic
from paper_1508_02435_gb300 import workloads as W

EIO, EINVAL = -8, -1
MASK = (1 << 64) - 1


def fold(c: int, data: bytes) -> int:
    data = data + b"\0" * (-len(data) % 8)
    for (w,) in struct.iter_unpack("<Q", data):
        c = ((c ^ w) * 0x9E3779B97F4A7C15) & MASK
        c ^= c >> 29
    return c


def pad(b: bytes) -> bytes:
    return b + b"\0" * (-len(b) % 8)


def checkpoint(split=True, d=2, depth=2, n=40, seed=0, version=1, track_ids=1, **edit) -> dict:
    """Fields of a small, valid checkpoint (split or FP64, one instance)."""
    rng = np.random.default_rng(seed)
    flags = W.uniform_tree_flags(d, depth)
    n_leaves = 3 ** (d * depth)
    n_vert = 3 ** (d * depth)  # periodic uniform tree: one vertex per leaf
    ft = np.float32 if split else np.float64
    f = dict(version=version, d=d, scheme=pic.PIT, precision=pic.FP32_SPLIT if split else pic.FP64,
             sweeps=5, track_ids=track_ids, path=0, n_inst=1, reserved=0, q=-1.0 / n, qm=-1.0, ion=1.0,
             omega=0.8, step=7, n=n, n_vert=n_vert, tuned=[1 if split else 0, 256, 256, 256],
             inst=[(len(flags), n, -1.0 / n)], flags=flags.astype(np.uint8),
             leaf=np.sort(rng.integers(0, n_leaves, n)).astype(np.int32) if split else None,
             pos=rng.random((d, n)).astype(ft), vel=(0.1 * rng.standard_normal((d, n))).astype(ft),
             ids=rng.permutation(n).astype(np.int32) if track_ids else None,
             V=rng.standard_normal(n_vert).astype(ft), E=rng.standard_normal((d, n_vert)).astype(ft))
    f.update(edit)
    return f


def encode(f: dict, corrupt=None) -> bytes:
    meta = struct.pack("<8i", f["d"], f["scheme"], f["precision"], f["sweeps"], f["track_ids"], f["path"],
                       f["n_inst"], f["reserved"])
    meta += struct.pack("<4d", f["q"], f["qm"], f["ion"], f["omega"])
    meta += struct.pack("<3q", f["step"], f["n"], f["n_vert"])
    meta += struct.pack("<4i", *f["tuned"])
    for nf, ni, qi in f["inst"]:
        meta += struct.pack("<qqd", nf, ni, qi)
    body = pad(meta) + pad(f["flags"].tobytes())
    if f["leaf"] is not None:
        body += pad(f["leaf"].tobytes())
    body += pad(f["pos"].tobytes()) + pad(f["vel"].tobytes())
    if f["ids"] is not None:
        body += pad(f["ids"].tobytes())
    body += pad(f["V"].tobytes()) + pad(f["E"].tobytes())
    if corrupt is not None:
        body = corrupt(body)
    head = b"PICSNAP\0" + struct.pack("<II", f["version"], len(meta)) + struct.pack("<Q", fold(0x243F6A8885A308D3,
                                                                                          body))
    return head + body


def load_error(path):
    with pytest.raises(pic.PicError) as e:
        pic.Pic.load(str(path))
    return e.value.code, str(e.value)


def write(tmp_path, data: bytes, name="c.ckpt"):
    p = tmp_path / name
    p.write_bytes(data)
    return p


def test_fold_matches_its_definition_on_a_worked_example():
    # one word 1: c = (seed ^ 1) * K mod 2^64, then c ^= c >> 29
    seed, k = 0x243F6A8885A308D3, 0x9E3779B97F4A7C15
    c = ((seed ^ 1) * k) % (1 << 64)
    c ^= c >> 29
    assert fold(seed, struct.pack("<Q", 1)) == c
    # a tail shorter than a word is zero-padded
    assert fold(seed, b"\x01") == c


def test_missing_file(tmp_path):
    code, msg = load_error(tmp_path / "absent.ckpt")
    assert code == EIO and "cannot open" in msg


def test_not_a_checkpoint(tmp_path):
    code, msg = load_error(write(tmp_path, bytes(range(256))))
    assert code == EIO and "magic" in msg


def test_empty_file(tmp_path):
    code, _ = load_error(write(tmp_path, b""))
    assert code == EIO


def test_other_format_version(tmp_path):
    code, msg = load_error(write(tmp_path, encode(checkpoint(version=2))))
    assert code == EIO and "version" in msg


@pytest.mark.parametrize("cut", [8, 1, 200])
def test_truncated_file(tmp_path, cut):
    data = encode(checkpoint(leaf=np.full(40, 10**6, np.int32)))  # complete, it would be EINVAL
    code, msg = load_error(write(tmp_path, data[:-cut]))
    assert code == EIO and "size" in msg


def test_appended_bytes(tmp_path):
    data = encode(checkpoint(leaf=np.full(40, 10**6, np.int32)))
    code, _ = load_error(write(tmp_path, data + b"\0" * 8))
    assert code == EIO


@pytest.mark.parametrize("at", [200, -9, -1])
def test_flipped_byte_fails_the_checksum(tmp_path, at):
    f = checkpoint(leaf=np.full(40, 10**6, np.int32))
    data = bytearray(encode(f))
    data[at] ^= 0x10
    code, msg = load_error(write(tmp_path, bytes(data)))
    assert code == EIO and "checksum" in msg


def test_nonzero_padding(tmp_path):
    # 40 particles x 4 bytes of leaf ids fill whole words; 3 uint8 flags need padding
    f = checkpoint(flags=np.array([0], np.uint8), inst=[(1, 40, -1.0 / 40)])

    def poke(body):
        meta_len = 104 + 24
        b = bytearray(body)
        b[meta_len + 1] = 1  # second byte of the flags section is padding
        return bytes(b)

    code, _ = load_error(write(tmp_path, encode(f, corrupt=poke)))
    assert code == EIO


@pytest.mark.parametrize("edit", [dict(d=4), dict(scheme=2), dict(precision=3), dict(sweeps=-1),
                                  dict(track_ids=2), dict(path=5), dict(reserved=1), dict(step=-1),
                                  dict(n_vert=0), dict(tuned=[2, 256, 256, 256]),
                                  dict(tuned=[1, 100, 256, 256])])
def test_meta_data_of_no_valid_configuration(tmp_path, edit):
    code, msg = load_error(write(tmp_path, encode(checkpoint(**edit))))
    assert code == EIO and "meta" in msg


def test_instance_counts_must_add_up(tmp_path):
    f = checkpoint()
    f["inst"] = [(f["inst"][0][0], 39, f["inst"][0][2])]
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EIO and "add up" in msg


def test_offset_outside_the_cell(tmp_path):
    f = checkpoint()
    f["pos"][1, 5] = np.float32(1.0)
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL and "offset" in msg


def test_nan_offset(tmp_path):
    f = checkpoint()
    f["pos"][0, 0] = np.float32("nan")
    code, _ = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL


def test_fp64_position_outside_the_box(tmp_path):
    f = checkpoint(split=False)
    f["pos"][0, 3] = -0.25
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL and "position" in msg


@pytest.mark.parametrize("split", [True, False])
def test_non_finite_velocity(tmp_path, split):
    f = checkpoint(split=split)
    f["vel"][1, 2] = np.inf
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL and "velocity" in msg


def test_ids_must_be_a_permutation(tmp_path):
    f = checkpoint()
    f["ids"][3] = f["ids"][4]
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL and "permutation" in msg


def test_leaf_outside_the_tree(tmp_path):
    f = checkpoint()
    f["leaf"][-1] = 81  # the depth-2 2D tree has leaves 0..80
    code, msg = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL and "leaf" in msg


def test_malformed_tree(tmp_path):
    # a refined root without its nine children
    f = checkpoint(flags=np.array([1, 0, 0], np.uint8), inst=[(3, 40, -1.0 / 40)])
    code, _ = load_error(write(tmp_path, encode(f)))
    assert code == EINVAL


def test_last_error_of_no_handle_names_the_file(tmp_path):
    p = tmp_path / "absent.ckpt"
    lib = pic.load()
    h = pic.C.c_void_p()
    rc = lib.pic_load(pic.C.byref(h), str(p).encode(), None)
    assert rc == EIO and h.value is None
    assert str(p) in lib.pic_last_error(None).decode()
    assert b"corrupt" in lib.pic_strerror(EIO)
