"""Thin Python binding of libpic's C ABI (include/pic.h).

Argument marshalling only: every step of the particle path runs in the CUDA
kernels of libpic.so.  Arrays are numpy (host memory) or torch CUDA tensors
(device memory; torch supplies the pointer and the stream).  There is no CPU
fallback: if libpic.so cannot be loaded, :func:`load` raises.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

PIT, PIDT = 0, 1
PERIODIC, REFLECT = 0, 1
PATH_AUTO, PATH_GENERIC = 0, 1
FP64, FP32_SPLIT = 0, 1
HOST, DEVICE = 0, 1

ERRORS = {0: "PIC_OK", -1: "PIC_EINVAL", -2: "PIC_ENOMEM", -3: "PIC_ERANGE", -4: "PIC_EHOOK",
          -5: "PIC_ETIMEOUT", -6: "PIC_ECUDA", -7: "PIC_ESTATE", -8: "PIC_EIO"}

_HERE = os.path.dirname(os.path.abspath(__file__))
_lock = threading.Lock()
_lib = None


class PicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class TreeDesc(C.Structure):
    _fields_ = [("d", C.c_int32), ("n_nodes", C.c_int64), ("flags", C.c_void_p)]


class ParticlesDesc(C.Structure):
    _fields_ = [("n", C.c_int64), ("x", C.c_void_p), ("v", C.c_void_p), ("where", C.c_int32)]


class Config(C.Structure):
    _fields_ = [("scheme", C.c_int32), ("precision", C.c_int32), ("q", C.c_double), ("qm", C.c_double),
                ("ion", C.c_double), ("sweeps", C.c_int32), ("omega", C.c_double),
                ("track_ids", C.c_int32), ("stream", C.c_void_p), ("path", C.c_int32)]


class Info(C.Structure):
    _fields_ = [("d", C.c_int32), ("scheme", C.c_int32), ("precision", C.c_int32), ("depth", C.c_int32),
                ("n_particles", C.c_int64), ("n_leaves", C.c_int64), ("n_vertices", C.c_int64),
                ("n_buckets", C.c_int64), ("n_keys", C.c_int64), ("uniform", C.c_int32),
                ("brick", C.c_int32), ("n_instances", C.c_int32), ("device_bytes", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("step", C.c_int64), ("movers", C.c_int64), ("max_bucket", C.c_int64),
                ("total_charge", C.c_double), ("residual", C.c_double), ("error", C.c_int32),
                ("tunnellers", C.c_int64)]


SOLVE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)

# (name, restype, argtypes) of every entry point declared in include/pic.h
SIGNATURES = [
    ("pic_create", C.c_int, [C.POINTER(C.c_void_p), C.POINTER(TreeDesc), C.POINTER(ParticlesDesc),
                             C.POINTER(Config)]),
    ("pic_destroy", None, [C.c_void_p]),
    ("pic_create_batch", C.c_int, [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(TreeDesc),
                                   C.POINTER(ParticlesDesc), C.c_void_p, C.POINTER(Config)]),
    ("pic_instances", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_strerror", C.c_char_p, [C.c_int]),
    ("pic_last_error", C.c_char_p, [C.c_void_p]),
    ("pic_info", C.c_int, [C.c_void_p, C.POINTER(Info)]),
    ("pic_init_leapfrog", C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    ("pic_step", C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    ("pic_step_fixed_field", C.c_int, [C.c_void_p, C.c_double]),
    ("pic_sync", C.c_int, [C.c_void_p]),
    ("pic_deposit", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_field", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_potential", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_bins", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_keys", C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_get_particles", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_get_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_set_state", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32]),
    ("pic_stats", C.c_int, [C.c_void_p, C.POINTER(Stats)]),
    ("pic_profile", C.c_int, [C.c_void_p, C.c_int32]),
    ("pic_graph_capture", C.c_int, [C.c_void_p, C.c_double]),
    ("pic_bucket_noalloc", C.c_int, [C.c_void_p, C.c_int64, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_stream_step", C.c_int, [C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_double, C.c_int32,
                                  C.c_void_p]),
    ("pic_tree_tabulate", C.c_int, [C.c_int32, C.c_void_p, C.c_int64, C.c_void_p] + [C.c_void_p] * 8),
    ("pic_graph_launch", C.c_int, [C.c_void_p, C.c_int32]),
    ("pic_graph_capture_step", C.c_int, [C.c_void_p, C.c_double]),
    ("pic_autotune", C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_void_p]),
    ("pic_set_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("pic_get_tuning", C.c_int, [C.c_void_p, C.c_void_p]),
    ("pic_phase_times", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_leaf_table", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_vertex_table", C.c_int, [C.c_void_p, C.c_void_p]),
    ("pic_pidt_table", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_grid_tables", C.c_int, [C.c_void_p, C.c_void_p] + [C.c_void_p] * 5),
    ("pic_retree", C.c_int, [C.c_void_p, C.POINTER(TreeDesc)]),
    ("pic_adapt", C.c_int, [C.c_void_p, C.c_int64, C.c_int32, C.c_int32]),
    ("pic_tree_flags", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_set_allocator", C.c_int, [ALLOC_FN, FREE_FN, C.c_void_p]),
    ("pic_count_lifts", C.c_int, [C.c_void_p, C.c_int32]),
    ("pic_lift_counts", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pic_save", C.c_int, [C.c_void_p, C.c_char_p]),
    ("pic_load", C.c_int, [C.POINTER(C.c_void_p), C.c_char_p, C.c_void_p]),
    ("pic_set_wait_limit", C.c_int, [C.c_void_p, C.c_int64]),
    ("pic_vmax", C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    ("pic_step_particles", C.c_int, [C.c_void_p, C.c_double, C.c_int32, C.c_int32]),
    ("pic_wait_selftest", C.c_int, [C.c_int64, C.c_void_p]),
]


def lib_path() -> str:
    return os.path.join(_HERE, "libpic.so")


def load(build_if_missing: bool = True):
    """Load libpic.so (building it in-tree first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if build_if_missing:
            from . import build as _build
            _build.build()
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libpic.so not found at {path}; run paper_1508_02435_gb300/build.py")
        lib = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _ptr(a):
    """(pointer, where) of a numpy array or a torch tensor."""
    if a is None:
        return None, HOST
    if isinstance(a, np.ndarray):
        assert a.flags.c_contiguous
        return a.ctypes.data_as(C.c_void_p), HOST
    if hasattr(a, "data_ptr"):
        assert a.is_contiguous()
        return C.c_void_p(a.data_ptr()), DEVICE if a.is_cuda else HOST
    raise TypeError(f"unsupported array type {type(a)}")


NOALLOC_MAX_KEYS = 1 << 20


class TreeSizes(C.Structure):
    _fields_ = [("d", C.c_int32), ("depth", C.c_int32), ("uniform", C.c_int32), ("reserved", C.c_int32),
                ("n_leaves", C.c_int64), ("n_vertices", C.c_int64), ("n_corner_entries", C.c_int64),
                ("n_pidt_vertices", C.c_int64)]


def tree_tables(d: int, flags) -> dict:
    """Host tabulation of a tree (pic_tree_tabulate; no GPU needed): vertex
    positions (d, n_vertices), PIDT owner levels and coordinates, and for
    non-uniform trees the vertex ion loads and stiffness diagonals and the
    leaf-corner expansions (ptr, vid, w)."""
    lib = load()
    fl = np.ascontiguousarray(flags, dtype=np.uint8)
    sz = TreeSizes()
    p = lambda a: C.c_void_p(a.ctypes.data) if a is not None else None  # noqa: E731
    rc = lib.pic_tree_tabulate(d, p(fl), len(fl), C.byref(sz), *([None] * 8))
    if rc != 0:
        raise PicError(rc, lib.pic_strerror(rc).decode())
    nv, npv, nlc = sz.n_vertices, sz.n_pidt_vertices, sz.n_leaves * (1 << d)
    out = {"uniform": bool(sz.uniform), "depth": int(sz.depth), "n_leaves": int(sz.n_leaves),
           "vertex_pos": np.zeros((d, nv), np.int64), "pidt_level": np.zeros(npv, np.int32),
           "pidt_j": np.zeros((npv, d), np.int64)}
    adaptive = not sz.uniform
    if adaptive:
        out.update(ion_load=np.zeros(nv), diag=np.zeros(nv), cexp_ptr=np.zeros(nlc + 1, np.int32),
                   cexp_vid=np.zeros(sz.n_corner_entries, np.int32), cexp_w=np.zeros(sz.n_corner_entries))
    g = lambda k: p(out[k]) if k in out else None  # noqa: E731
    rc = lib.pic_tree_tabulate(d, p(fl), len(fl), C.byref(sz), g("vertex_pos"), g("ion_load"), g("diag"),
                               g("cexp_ptr"), g("cexp_vid"), g("cexp_w"), g("pidt_level"), g("pidt_j"))
    if rc != 0:
        raise PicError(rc, lib.pic_strerror(rc).decode())
    return out


def _torch_alloc(user, nbytes, stream):
    try:
        import torch
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
    except Exception:  # out of memory or no CUDA: the library reports PIC_ENOMEM
        return None


def _torch_free(user, ptr, nbytes, stream):
    try:
        import torch
        torch.cuda.caching_allocator_delete(int(ptr))
    except Exception:  # interpreter shutdown
        pass


# the callbacks must outlive every handle created while they are set
_TORCH_CALLBACKS = (ALLOC_FN(_torch_alloc), FREE_FN(_torch_free))


def use_torch_allocator(enable: bool = True):
    """Take the device memory of handles created from now on from PyTorch's
    caching allocator (pic_set_allocator); False restores cudaMalloc.  Handles
    keep the allocator they were created with."""
    lib = load()
    if enable:
        rc = lib.pic_set_allocator(_TORCH_CALLBACKS[0], _TORCH_CALLBACKS[1], None)
    else:
        rc = lib.pic_set_allocator(ALLOC_FN(), FREE_FN(), None)
    if rc != 0:
        raise PicError(rc, lib.pic_strerror(rc).decode())


def stream_step(x, v, dt: float, steps: int = 1, stream=None):
    """Stream-like calibration update (pic_stream_step): `steps` passes of
    x += v dt with reflection at the unit-box walls, in place on the device
    tensors x[d][n], v[d][n] (float32 or float64).  Queued on `stream`."""
    lib = load()
    d, n = int(x.shape[0]), int(x.shape[1])
    prec = FP64 if str(x.dtype) == "torch.float64" else FP32_SPLIT
    st = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    rc = lib.pic_stream_step(d, prec, C.c_void_p(x.data_ptr()), C.c_void_p(v.data_ptr()), n, float(dt), int(steps),
                             C.c_void_p(st))
    if rc != 0:
        raise PicError(rc, lib.pic_strerror(rc).decode())


def wait_selftest(cycles: int, stream=None) -> int:
    """Run the bounded-wait self-test kernel (pic_wait_selftest); returns the
    library's code: PIC_ETIMEOUT (-5) when the wait gave up as designed."""
    st = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    return int(load().pic_wait_selftest(int(cycles), C.c_void_p(st)))


def bucket_noalloc(keys, n_keys: int, start, perm, stream=None):
    """Stable bucket sort of device int32 `keys` into the caller's device
    tensors start[n_keys + 1] and perm[len(keys)], with no device allocation
    inside the library (pic_bucket_noalloc).  Queued on `stream`."""
    lib = load()
    n = int(keys.numel())
    if n_keys > NOALLOC_MAX_KEYS:
        raise PicError(-1, f"n_keys = {n_keys} is above the fixed scratch of {NOALLOC_MAX_KEYS} buckets")
    # the kernels write start[0..n_keys] and perm[0..n) through raw pointers:
    # check every tensor before anything is launched
    import torch
    for name, t in (("keys", keys), ("start", start), ("perm", perm)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.int32 or not t.is_cuda or not t.is_contiguous():
            raise PicError(-1, f"{name} must be a contiguous int32 CUDA tensor")
        if t.device != keys.device:
            raise PicError(-1, f"{name} is on {t.device}, keys on {keys.device}")
    if keys.device.index != torch.cuda.current_device():
        raise PicError(-1, f"keys are on {keys.device}, the current device is cuda:{torch.cuda.current_device()}")
    if start.numel() < n_keys + 1:
        raise PicError(-1, f"start holds {start.numel()} entries, n_keys + 1 = {n_keys + 1} needed")
    if perm.numel() < n:
        raise PicError(-1, f"perm holds {perm.numel()} entries, len(keys) = {n} needed")
    st = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
    rc = lib.pic_bucket_noalloc(C.c_void_p(keys.data_ptr()), n, int(n_keys), C.c_void_p(start.data_ptr()),
                                C.c_void_p(perm.data_ptr()), C.c_void_p(st))
    if rc != 0:
        raise PicError(rc, lib.pic_strerror(rc).decode())


class Pic:
    """One plasma instance on the GPU (a libpic handle)."""

    def __init__(self, d: int, flags: np.ndarray, x, v, *, scheme: int = PIT, precision: int = FP64,
                 q: float = -1.0, qm: float = -1.0, ion: float = 1.0, sweeps: int = 100,
                 omega: float = 0.8, track_ids: bool = True, stream=None, path: int = PATH_AUTO):
        self.lib = load()
        self.d = d
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        self._flags = flags
        tree = TreeDesc(d, len(flags), flags.ctypes.data_as(C.c_void_p))
        if isinstance(x, np.ndarray):
            x = np.ascontiguousarray(x, dtype=np.float64)
            v = np.ascontiguousarray(v, dtype=np.float64)
        xp, where = _ptr(x)
        vp, _ = _ptr(v)
        n = int(x.shape[1]) if x.ndim == 2 else 0
        parts = ParticlesDesc(n, xp, vp, where)
        st = C.c_void_p(stream.cuda_stream) if stream is not None and hasattr(stream, "cuda_stream") else \
            C.c_void_p(stream)
        self.cfg = Config(scheme, precision, q, qm, ion, sweeps, omega, 1 if track_ids else 0, st, path)
        self._stream = stream  # the handle launches on it: keep it alive
        h = C.c_void_p()
        rc = self.lib.pic_create(C.byref(h), C.byref(tree), C.byref(parts), C.byref(self.cfg))
        if rc != 0:
            raise PicError(rc, self.lib.pic_strerror(rc).decode())
        self.h = h
        self.n = n
        self.scheme = scheme
        self.precision = precision
        self._info = self.info()

    @classmethod
    def batch(cls, d: int, flags_list, xs, vs, qs=None, *, scheme: int = PIT, precision: int = FP64,
              q: float = -1.0, qm: float = -1.0, ion: float = 1.0, sweeps: int = 100, omega: float = 0.8,
              track_ids: bool = True, stream=None, path: int = PATH_AUTO) -> "Pic":
        """Several independent plasmas (uniform trees) in one handle."""
        self = cls.__new__(cls)
        self.lib = load()
        self.d = d
        n_inst = len(flags_list)
        self._keep = []
        trees = (TreeDesc * n_inst)()
        parts = (ParticlesDesc * n_inst)()
        for i in range(n_inst):
            f = np.ascontiguousarray(flags_list[i], dtype=np.uint8)
            x = xs[i]
            v = vs[i]
            if isinstance(x, np.ndarray):
                x = np.ascontiguousarray(x, dtype=np.float64)
                v = np.ascontiguousarray(v, dtype=np.float64)
            self._keep += [f, x, v]
            trees[i] = TreeDesc(d, len(f), f.ctypes.data_as(C.c_void_p))
            xp, where = _ptr(x)
            vp, _ = _ptr(v)
            parts[i] = ParticlesDesc(int(x.shape[1]), xp, vp, where)
        qarr = None
        if qs is not None:
            qarr = np.ascontiguousarray(qs, dtype=np.float64)
            self._keep.append(qarr)
        st = C.c_void_p(stream.cuda_stream) if stream is not None and hasattr(stream, "cuda_stream") else \
            C.c_void_p(stream)
        self.cfg = Config(scheme, precision, q, qm, ion, sweeps, omega, 1 if track_ids else 0, st, path)
        self._stream = stream
        h = C.c_void_p()
        rc = self.lib.pic_create_batch(C.byref(h), n_inst, trees, parts,
                                       None if qarr is None else qarr.ctypes.data_as(C.c_void_p),
                                       C.byref(self.cfg))
        if rc != 0:
            raise PicError(rc, self.lib.pic_strerror(rc).decode())
        self.h = h
        self.n = sum(int(p.n) for p in parts)
        self.scheme = scheme
        self.precision = precision
        self._info = self.info()
        return self

    @classmethod
    def load(cls, path, stream=None) -> "Pic":
        """A handle restored from a checkpoint file written by :meth:`save`
        (pic_load), launching on `stream`."""
        self = cls.__new__(cls)
        self.lib = load()
        st = stream.cuda_stream if stream is not None and hasattr(stream, "cuda_stream") else stream
        self._stream = stream
        h = C.c_void_p()
        rc = self.lib.pic_load(C.byref(h), os.fsencode(path), C.c_void_p(st))
        if rc != 0:
            raise PicError(rc, self.lib.pic_last_error(None).decode())
        self.h = h
        info = self.info()
        self.d = int(info.d)
        self.n = int(info.n_particles)
        self.scheme = int(info.scheme)
        self.precision = int(info.precision)
        self._info = info
        self._flags = self.tree_flags()
        return self

    def save(self, path):
        """Write a checkpoint of the handle to `path` (pic_save)."""
        self._check(self.lib.pic_save(self.h, os.fsencode(path)))

    def instances(self):
        """(particle_start, vertex_start, bucket_start), each n_instances + 1 long."""
        ni = int(self._info.n_instances)
        ps = np.zeros(ni + 1, np.int64)
        vs = np.zeros(ni + 1, np.int64)
        bs = np.zeros(ni + 1, np.int64)
        self._check(self.lib.pic_instances(self.h, _ptr(ps)[0], _ptr(vs)[0], _ptr(bs)[0]))
        return ps, vs, bs

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            self.lib.pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc != 0:
            raise PicError(rc, self.lib.pic_last_error(self.h).decode())

    # ---- calls ---------------------------------------------------------
    def info(self) -> Info:
        out = Info()
        self._check(self.lib.pic_info(self.h, C.byref(out)))
        return out

    def init_leapfrog(self, dt: float, hook=None, user=None):
        self._check(self.lib.pic_init_leapfrog(self.h, dt, hook, user))

    def step(self, dt: float, hook=None, user=None):
        self._check(self.lib.pic_step(self.h, dt, hook, user))

    def step_particles(self, dt: float, reflect: bool = True, flops: int = 0):
        """The particle-handling step of the paper's experiments: move by
        v dt (no field), reflecting or periodic walls, flops per move,
        re-bin (pic_step_particles)."""
        self._check(self.lib.pic_step_particles(self.h, dt, 1 if reflect else 0, int(flops)))

    def step_fixed_field(self, dt: float):
        self._check(self.lib.pic_step_fixed_field(self.h, dt))

    def sync(self):
        self._check(self.lib.pic_sync(self.h))

    def vmax(self, dt: float = 0.0):
        """(v_max per tree node in level order, nodes closed for a step of dt)
        -- the raPIDT tree attribute (pic_vmax)."""
        nn = C.c_int64(0)
        self._check(self.lib.pic_tree_flags(self.h, None, C.byref(nn)))
        out = np.zeros(nn.value)
        closed = C.c_int64(0)
        self._check(self.lib.pic_vmax(self.h, _ptr(out)[0], float(dt), C.byref(closed)))
        return out, closed.value

    def set_wait_limit(self, cycles: int):
        """Limit (SM clocks) of the bounded device waits of later steps."""
        self._check(self.lib.pic_set_wait_limit(self.h, int(cycles)))

    def count_lifts(self, enable: bool = True):
        """Start (from zero) or stop counting the lifts, drops and tunnellers
        of every step (pic_count_lifts; handles with tracked ids)."""
        self._check(self.lib.pic_count_lifts(self.h, 1 if enable else 0))

    def lift_counts(self):
        """(lifts, drops, tunnellers, steps) since counting started
        (pic_lift_counts)."""
        lifts, drops, tun, steps = C.c_int64(0), C.c_int64(0), C.c_int64(0), C.c_int64(0)
        self._check(self.lib.pic_lift_counts(self.h, C.byref(lifts), C.byref(drops), C.byref(tun),
                                             C.byref(steps)))
        return lifts.value, drops.value, tun.value, steps.value

    def stats(self) -> Stats:
        out = Stats()
        self._check(self.lib.pic_stats(self.h, C.byref(out)))
        return out

    @property
    def n_vertices(self) -> int:
        return int(self._info.n_vertices)

    @property
    def n_buckets(self) -> int:
        return int(self._info.n_buckets)

    def deposit(self, out=None):
        out = np.zeros(self.n_vertices) if out is None else out
        p, w = _ptr(out)
        self._check(self.lib.pic_deposit(self.h, p, w))
        return out

    def field(self, out=None):
        out = np.zeros((self.d, self.n_vertices)) if out is None else out
        p, w = _ptr(out)
        self._check(self.lib.pic_field(self.h, p, w))
        return out

    def potential(self, out=None):
        out = np.zeros(self.n_vertices) if out is None else out
        p, w = _ptr(out)
        self._check(self.lib.pic_potential(self.h, p, w))
        return out

    def bins(self, with_ids: bool = True):
        start = np.zeros(self.n_buckets + 1, np.int64)
        perm = np.zeros(self.n, np.int32) if with_ids else None
        sp, _ = _ptr(start)
        pp, _ = _ptr(perm)
        self._check(self.lib.pic_bins(self.h, sp, pp, HOST))
        return start, perm

    def keys(self):
        out = np.zeros(self.n, np.int32)
        p, w = _ptr(out)
        self._check(self.lib.pic_keys(self.h, p, w))
        return out

    def particles(self):
        x = np.zeros((self.d, self.n))
        v = np.zeros((self.d, self.n))
        self._check(self.lib.pic_get_particles(self.h, _ptr(x)[0], _ptr(v)[0], HOST))
        return x, v

    def get_state(self, leaf=None, pos=None, vel=None):
        """Native state in storage order into the given arrays (numpy or CUDA
        tensors); allocates numpy arrays when none are given."""
        if pos is None:
            dt = np.float32 if self.precision == FP32_SPLIT else np.float64
            leaf = np.zeros(self.n, np.int32)
            pos = np.zeros((self.d, self.n), dt)
            vel = np.zeros((self.d, self.n), dt)
        lp, w = _ptr(leaf)
        pp, w2 = _ptr(pos)
        vp, _ = _ptr(vel)
        self._check(self.lib.pic_get_state(self.h, lp, pp, vp, w2))
        return leaf, pos, vel

    def set_state(self, leaf, pos, vel):
        lp, _ = _ptr(leaf)
        pp, w = _ptr(pos)
        vp, _ = _ptr(vel)
        self._check(self.lib.pic_set_state(self.h, lp, pp, vp, w))

    PHASES = ("deposit", "solve", "push", "rebin", "permute")

    def graph_capture(self, dt: float):
        self._check(self.lib.pic_graph_capture(self.h, dt))

    def graph_capture_step(self, dt: float):
        """Capture the whole step with the built-in solve (pic_graph_capture_step)."""
        self._check(self.lib.pic_graph_capture_step(self.h, dt))

    def graph_launch(self, steps: int):
        self._check(self.lib.pic_graph_launch(self.h, steps))

    def tuning(self):
        out = np.zeros(4, np.int32)
        self._check(self.lib.pic_get_tuning(self.h, _ptr(out)[0]))
        return [int(x) for x in out]

    def set_tuning(self, tuned):
        arr = np.ascontiguousarray(tuned, dtype=np.int32)
        self._check(self.lib.pic_set_tuning(self.h, _ptr(arr)[0]))

    def autotune(self, dt: float, trials: int = 3, cache: str | None = None):
        """Pick the path and block shapes by timing them on this handle's own
        particles (state restored afterwards).  With `cache`, results are kept
        in that JSON file keyed by the workload's shape."""
        import json
        info = self.info()
        key = json.dumps([int(info.d), int(info.depth), int(info.n_instances), int(info.n_particles),
                          int(info.scheme), int(info.precision), int(info.uniform)])
        store = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
        if key in store:
            self.set_tuning(store[key])
            return store[key]
        out = np.zeros(4, np.int32)
        self._check(self.lib.pic_autotune(self.h, dt, trials, _ptr(out)[0]))
        tuned = [int(x) for x in out]
        if cache:
            store[key] = tuned
            tmp = cache + f".tmp{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(store, f, indent=1)
            os.replace(tmp, cache)
        return tuned

    def profile(self, enable: bool = True):
        self._check(self.lib.pic_profile(self.h, 1 if enable else 0))

    def phase_times(self):
        """{phase: (device ms, kernels launched)} since profile(True)."""
        ms = np.zeros(5)
        k = np.zeros(5, np.int64)
        self._check(self.lib.pic_phase_times(self.h, _ptr(ms)[0], _ptr(k)[0]))
        return {name: (float(ms[i]), int(k[i])) for i, name in enumerate(self.PHASES)}

    def leaf_table(self):
        nl = int(self._info.n_leaves)
        lev = np.zeros(nl, np.int32)
        co = np.zeros((nl, self.d), np.int64)
        self._check(self.lib.pic_leaf_table(self.h, _ptr(lev)[0], _ptr(co)[0]))
        return lev, co

    def vertex_table(self):
        pos = np.zeros((self.d, self.n_vertices), np.int64)
        self._check(self.lib.pic_vertex_table(self.h, _ptr(pos)[0]))
        return pos

    def pidt_table(self):
        if self.scheme != PIDT:
            raise ValueError("PIDT owner vertices exist only for the PIDT scheme")
        nb = self.n_buckets
        lev = np.zeros(nb, np.int32)
        j = np.zeros((nb, self.d), np.int64)
        self._check(self.lib.pic_pidt_table(self.h, _ptr(lev)[0], _ptr(j)[0]))
        return lev, j

    def grid_tables(self) -> dict:
        """The finite-element tables the kernels read (adaptive single-instance
        handles): cexp_ptr, cexp_vid, cexp_w, ion_load, diag (pic_grid_tables)."""
        nnz = C.c_int64(0)
        self._check(self.lib.pic_grid_tables(self.h, C.byref(nnz), None, None, None, None, None))
        nlc = int(self._info.n_leaves) * (1 << self.d)
        out = {"cexp_ptr": np.zeros(nlc + 1, np.int32), "cexp_vid": np.zeros(nnz.value, np.int32),
               "cexp_w": np.zeros(nnz.value), "ion_load": np.zeros(self.n_vertices), "diag": np.zeros(self.n_vertices)}
        self._check(self.lib.pic_grid_tables(self.h, None, *(_ptr(out[k])[0] for k in
                                                             ("cexp_ptr", "cexp_vid", "cexp_w", "ion_load", "diag"))))
        return out

    def retree(self, flags):
        flags = np.ascontiguousarray(flags, dtype=np.uint8)
        tree = TreeDesc(self.d, len(flags), flags.ctypes.data_as(C.c_void_p))
        self._check(self.lib.pic_retree(self.h, C.byref(tree)))
        self._flags = flags
        self._info = self.info()

    def tree_flags(self) -> np.ndarray:
        nn = C.c_int64(0)
        self._check(self.lib.pic_tree_flags(self.h, None, C.byref(nn)))
        out = np.zeros(nn.value, np.uint8)
        self._check(self.lib.pic_tree_flags(self.h, _ptr(out)[0], None))
        return out

    def adapt(self, ppc: int, dmin: int, dmax: int):
        self._check(self.lib.pic_adapt(self.h, ppc, dmin, dmax))
        self._info = self.info()
