"""Python binding of the FliX C ABI (include/flix.h): argument marshalling only.

PyTorch provides device memory and streams; every step of every operation runs in libflix.so's
CUDA kernels.  There is no fallback: if the library cannot be loaded, or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

OP_NOP, OP_LOOKUP, OP_SUCC, OP_RANGE, OP_INSERT, OP_DELETE, OP_PRED = 0, 1, 2, 3, 4, 5, 6
KEY_U32, KEY_U64 = 0, 1

_STATUS = {0: "FLIX_OK", -1: "FLIX_EINVAL", -2: "FLIX_ENOMEM", -3: "FLIX_ECUDA", -4: "FLIX_ETYPE",
           -5: "FLIX_ETIMEDOUT", -6: "FLIX_EINTERNAL", -7: "FLIX_ENOTIMPL"}


class FlixError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__("%s failed: %s (%d)%s" % (where, _STATUS.get(code, "?"), code,
                                                  (": " + detail) if detail else ""))


class Config(ctypes.Structure):
    _fields_ = [("key_type", ctypes.c_int), ("node_size", ctypes.c_uint32), ("fill_pct", ctypes.c_uint32),
                ("grow", ctypes.c_uint32), ("pool_nodes", ctypes.c_uint64), ("sort_digit_bits", ctypes.c_uint32),
                ("sort_variant", ctypes.c_uint32), ("restructure_in_one_pass", ctypes.c_uint32),
                ("split_chains_over", ctypes.c_uint32), ("merge_underfull", ctypes.c_uint32),
                ("bucket_threads", ctypes.c_uint32), ("reserved", ctypes.c_uint32 * 2), ("dev_alloc", ctypes.c_void_p), ("dev_free", ctypes.c_void_p),
                ("alloc_ctx", ctypes.c_void_p)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


def _torch_allocator(device):
    """Device allocator callbacks backed by PyTorch's caching allocator (the library synchronises
    the device before it frees)."""
    def alloc(nbytes, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(nbytes, device)
        except RuntimeError:   # out of memory: the library reports FLIX_ECUDA / FLIX_ENOMEM
            return None

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return _ALLOC_FN(alloc), _FREE_FN(free)


class Batch(ctypes.Structure):
    """flix_batch: one batch of a persistent queue (device pointers)."""
    _fields_ = [("ops", ctypes.c_void_p), ("keys", ctypes.c_void_p), ("aux", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("keys_out", ctypes.c_void_p), ("vals_out", ctypes.c_void_p), ("found", ctypes.c_void_p),
                ("range_off", ctypes.c_void_p), ("range_keys", ctypes.c_void_p), ("range_vals", ctypes.c_void_p),
                ("range_cap", ctypes.c_uint64), ("status", ctypes.c_void_p), ("ready", ctypes.c_void_p)]


QUEUE_BATCH_MAX = 2048


class Stats(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in ("buckets", "nodes_used", "nodes_free", "pool_nodes", "live_keys",
                                               "max_chain", "node_bytes", "used_bytes", "reserved_bytes")]


_lib = None

# every function the header declares, with its ctypes signature
_VP, _U64, _U32, _INT = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
SIGNATURES = {
    "flix_config_default": (None, [_VP, _INT]),
    "flix_create": (_INT, [_VP, _VP]),
    "flix_destroy": (_INT, [_VP]),
    "flix_bulk_load": (_INT, [_VP, _VP, _VP, _U64, _VP]),
    "flix_lookup": (_INT, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "flix_lookup_noalloc": (_INT, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "flix_successor": (_INT, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "flix_predecessor": (_INT, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "flix_range": (_INT, [_VP, _VP, _VP, _U64, _VP, _VP, _VP, _U64, _VP, _VP]),
    "flix_insert": (_INT, [_VP, _VP, _VP, _U64, _VP]),
    "flix_delete": (_INT, [_VP, _VP, _U64, _VP]),
    "flix_apply": (_INT, [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP, _VP, _U64, _VP, _VP]),
    "flix_apply_async": (_INT, [_VP, _VP, _VP, _VP, _U64, _VP, _VP, _VP, _VP, _VP, _VP, _U64, _VP, _VP]),
    "flix_reserve": (_INT, [_VP, _U64, _U64, _VP]),
    "flix_restructure": (_INT, [_VP, _VP]),
    "flix_split_chains": (_INT, [_VP, ctypes.c_uint32, _VP, _VP]),
    "flix_merge_underfull": (_INT, [_VP, _VP, _VP]),
    "flix_stats": (_INT, [_VP, _VP, _VP]),
    "flix_export": (_INT, [_VP, _VP, _VP, _U64, _VP, _VP]),
    "flix_dump_layout": (_INT, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "flix_sort_pairs": (_INT, [_VP, _VP, _U64, _VP, _VP, _VP]),
    "flix_apply_queue": (_INT, [_VP, _VP, _U32, _U32, _VP, _VP]),
    "flix_profile_enable": (_INT, [_VP, _INT]),
    "flix_profile_reset": (_INT, [_VP]),
    "flix_profile_read": (_INT, [_VP, _U32, _VP, _VP, _VP, _VP, _VP]),
    "flix_launch_count": (_U64, [_VP]),
    "flix_strerror": (ctypes.c_char_p, [_INT]),
    "flix_last_error": (ctypes.c_char_p, [_VP]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libflix.so (building it with nvcc if needed).  Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError("libflix.so is missing (%s); build it with paper_2604_16725_gb300.build" % path)
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(code: int, where: str, h=None):
    if code != 0:
        detail = load().flix_last_error(h).decode() if h else ""
        raise FlixError(code, where, detail)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Index:
    """A FliX ordered map on one GPU (uint32 or uint64 keys with values of the same width).

    Tensors are taken as raw words: key and value tensors may be int32/uint32 (32-bit index) or
    int64/uint64 (64-bit index); numpy arrays are copied to the device first.
    """

    def __init__(self, key_bits: int = 64, node_size: int | None = None, fill_pct: int = 50,
                 pool_nodes: int = 0, grow: bool = True, device=None, sort_variant: int = 0,
                 restructure_in_one_pass: bool = True, split_chains_over: int = 0,
                 merge_underfull: bool = False, allocator: str | None = None, bucket_threads: int = 0):
        """allocator: None (cudaMalloc) or "torch" (every device buffer of the index comes from
        PyTorch's caching allocator and counts in torch.cuda.memory_allocated).  bucket_threads: 0 (one
        thread for a light one-node bucket, a warp otherwise) or 32 (a warp for every bucket)."""
        if not torch.cuda.is_available():
            raise RuntimeError("FliX needs a CUDA device; none is available")
        L = load()
        self.kw = key_bits
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.tdtype = torch.int32 if key_bits == 32 else torch.int64
        self.ndtype = np.uint32 if key_bits == 32 else np.uint64
        cfg = Config()
        L.flix_config_default(ctypes.byref(cfg), KEY_U32 if key_bits == 32 else KEY_U64)
        if node_size:
            cfg.node_size = node_size
        cfg.fill_pct = fill_pct
        cfg.pool_nodes = pool_nodes
        cfg.grow = 1 if grow else 0
        cfg.sort_variant = sort_variant
        cfg.restructure_in_one_pass = 1 if restructure_in_one_pass else 0
        cfg.split_chains_over = split_chains_over
        cfg.merge_underfull = 1 if merge_underfull else 0
        cfg.bucket_threads = bucket_threads
        self._alloc_cbs = None
        if allocator == "torch":
            self._alloc_cbs = _torch_allocator(self.device)   # kept alive as long as the index
            cfg.dev_alloc = ctypes.cast(self._alloc_cbs[0], ctypes.c_void_p)
            cfg.dev_free = ctypes.cast(self._alloc_cbs[1], ctypes.c_void_p)
        elif allocator is not None:
            raise ValueError("allocator must be None or 'torch'")
        self.node_size = cfg.node_size
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(L.flix_create(ctypes.byref(cfg), ctypes.byref(h)), "flix_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().flix_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- marshalling helpers ------------------------------------------------------------------
    def _dev(self, a, dtype=None):
        dtype = dtype or self.tdtype
        if a is None:
            return None
        if isinstance(a, np.ndarray):
            a = torch.from_numpy(np.ascontiguousarray(a).view(np.int32 if a.dtype.itemsize == 4 else
                                                              (np.int64 if a.dtype.itemsize == 8 else np.uint8)))
        if a.device != self.device:
            a = a.to(self.device, non_blocking=True)
        if a.dtype != dtype and a.element_size() == torch.empty(0, dtype=dtype).element_size():
            a = a.view(dtype)
        assert a.dtype == dtype, "expected %s, got %s" % (dtype, a.dtype)
        return a.contiguous()

    def _empty(self, n, dtype=None):
        return torch.empty(max(n, 0), dtype=dtype or self.tdtype, device=self.device)

    # -- operations ---------------------------------------------------------------------------
    def bulk_load(self, keys, vals, stream=None):
        k, v = self._dev(keys), self._dev(vals)
        _check(load().flix_bulk_load(self._h, _ptr(k), _ptr(v), k.numel(), _stream(stream)), "flix_bulk_load", self._h)

    def lookup(self, keys, stream=None, out=None, found=True):
        q = self._dev(keys)
        vals = out if out is not None else self._empty(q.numel())
        f = self._empty(q.numel(), torch.uint8) if found else None
        _check(load().flix_lookup(self._h, _ptr(q), q.numel(), _ptr(vals), _ptr(f), _stream(stream)),
               "flix_lookup", self._h)
        return vals, f

    def sort_pairs(self, keys, stream=None):
        """Test hook: the batch sort alone.  Returns (keys ascending, input position of each)."""
        q = self._dev(keys)
        ko = self._empty(q.numel())
        po = self._empty(q.numel(), torch.int32)
        _check(load().flix_sort_pairs(self._h, _ptr(q), q.numel(), _ptr(ko), _ptr(po), _stream(stream)),
               "flix_sort_pairs", self._h)
        return ko, po

    def successor(self, keys, stream=None, out=None):
        """out: optional (keys_out, vals_out) device tensors of at least len(keys) elements."""
        q = self._dev(keys)
        ko, vo = out if out is not None else (self._empty(q.numel()), self._empty(q.numel()))
        _check(load().flix_successor(self._h, _ptr(q), q.numel(), _ptr(ko), _ptr(vo), _stream(stream)),
               "flix_successor", self._h)
        return ko, vo

    def predecessor(self, keys, stream=None, out=None):
        """out: optional (keys_out, vals_out) device tensors of at least len(keys) elements."""
        q = self._dev(keys)
        ko, vo = out if out is not None else (self._empty(q.numel()), self._empty(q.numel()))
        _check(load().flix_predecessor(self._h, _ptr(q), q.numel(), _ptr(ko), _ptr(vo), _stream(stream)),
               "flix_predecessor", self._h)
        return ko, vo

    def range(self, lo, hi, capacity=None, stream=None, out=None):
        """out: optional (offsets, keys, vals) device tensors: offsets of len(lo) + 1 int64, keys and
        vals of `capacity` elements (default: their length)."""
        lo, hi = self._dev(lo), self._dev(hi)
        n = lo.numel()
        off = out[0] if out is not None else self._empty(n + 1, torch.int64)
        total = ctypes.c_uint64(0)
        L = load()
        if out is not None:
            rk, rv = out[1], out[2]
            cap = min(rk.numel(), rv.numel()) if capacity is None else capacity
            _check(L.flix_range(self._h, _ptr(lo), _ptr(hi), n, _ptr(off), _ptr(rk), _ptr(rv), cap,
                                ctypes.byref(total), _stream(stream)), "flix_range", self._h)
            t = int(total.value)
            return off[:n + 1], rk[:t], rv[:t]
        if capacity is None:
            # size the output from the counts, then fill
            code = L.flix_range(self._h, _ptr(lo), _ptr(hi), n, _ptr(off), None, None, 0, ctypes.byref(total),
                                _stream(stream))
            if code not in (0, -2):
                _check(code, "flix_range", self._h)
            capacity = int(total.value)
            if code == 0:
                return off, self._empty(0), self._empty(0)
        rk, rv = self._empty(capacity), self._empty(capacity)
        _check(L.flix_range(self._h, _ptr(lo), _ptr(hi), n, _ptr(off), _ptr(rk), _ptr(rv), capacity,
                            ctypes.byref(total), _stream(stream)), "flix_range", self._h)
        t = int(total.value)
        return off, rk[:t], rv[:t]

    def insert(self, keys, vals, stream=None):
        k, v = self._dev(keys), self._dev(vals)
        _check(load().flix_insert(self._h, _ptr(k), _ptr(v), k.numel(), _stream(stream)), "flix_insert", self._h)

    def delete(self, keys, stream=None):
        k = self._dev(keys)
        _check(load().flix_delete(self._h, _ptr(k), k.numel(), _stream(stream)), "flix_delete", self._h)

    def apply(self, ops, keys, aux, range_capacity=None, stream=None):
        """Mixed batch.  Returns dict(keys, vals, found, range_off, range_keys, range_vals)."""
        o = self._dev(ops, torch.uint8)
        k, a = self._dev(keys), self._dev(aux)
        n = k.numel()
        ko, vo, f = self._empty(n), self._empty(n), self._empty(n, torch.uint8)
        off = self._empty(n + 1, torch.int64)
        total = ctypes.c_uint64(0)
        L = load()
        cap = range_capacity
        if cap is None:
            cap = max(16, 64 * n)
        rk, rv = self._empty(cap), self._empty(cap)
        code = L.flix_apply(self._h, _ptr(o), _ptr(k), _ptr(a), n, _ptr(ko), _ptr(vo), _ptr(f), _ptr(off),
                            _ptr(rk), _ptr(rv), cap, ctypes.byref(total), _stream(stream))
        if code == -2 and range_capacity is None and total.value > cap:
            cap = int(total.value)
            rk, rv = self._empty(cap), self._empty(cap)
            code = L.flix_apply(self._h, _ptr(o), _ptr(k), _ptr(a), n, _ptr(ko), _ptr(vo), _ptr(f), _ptr(off),
                                _ptr(rk), _ptr(rv), cap, ctypes.byref(total), _stream(stream))
        _check(code, "flix_apply", self._h)
        t = int(total.value)
        return dict(keys=ko, vals=vo, found=f, range_off=off, range_keys=rk[:t], range_vals=rv[:t])

    def apply_async(self, ops, keys, aux, out, stream=None):
        """Mixed batch with no host synchronisation (graph-capturable).  `out` holds preallocated
        device tensors: keys, vals, found, range_off (n+1), range_keys, range_vals, status (4 x
        int64).  Nothing is returned; read out["status"] after the stream reaches the call."""
        o = self._dev(ops, torch.uint8)
        k, a = self._dev(keys), self._dev(aux)
        cap = out["range_keys"].numel()
        _check(load().flix_apply_async(self._h, _ptr(o), _ptr(k), _ptr(a), k.numel(), _ptr(out["keys"]),
                                       _ptr(out["vals"]), _ptr(out["found"]), _ptr(out["range_off"]),
                                       _ptr(out["range_keys"]), _ptr(out["range_vals"]), cap, _ptr(out["status"]),
                                       _stream(stream)), "flix_apply_async", self._h)

    def apply_queue(self, batches, wait_us: int = 2_000_000, flags_or=None, stream=None):
        """Run a queue of small mixed batches in one persistent kernel (flix_apply_queue).  batches:
        list of dicts with device tensors ops, keys, aux and outputs keys_out, vals_out, found,
        range_off (n+1), range_keys, range_vals, status (4 x int64), and optionally `ready` (an int32
        device word the kernel waits on).  flags_or: optional int64 device word that every batch's
        status flags are OR-ed into.  Asynchronous: read the outputs once the stream has run."""
        arr = (Batch * len(batches))()
        for i, b in enumerate(batches):
            o = self._dev(b["ops"], torch.uint8)
            k, a = self._dev(b["keys"]), self._dev(b["aux"])
            arr[i] = Batch(_ptr(o).value if o.numel() else None, _ptr(k).value if k.numel() else None,
                           _ptr(a).value if a.numel() else None, k.numel(),
                           *(_ptr(b[f]).value if b.get(f) is not None else None
                             for f in ("keys_out", "vals_out", "found", "range_off", "range_keys", "range_vals")),
                           b["range_keys"].numel() if b.get("range_keys") is not None else 0,
                           _ptr(b["status"]).value, _ptr(b["ready"]).value if b.get("ready") is not None else None)
        _check(load().flix_apply_queue(self._h, arr, len(batches), wait_us, _ptr(flags_or), _stream(stream)),
               "flix_apply_queue", self._h)

    def reserve(self, batch_max: int, free_nodes_min: int = 0, stream=None):
        _check(load().flix_reserve(self._h, batch_max, free_nodes_min, _stream(stream)), "flix_reserve", self._h)

    def split_chains(self, max_chain: int, stream=None) -> int:
        """Elastic split of every bucket whose chain is longer than max_chain; returns buckets added."""
        added = ctypes.c_uint64(0)
        _check(load().flix_split_chains(self._h, max_chain, ctypes.byref(added), _stream(stream)),
               "flix_split_chains", self._h)
        return int(added.value)

    def merge_underfull(self, stream=None) -> int:
        """Underfull-neighbour merge in every bucket; returns nodes freed."""
        freed = ctypes.c_uint64(0)
        _check(load().flix_merge_underfull(self._h, ctypes.byref(freed), _stream(stream)),
               "flix_merge_underfull", self._h)
        return int(freed.value)

    def restructure(self, stream=None):
        _check(load().flix_restructure(self._h, _stream(stream)), "flix_restructure", self._h)

    def stats(self, stream=None) -> dict:
        s = Stats()
        _check(load().flix_stats(self._h, ctypes.byref(s), _stream(stream)), "flix_stats", self._h)
        return {n: int(getattr(s, n)) for n, _ in Stats._fields_}

    def export(self, stream=None):
        L = load()
        n = ctypes.c_uint64(0)
        code = L.flix_export(self._h, None, None, 0, ctypes.byref(n), _stream(stream))
        if code not in (0, -2):
            _check(code, "flix_export", self._h)
        k, v = self._empty(n.value), self._empty(n.value)
        _check(L.flix_export(self._h, _ptr(k), _ptr(v), n.value, ctypes.byref(n), _stream(stream)),
               "flix_export", self._h)
        return k, v

    def dump_layout(self, stream=None) -> dict:
        L = load()
        c = (ctypes.c_uint64 * 3)()
        _check(L.flix_dump_layout(self._h, c, None, None, None, None, None, None, _stream(stream)),
               "flix_dump_layout", self._h)
        nb, nn, nk = int(c[0]), int(c[1]), int(c[2])
        dt = self.ndtype
        mk, cl = np.empty(nb, dt), np.empty(nb, np.uint32)
        ns, bd = np.empty(nn, np.uint32), np.empty(nn, dt)
        k, v = np.empty(nk, dt), np.empty(nk, dt)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        _check(L.flix_dump_layout(self._h, c, p(mk), p(cl), p(ns), p(bd), p(k), p(v), _stream(stream)),
               "flix_dump_layout", self._h)
        return dict(mkba=mk, chain_len=cl, node_size=ns, node_bound=bd, keys=k, vals=v)

    # -- profiling ------------------------------------------------------------------------------
    def profile(self, enable: bool = True):
        _check(load().flix_profile_enable(self._h, 1 if enable else 0), "flix_profile_enable")

    def profile_reset(self):
        _check(load().flix_profile_reset(self._h), "flix_profile_reset")

    def profile_read(self) -> dict:
        L = load()
        m = 64
        names = ctypes.create_string_buffer(48 * m)
        la = (ctypes.c_uint64 * m)()
        ms = (ctypes.c_double * m)()
        by = (ctypes.c_double * m)()
        k = ctypes.c_uint32(0)
        _check(L.flix_profile_read(self._h, m, names, la, ms, by, ctypes.byref(k)), "flix_profile_read", self._h)
        out = {}
        for i in range(k.value):
            nm = names.raw[48 * i:48 * (i + 1)].split(b"\0", 1)[0].decode()
            out[nm] = dict(launches=int(la[i]), ms=float(ms[i]), bytes=float(by[i]))
        return out

    def launch_count(self) -> int:
        return int(load().flix_launch_count(self._h))
