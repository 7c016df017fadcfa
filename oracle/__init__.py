"""CPU oracle for FliX -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of ``bench.py``
may import this package.  The product path (``paper_2604_16725_gb300``) never imports it and shares
no code with it.

``flix_oracle.c`` holds the plain C oracle (a semantic ordered map and a structural model of the
bucket/node layout, see its header); this module builds it with gcc and wraps it with ctypes.  All
arrays cross the boundary as uint64 whatever the key width.

Parity pins: every function here is pinned by ``tests/test_oracle_*.py`` against the paper's worked
examples (Tab. 2, Tab. 3, the build example of Sec. 3.2), brute force on tiny key domains, linear
scans and structural invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "flix_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

OP_NOP, OP_LOOKUP, OP_SUCC, OP_RANGE, OP_INSERT, OP_DELETE, OP_PRED = 0, 1, 2, 3, 4, 5, 6

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no target-specific flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-pthread", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp, u64, u32, sz, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
        L.om_map_create.restype = vp
        L.om_map_create.argtypes = [i32]
        L.om_map_destroy.argtypes = [vp]
        L.om_map_size.restype = sz
        L.om_map_size.argtypes = [vp]
        L.om_map_export.argtypes = [vp, vp, vp]
        L.om_map_bulk_load.restype = i32
        L.om_map_bulk_load.argtypes = [vp, vp, vp, sz]
        L.om_map_read.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp, vp]
        L.om_map_range_fill.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp]
        L.om_map_update.restype = i32
        L.om_map_update.argtypes = [vp, sz, vp, vp, vp]
        L.om_map_read_mt.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp, vp, i32]
        L.om_map_range_fill_mt.argtypes = [vp, sz, vp, vp, vp, vp, vp, vp, i32]
        L.om_map_update_mt.restype = i32
        L.om_map_update_mt.argtypes = [vp, sz, vp, vp, vp, i32]
        L.om_delete_compact.restype = u32
        L.om_delete_compact.argtypes = [vp, u32, vp, u32, vp, vp]
        L.om_merge_insert.restype = u32
        L.om_merge_insert.argtypes = [vp, u32, vp, u32, vp]
        L.om_canonical_layout.restype = u32
        L.om_canonical_layout.argtypes = [u64, u32, vp]
        L.om_model_create.restype = vp
        L.om_model_create.argtypes = [i32, u32, u32]
        L.om_model_destroy.argtypes = [vp]
        L.om_model_bulk_load.restype = i32
        L.om_model_bulk_load.argtypes = [vp, vp, vp, u64]
        L.om_model_update.restype = i32
        L.om_model_update.argtypes = [vp, u64, vp, vp, vp]
        L.om_model_restructure.restype = ctypes.c_int64
        L.om_model_restructure.argtypes = [vp]
        L.om_model_split_chains.restype = u64
        L.om_model_split_chains.argtypes = [vp, u64]
        L.om_model_merge_underfull_all.restype = u64
        L.om_model_merge_underfull_all.argtypes = [vp]
        L.om_model_set_policy.argtypes = [vp, u64, i32]
        L.om_model_read.argtypes = [vp, u64, vp, vp, vp, vp, vp]
        L.om_model_dump.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
        L.om_model_check.restype = i32
        L.om_model_check.argtypes = [vp, i32]
        for f in ("om_model_live_keys", "om_model_nodes_used", "om_model_buckets", "om_model_max_chain"):
            getattr(L, f).restype = u64
            getattr(L, f).argtypes = [vp]
        _lib = L
    return _lib


def _u64(a) -> np.ndarray:
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a.astype(np.uint64, copy=False))
    return np.ascontiguousarray(np.array(list(a), dtype=np.uint64))


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).astype(np.uint8))


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def key_max(kw: int) -> int:
    return (1 << kw) - 1


class Map:
    """Semantic ordered map (the result every FliX batch must reach)."""

    def __init__(self, kw: int):
        self.kw = kw
        self._h = lib().om_map_create(kw)
        if not self._h:
            raise ValueError("key width must be 32 or 64")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().om_map_destroy(self._h)
            self._h = None

    def __len__(self):
        return int(lib().om_map_size(self._h))

    def bulk_load(self, keys, vals) -> int:
        k, v = _u64(keys), _u64(vals)
        return lib().om_map_bulk_load(self._h, _p(k), _p(v), k.size)

    def export(self):
        n = len(self)
        k = np.empty(n, np.uint64)
        v = np.empty(n, np.uint64)
        lib().om_map_export(self._h, _p(k), _p(v))
        return k, v

    def read(self, ops, keys, aux=None):
        """Snapshot reads: returns dict(keys, vals, found, range_off, range_keys, range_vals)."""
        o, k = _u8(ops), _u64(keys)
        a = _u64(aux) if aux is not None else np.zeros(k.size, np.uint64)
        n = k.size
        ok = np.empty(n, np.uint64)
        ov = np.empty(n, np.uint64)
        of = np.empty(n, np.uint8)
        off = np.empty(n + 1, np.uint64)
        lib().om_map_read(self._h, n, _p(o), _p(k), _p(a), _p(ov), _p(of), _p(ok), _p(off))
        tot = int(off[-1])
        rk = np.empty(tot, np.uint64)
        rv = np.empty(tot, np.uint64)
        if tot:
            lib().om_map_range_fill(self._h, n, _p(o), _p(k), _p(a), _p(off), _p(rk), _p(rv))
        return dict(keys=ok, vals=ov, found=of, range_off=off, range_keys=rk, range_vals=rv)

    def update(self, ops, keys, aux=None) -> int:
        o, k = _u8(ops), _u64(keys)
        a = _u64(aux) if aux is not None else np.zeros(k.size, np.uint64)
        return lib().om_map_update(self._h, k.size, _p(o), _p(k), _p(a))

    def read_mt(self, ops, keys, aux=None, threads: int = 1, ranges: bool = True):
        """read() on `threads` host threads (the batch-synchronous CPU baseline); same outputs."""
        o, k = _u8(ops), _u64(keys)
        a = _u64(aux) if aux is not None else np.zeros(k.size, np.uint64)
        n = k.size
        ok = np.empty(n, np.uint64)
        ov = np.empty(n, np.uint64)
        of = np.empty(n, np.uint8)
        off = np.empty(n + 1, np.uint64)
        lib().om_map_read_mt(self._h, n, _p(o), _p(k), _p(a), _p(ov), _p(of), _p(ok), _p(off), threads)
        tot = int(off[-1])
        rk = np.empty(tot, np.uint64)
        rv = np.empty(tot, np.uint64)
        if tot and ranges:
            lib().om_map_range_fill_mt(self._h, n, _p(o), _p(k), _p(a), _p(off), _p(rk), _p(rv), threads)
        return dict(keys=ok, vals=ov, found=of, range_off=off, range_keys=rk, range_vals=rv)

    def update_mt(self, ops, keys, aux=None, threads: int = 1) -> int:
        """update() on `threads` host threads; same result."""
        o, k = _u8(ops), _u64(keys)
        a = _u64(aux) if aux is not None else np.zeros(k.size, np.uint64)
        return lib().om_map_update_mt(self._h, k.size, _p(o), _p(k), _p(a), threads)

    def apply(self, ops, keys, aux=None):
        """A mixed batch: reads on the snapshot, then updates.  Returns (reads, status)."""
        r = self.read(ops, keys, aux)
        st = self.update(ops, keys, aux)
        return r, st


class Model:
    """Structural model of FliX's buckets, node chains and MKBA."""

    def __init__(self, kw: int, node_size: int, fill_pct: int = 50):
        self.kw, self.NS, self.fill_pct = kw, node_size, fill_pct
        self._h = lib().om_model_create(kw, node_size, fill_pct)
        if not self._h:
            raise ValueError("bad model parameters")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().om_model_destroy(self._h)
            self._h = None

    def bulk_load(self, keys, vals) -> int:
        k, v = _u64(keys), _u64(vals)
        return lib().om_model_bulk_load(self._h, _p(k), _p(v), k.size)

    def update(self, ops, keys, aux=None) -> int:
        o, k = _u8(ops), _u64(keys)
        a = _u64(aux) if aux is not None else np.zeros(k.size, np.uint64)
        return lib().om_model_update(self._h, k.size, _p(o), _p(k), _p(a))

    def restructure(self) -> int:
        return int(lib().om_model_restructure(self._h))

    def split_chains(self, max_chain: int) -> int:
        """Elastic split of every bucket whose chain is longer than max_chain; returns buckets added."""
        return int(lib().om_model_split_chains(self._h, max_chain))

    def merge_underfull_all(self) -> int:
        """Underfull-neighbour merge in every bucket; returns nodes freed."""
        return int(lib().om_model_merge_underfull_all(self._h))

    def set_policy(self, split_over: int = 0, merge_underfull: bool = False):
        """Maintenance after every update batch, in the buckets the batch touched: merge underfull
        neighbours, then split chains longer than split_over (0: off)."""
        lib().om_model_set_policy(self._h, split_over, 1 if merge_underfull else 0)

    def read(self, ops, keys):
        o, k = _u8(ops), _u64(keys)
        n = k.size
        ok = np.empty(n, np.uint64)
        ov = np.empty(n, np.uint64)
        of = np.empty(n, np.uint8)
        lib().om_model_read(self._h, n, _p(o), _p(k), _p(ov), _p(of), _p(ok))
        return dict(keys=ok, vals=ov, found=of)

    def check(self, build_shape: bool = False) -> int:
        return int(lib().om_model_check(self._h, 1 if build_shape else 0))

    def stats(self):
        L = lib()
        return dict(buckets=int(L.om_model_buckets(self._h)), nodes=int(L.om_model_nodes_used(self._h)),
                    keys=int(L.om_model_live_keys(self._h)), max_chain=int(L.om_model_max_chain(self._h)))

    def dump(self):
        """Layout in bucket and chain order: mkba, chain_len, node_size, node_bound, keys, vals."""
        c = np.zeros(3, np.uint64)
        L = lib()
        L.om_model_dump(self._h, _p(c), None, None, None, None, None, None)
        nb, nn, nk = (int(x) for x in c)
        mk = np.empty(nb, np.uint64)
        cl = np.empty(nb, np.uint32)
        ns = np.empty(nn, np.uint32)
        bd = np.empty(nn, np.uint64)
        k = np.empty(nk, np.uint64)
        v = np.empty(nk, np.uint64)
        L.om_model_dump(self._h, _p(c), _p(mk), _p(cl), _p(ns), _p(bd), _p(k), _p(v))
        return dict(mkba=mk, chain_len=cl, node_size=ns, node_bound=bd, keys=k, vals=v)


def delete_compact(keys, dels):
    """Tab. 3 step: returns (compacted keys, shift distance per slot, -1 for deleted slots)."""
    k, d = _u64(keys), _u64(dels)
    out = np.zeros(max(k.size, 1), np.uint64)
    sh = np.zeros(max(k.size, 1), np.int32)
    n = lib().om_delete_compact(_p(k), k.size, _p(d), d.size, _p(out), _p(sh))
    return out[:n], sh[:k.size]


def merge_insert(keys, ins):
    """Tab. 2 step: the node's keys merged with the insert sublist (present keys not repeated)."""
    k, i = _u64(keys), _u64(ins)
    out = np.zeros(k.size + i.size + 1, np.uint64)
    n = lib().om_merge_insert(_p(k), k.size, _p(i), i.size, _p(out))
    return out[:n]


def canonical_layout(t: int, node_size: int):
    """Piece sizes of a merged run of t keys under the canonical split rule."""
    ps = np.zeros(t // max(node_size // 2, 1) + 2, np.uint32)
    q = lib().om_canonical_layout(t, node_size, _p(ps))
    return ps[:q].tolist()


# -------------------------------------------------------------------------------------------------
# Sampled checks at full size: plain definitions over the sorted stored set (numpy searchsorted is a
# library binary search over the sorted keys, used as a step of the definition).
# -------------------------------------------------------------------------------------------------

def sorted_lookup(sorted_keys: np.ndarray, sorted_vals: np.ndarray, q: np.ndarray, kw: int):
    p = np.searchsorted(sorted_keys, q, side="left")
    pc = np.minimum(p, max(sorted_keys.size - 1, 0))
    hit = (p < sorted_keys.size) & (sorted_keys[pc] == q) if sorted_keys.size else np.zeros(q.size, bool)
    none = np.uint64(key_max(kw))
    vals = np.where(hit, sorted_vals[pc] if sorted_keys.size else none, none).astype(np.uint64)
    return vals, hit.astype(np.uint8)


def sorted_predecessor(sorted_keys: np.ndarray, sorted_vals: np.ndarray, q: np.ndarray, kw: int):
    """Largest stored key <= q (KEY_MAX, VAL_NONE, not found when none), by binary search."""
    p = np.searchsorted(sorted_keys, q, side="right")
    ok = p > 0
    pc = np.maximum(p - 1, 0)
    none = np.uint64(key_max(kw))
    if sorted_keys.size == 0:
        return np.full(q.size, none), np.full(q.size, none), np.zeros(q.size, np.uint8)
    return (np.where(ok, sorted_keys[pc], none).astype(np.uint64),
            np.where(ok, sorted_vals[pc], none).astype(np.uint64), ok.astype(np.uint8))


def sorted_successor(sorted_keys: np.ndarray, sorted_vals: np.ndarray, q: np.ndarray, kw: int):
    p = np.searchsorted(sorted_keys, q, side="left")
    ok = p < sorted_keys.size
    pc = np.minimum(p, max(sorted_keys.size - 1, 0))
    none = np.uint64(key_max(kw))
    if sorted_keys.size == 0:
        return np.full(q.size, none), np.full(q.size, none), np.zeros(q.size, np.uint8)
    return (np.where(ok, sorted_keys[pc], none).astype(np.uint64),
            np.where(ok, sorted_vals[pc], none).astype(np.uint64), ok.astype(np.uint8))


def sorted_range_counts(sorted_keys: np.ndarray, lo: np.ndarray, hi: np.ndarray):
    a = np.searchsorted(sorted_keys, lo, side="left")
    b = np.searchsorted(sorted_keys, hi, side="right")
    return np.where(lo <= hi, b - a, 0).astype(np.uint64)
