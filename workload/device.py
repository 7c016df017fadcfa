"""The batched-form stream (see gen.mixed_stream) generated on the GPU, for benchmark streams too
large to draw on the host (10,000 batches of log-uniform sizes 2^8..2^22: about 4.3e9 ops).

Same recipe as gen.mixed_stream: the same batch sizes, op mix, hit rate and range spans; hits and
deletes draw from the preload and the keys inserted earlier in the stream, inserts take fresh keys
of the same seeded universe (gen.universe's bijection of counters), so keys stay distinct.  The
per-op random draws come from torch's generator instead of the counter-based words, so the ops
differ from gen.mixed_stream's; parity tests use gen.mixed_stream, this module feeds timing runs
only.  No arithmetic of the FliX method is here.
"""
from __future__ import annotations

import numpy as np

from . import gen

_M = (1 << 64) - 1


def _i64(x: int) -> int:
    """A uint64 constant as the int64 with the same bits (torch has no uint64 arithmetic)."""
    x &= _M
    return x - (1 << 64) if x >> 63 else x


def _shr(t, s: int):
    """Logical right shift of int64 tensors holding uint64 bits."""
    import torch
    return (t >> s) & torch.tensor((1 << (64 - s)) - 1, dtype=torch.int64, device=t.device)


def mix64(t):
    """gen.mix64 (SplitMix64 finaliser) on int64 tensors holding uint64 bits (wrapping arithmetic)."""
    z = t.clone()
    z = (z ^ _shr(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _shr(z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _shr(z, 31)


def universe_at64(seed: int, ctr):
    """gen.universe_at(64, seed, ctr) on the device (ctr: int64 tensor of counters)."""
    import torch
    s = int(gen._stream_words(seed, 0xC0FFEE, 1)[0])
    k = mix64(ctr ^ _i64(s))
    bad = k == -1
    if bool(bad.any()):
        k = torch.where(bad, mix64(torch.tensor([_i64(_M ^ s)], dtype=torch.int64, device=k.device)), k)
    return k


def values_for64(keys, salt: int = 0):
    """gen.values_for(64, keys, salt) on the device."""
    return mix64(keys ^ _i64(0x5DEECE66D + salt)) & _i64(0xFFFFFFFFFFFFFFFE)


def mixed_stream_device(seed: int = 4000, n_preload: int = 1 << 27, n_batches: int = 10000, lo_exp: float = 8,
                        hi_exp: float = 22, hit_rate: float = 0.7, max_len: int = 1000,
                        mix=(0.60, 0.15, 0.05, 0.10, 0.10), device="cuda"):
    """uint64 stream: dict(preload_keys, preload_vals (int64 device tensors), sizes, batches) where
    batches() yields (ops uint8, keys int64, aux int64) device tensors."""
    import torch
    sizes = gen.log_uniform_sizes(seed, 1, n_batches, lo_exp, hi_exp)
    pre = universe_at64(seed, torch.arange(n_preload, dtype=torch.int64, device=device))
    cum = torch.tensor(np.cumsum(np.array(mix) / np.sum(mix)), dtype=torch.float64, device=device)
    km1 = _i64((1 << 64) - 2)

    def batches():
        g = torch.Generator(device=device)
        g.manual_seed(seed)
        n_ins = 0
        miss_ctr = 0
        for b, m in enumerate(sizes):
            m = int(m)
            u = torch.rand(m, generator=g, dtype=torch.float64, device=device)
            ops = (torch.searchsorted(cum, u, right=True) + 1).clamp(max=gen.OP_DELETE).to(torch.uint8)
            src = torch.randint(0, n_preload + n_ins, (m,), generator=g, device=device, dtype=torch.int64)
            kk = universe_at64(seed, src)
            hit = torch.rand(m, generator=g, device=device) < hit_rate
            miss = universe_at64(seed ^ 0x5A5A, torch.arange(miss_ctr, miss_ctr + m, dtype=torch.int64, device=device))
            miss_ctr += m
            kk = torch.where(hit, kk, miss)
            is_ins = ops == gen.OP_INSERT
            k_ins = int(is_ins.sum())
            fresh = universe_at64(seed, torch.arange(n_preload + n_ins, n_preload + n_ins + k_ins, dtype=torch.int64,
                                                     device=device))
            n_ins += k_ins
            kk[is_ins] = fresh
            aux = torch.zeros(m, dtype=torch.int64, device=device)
            aux[is_ins] = values_for64(fresh, salt=b + 7)
            is_rng = ops == gen.OP_RANGE
            if bool(is_rng.any()):
                gap = (1 << 64) // max(n_preload + n_ins, 1)     # the mean gap of the keys generated so far
                span = (torch.randint(0, max_len, (m,), generator=g, device=device, dtype=torch.int64) + 1)
                lo = kk.double() % float(1 << 64)
                lo = torch.where(lo < 0, lo + float(1 << 64), lo)
                # hi = lo + span * gap, capped below the reserved key (computed in floating point:
                # a range's end only needs to land about span stored keys above lo)
                hi_f = torch.clamp(lo + span.double() * float(gap), max=float((1 << 64) - 4096))
                hi = torch.where(hi_f >= float(1 << 63), (hi_f - float(1 << 64)), hi_f).to(torch.int64)
                # unsigned order: hi must not fall below lo (lo close to the top of the key range)
                lo_u = kk ^ _i64(1 << 63)
                hi_u = hi ^ _i64(1 << 63)
                hi = torch.where(hi_u < lo_u, torch.full_like(hi, km1), hi)
                aux[is_rng] = hi[is_rng]
            yield ops, kk, aux

    return dict(preload_keys=pre, preload_vals=values_for64(pre), sizes=sizes, batches=batches)
