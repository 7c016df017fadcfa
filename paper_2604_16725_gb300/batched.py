"""Batched form: a stream of uneven mixed batches through captured CUDA graphs.

Each batch is padded to the next power of two (padding ops are NOPs on the reserved key, which
sort to the end and change nothing) and replayed through a CUDA graph captured once per size class
around flix_apply_async, so a batch costs one graph launch and no host synchronisation.  Admission
(free nodes, range capacity, reserved keys) is decided on the device; each batch leaves its status
words on the device and the runner checks them every `check_every` batches.

Graphs hold the index's pool pointers and bucket count, so they are re-captured after a
restructure (the runner's `restructure_if_needed` does both).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .flix import OP_NOP, FlixError, Index


class _Class:
    def __init__(self, idx: Index, size: int, range_cap: int, stream):
        dev, dt = idx.device, idx.tdtype
        self.size = size
        self.ops = torch.zeros(size, dtype=torch.uint8, device=dev)
        self.keys = torch.full((size,), -1, dtype=dt, device=dev)       # reserved key: padding
        self.aux = torch.zeros(size, dtype=dt, device=dev)
        self.out = dict(keys=torch.empty(size, dtype=dt, device=dev), vals=torch.empty(size, dtype=dt, device=dev),
                        found=torch.empty(size, dtype=torch.uint8, device=dev),
                        range_off=torch.empty(size + 1, dtype=torch.int64, device=dev),
                        range_keys=torch.empty(max(range_cap, 1), dtype=dt, device=dev),
                        range_vals=torch.empty(max(range_cap, 1), dtype=dt, device=dev),
                        status=torch.zeros(4, dtype=torch.int64, device=dev))
        self.filled = size          # padding is valid beyond this many real ops
        self.graph = None
        self.stream = stream

    def capture(self, idx: Index):
        s = self.stream
        with torch.cuda.stream(s):
            # the warm-up runs for real: give it an all-padding batch so that it changes nothing
            self.ops.fill_(OP_NOP)
            self.keys.fill_(-1)
            self.aux.zero_()
            self.filled = self.size
            idx.apply_async(self.ops, self.keys, self.aux, self.out, stream=s)   # warm-up, not captured
        s.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            idx.apply_async(self.ops, self.keys, self.aux, self.out, stream=s)
        self.graph = g


class BatchedRunner:
    """Run mixed batches (device tensors ops/keys/aux) on `idx` through per-size-class CUDA graphs."""

    def __init__(self, idx: Index, max_batch: int, min_log: int = 8, range_per_op: int = 64,
                 free_nodes_min: int = 0, check_every: int = 64):
        self.idx = idx
        self.min_log = min_log
        self.max_log = max(min_log, math.ceil(math.log2(max(max_batch, 2))))
        self.range_per_op = range_per_op
        self.stream = torch.cuda.Stream(device=idx.device)
        self.check_every = check_every
        self.classes: dict[int, _Class] = {}
        self.batches = 0
        self.flags = torch.zeros(1, dtype=torch.int64, device=idx.device)   # OR of every batch's status flags
        idx.reserve(1 << self.max_log, free_nodes_min, stream=self.stream)

    def _class(self, n: int) -> _Class:
        c = max(self.min_log, math.ceil(math.log2(max(n, 1))))
        if c > self.max_log:
            raise ValueError("batch of %d ops exceeds the reserved maximum 2^%d" % (n, self.max_log))
        cl = self.classes.get(c)
        if cl is None:
            cl = _Class(self.idx, 1 << c, self.range_per_op * (1 << c), self.stream)
            self.classes[c] = cl
        if cl.graph is None:
            cl.capture(self.idx)
        return cl

    def invalidate(self):
        """Drop every captured graph (after a restructure, a bulk load or pool growth)."""
        for cl in self.classes.values():
            cl.graph = None

    def run(self, ops, keys, aux):
        """Enqueue one batch; returns views of its result tensors (valid once the stream reaches
        them, and until the next batch of the same size class)."""
        n = int(keys.numel())
        cl = self._class(n)
        s = self.stream
        with torch.cuda.stream(s):
            cl.ops[:n].copy_(ops, non_blocking=True)
            cl.keys[:n].copy_(keys.view(cl.keys.dtype), non_blocking=True)
            cl.aux[:n].copy_(aux.view(cl.aux.dtype), non_blocking=True)
            if n < cl.filled:                       # restore the padding of the previous, longer batch
                cl.ops[n:cl.filled].fill_(OP_NOP)
                cl.keys[n:cl.filled].fill_(-1)
                cl.aux[n:cl.filled].zero_()
            cl.filled = n
            cl.graph.replay()
            self.flags.bitwise_or_(cl.out["status"][:1])
        self.batches += 1
        if self.batches % self.check_every == 0:
            self.check()
        o = cl.out
        return dict(keys=o["keys"][:n], vals=o["vals"][:n], found=o["found"][:n], range_off=o["range_off"][:n + 1],
                    range_keys=o["range_keys"], range_vals=o["range_vals"], status=o["status"])

    def check(self):
        """Synchronise and raise if a batch since the last check was not admitted."""
        self.stream.synchronize()
        f = int(self.flags.item())
        if f:
            self.flags.zero_()
            raise FlixError(-1 if f == 1 else -2, "batched apply",
                            "status flags %d: 1 reserved key, 2 node pool short, 4 range capacity short" % f)

    def restructure_if_needed(self, max_nodes_per_bucket: float = 2.0, max_chain: int = 64) -> bool:
        """Restructure when nodes > 2 * buckets or a chain exceeds 64 nodes; graphs are re-captured."""
        self.check()
        s = self.idx.stats(stream=self.stream)
        if s["nodes_used"] > max_nodes_per_bucket * s["buckets"] or s["max_chain"] > max_chain:
            self.idx.restructure(stream=self.stream)
            self.idx.reserve(1 << self.max_log, 0, stream=self.stream)
            self.invalidate()
            return True
        return False

    def synchronize(self):
        self.check()
