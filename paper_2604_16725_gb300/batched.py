"""Batched form: a stream of uneven mixed batches through captured CUDA graphs.

Each batch is padded up to the nearest size class (four classes per power of two, rounded up to
multiples of 256 ops, so padding stays under 20% from 1024 ops and under 18% from 8192; padding ops
are NOPs on the reserved key, which sort to the end and change nothing) and replayed through a CUDA graph captured once per class around flix_apply_async, so a
batch costs one graph launch and no host synchronisation.  All classes share one set of input and
result buffers; a batch's results stay valid until the next batch runs.  Admission (free nodes,
range capacity, reserved keys) is decided on the device; each batch's status flags are OR-ed into
one device word that the runner checks every `check_every` batches.

Graphs hold the index's pool pointers and bucket count, so they are re-captured after a
restructure, a bulk load or pool growth (`invalidate`; `restructure_if_needed` does both).

With `queue_depth` > 0 (the persistent path), batches of at most QUEUE_BATCH_MAX ops are not
launched one by one: their inputs go into one of `queue_depth` slots, and a full queue (or a larger
batch, or a check) runs every queued batch in order through ONE launch of the library's persistent
kernel (flix_apply_queue).  A queued batch's results are in its slot once that launch has run, and
stay there until the slot is reused `queue_depth` batches later.
"""
from __future__ import annotations

import math

import torch

from .flix import OP_NOP, QUEUE_BATCH_MAX, FlixError, Index


def class_sizes(min_log: int, max_log: int, per_octave: int = 4, align: int = 256):
    """Batch size classes from 2^min_log to 2^max_log, `per_octave` per power of two."""
    out = set()
    for c in range(min_log * per_octave, max_log * per_octave + 1):
        s = int(math.ceil(2.0 ** (c / per_octave)))
        s = max(align, (s + align - 1) // align * align) if s > align else max(s, 1 << min_log)
        out.add(s)
    return sorted(out)


class BatchedRunner:
    """Run mixed batches (device tensors ops/keys/aux) on `idx` through per-size-class CUDA graphs."""

    def __init__(self, idx: Index, max_batch: int, min_log: int = 8, range_per_op: int = 64,
                 free_nodes_min: int = 0, check_every: int = 64, per_octave: int = 4, queue_depth: int = 0):
        self.idx = idx
        self.min_log = min_log
        self.max_log = max(min_log, math.ceil(math.log2(max(max_batch, 2))))
        self.sizes = class_sizes(min_log, self.max_log, per_octave)
        S = self.sizes[-1]
        dev, dt = idx.device, idx.tdtype
        self.stream = torch.cuda.Stream(device=idx.device)
        self.check_every = check_every
        self.ops = torch.zeros(S, dtype=torch.uint8, device=dev)
        self.keys = torch.full((S,), -1, dtype=dt, device=dev)          # reserved key: padding
        self.aux = torch.zeros(S, dtype=dt, device=dev)
        self.out = dict(keys=torch.empty(S, dtype=dt, device=dev), vals=torch.empty(S, dtype=dt, device=dev),
                        found=torch.empty(S, dtype=torch.uint8, device=dev),
                        range_off=torch.empty(S + 1, dtype=torch.int64, device=dev),
                        range_keys=torch.empty(max(range_per_op * S, 1), dtype=dt, device=dev),
                        range_vals=torch.empty(max(range_per_op * S, 1), dtype=dt, device=dev),
                        status=torch.zeros(4, dtype=torch.int64, device=dev))
        self.graphs: dict[int, torch.cuda.CUDAGraph] = {}
        self.batches = 0
        # persistent path: slots of queued small batches
        self.queue_depth = queue_depth
        self.pending = []
        self.slots = []
        Q = QUEUE_BATCH_MAX
        for _ in range(queue_depth):
            self.slots.append(dict(keys=torch.empty(0, dtype=dt, device=dev), keys_out=torch.empty(Q, dtype=dt, device=dev),
                                   vals_out=torch.empty(Q, dtype=dt, device=dev),
                                   found=torch.empty(Q, dtype=torch.uint8, device=dev),
                                   range_off=torch.empty(Q + 1, dtype=torch.int64, device=dev),
                                   range_keys=torch.empty(max(range_per_op * Q, 1), dtype=dt, device=dev),
                                   range_vals=torch.empty(max(range_per_op * Q, 1), dtype=dt, device=dev),
                                   status=torch.zeros(4, dtype=torch.int64, device=dev)))
        self.next_slot = 0
        self.queues = 0
        self.on_flush = None      # called on self.stream right after each queue launch
        self.flags = torch.zeros(1, dtype=torch.int64, device=dev)   # OR of every batch's status flags
        idx.reserve(S, free_nodes_min, stream=self.stream)
        # run the flag accumulation once now: a first use inside the stream of batches would load
        # its kernel then (measured at ~0.7 s under lazy module loading)
        with torch.cuda.stream(self.stream):
            self.flags.bitwise_or_(self.out["status"][:1])
        self.stream.synchronize()

    def _views(self, s):
        o = self.out
        return dict(keys=o["keys"][:s], vals=o["vals"][:s], found=o["found"][:s], range_off=o["range_off"][:s + 1],
                    range_keys=o["range_keys"], range_vals=o["range_vals"], status=o["status"])

    def size_for(self, n: int) -> int:
        for s in self.sizes:
            if s >= n:
                return s
        raise ValueError("batch of %d ops exceeds the reserved maximum %d" % (n, self.sizes[-1]))

    def graph_for(self, s: int):
        g = self.graphs.get(s)
        if g is None:
            st = self.stream
            with torch.cuda.stream(st):
                # the warm-up runs for real: give it an all-padding batch so that it changes nothing
                self.ops[:s].fill_(OP_NOP)
                self.keys[:s].fill_(-1)
                self.aux[:s].zero_()
                self.idx.apply_async(self.ops[:s], self.keys[:s], self.aux[:s], self._views(s), stream=st)
            st.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=st):
                self.idx.apply_async(self.ops[:s], self.keys[:s], self.aux[:s], self._views(s), stream=st)
            self.graphs[s] = g
        return g

    def invalidate(self):
        """Drop every captured graph (after a restructure, a bulk load or pool growth)."""
        self.graphs.clear()

    def flush(self):
        """Run every queued small batch through one persistent-kernel launch on `self.stream`."""
        if not self.pending:
            return
        with torch.cuda.stream(self.stream):
            self.idx.apply_queue(self.pending, flags_or=self.flags, stream=self.stream)
            if self.on_flush is not None:
                self.on_flush()
        self.pending = []
        self.queues += 1

    def _enqueue(self, ops, keys, aux, n):
        slot = self.slots[self.next_slot]
        self.next_slot = (self.next_slot + 1) % self.queue_depth
        # the batch's own input tensors go into the queue (held until its launch): no copies
        dt = slot["keys"].dtype
        ops, keys, aux = ops.contiguous(), keys.view(dt).contiguous(), aux.view(dt).contiguous()
        for t in (ops, keys, aux):
            t.record_stream(self.stream)     # not reused by the allocator before the queue has run
        b = dict(ops=ops, keys=keys, aux=aux, keys_out=slot["keys_out"],
                 vals_out=slot["vals_out"], found=slot["found"], range_off=slot["range_off"][:n + 1],
                 range_keys=slot["range_keys"], range_vals=slot["range_vals"], status=slot["status"])
        self.pending.append(b)
        self.batches += 1
        if len(self.pending) == self.queue_depth:
            self.flush()
        if self.batches % self.check_every == 0:
            self.check()
        return dict(keys=slot["keys_out"][:n], vals=slot["vals_out"][:n], found=slot["found"][:n],
                    range_off=slot["range_off"][:n + 1], range_keys=slot["range_keys"],
                    range_vals=slot["range_vals"], status=slot["status"])

    def run(self, ops, keys, aux):
        """Enqueue one batch on `self.stream`; returns views of its results (valid once the stream
        reaches them, until the next batch; on the persistent path, once its queue has run and until
        its slot is reused)."""
        n = int(keys.numel())
        if self.queue_depth and n <= QUEUE_BATCH_MAX:
            self.stream.wait_stream(torch.cuda.current_stream(self.idx.device))
            return self._enqueue(ops, keys, aux, n)
        self.flush()
        s = self.size_for(n)
        g = self.graph_for(s)
        with torch.cuda.stream(self.stream):
            self.ops[:n].copy_(ops, non_blocking=True)
            self.keys[:n].copy_(keys.view(self.keys.dtype), non_blocking=True)
            self.aux[:n].copy_(aux.view(self.aux.dtype), non_blocking=True)
            if n < s:
                self.ops[n:s].fill_(OP_NOP)
                self.keys[n:s].fill_(-1)
                self.aux[n:s].zero_()
            g.replay()
            self.flags.bitwise_or_(self.out["status"][:1])
        self.batches += 1
        if self.batches % self.check_every == 0:
            self.check()
        o = self.out
        return dict(keys=o["keys"][:n], vals=o["vals"][:n], found=o["found"][:n], range_off=o["range_off"][:n + 1],
                    range_keys=o["range_keys"], range_vals=o["range_vals"], status=o["status"])

    def check(self):
        """Run the queued batches, synchronise and raise if a batch since the last check was not
        admitted."""
        self.flush()
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
            self.idx.reserve(self.sizes[-1], 0, stream=self.stream)
            self.invalidate()
            return True
        return False

    def split_chains(self, max_chain: int) -> int:
        """Elastic split of every chain longer than max_chain between graph replays (the captured
        graphs hold the bucket count and arrays, so they are re-captured when buckets were added)."""
        self.check()
        added = self.idx.split_chains(max_chain, stream=self.stream)
        if added:
            self.idx.reserve(self.sizes[-1], 0, stream=self.stream)
            self.invalidate()
        return added

    def synchronize(self):
        self.check()
