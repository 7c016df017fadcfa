"""Serving form: continuous batching of client requests into device batches.

Requests (runs of lookup/insert/delete/... ops, in CSR order in a pinned host request ring) arrive on
a schedule.  Whenever fewer than `depth` batches are in flight, the loop coalesces every request that
has arrived (up to `max_batch` ops, and only as many inserts as the free-node budget admits) into one
device batch: the batch's ops are copied host-to-device on a copy stream while earlier batches
compute, the batch runs on the compute stream through the batched runner (a batch of at most 2048
ops through the persistent kernel, a larger one through its size class's CUDA graph), and its
results are copied back on the copy stream.  A request completes when its batch's results are on
the host; its latency is that time minus its scheduled arrival.

Admission by memory: an insert adds one key, so a batch needs at most one new node per insert (two
for node size 2); the loop keeps a budget of free nodes, charges each batch that bound when it is
dispatched and, when the batch completes, gives back the part its device status says it did not
use; it refreshes the budget from the device when it runs low, and grows the pool (re-capturing
the graphs) only when even a refreshed budget cannot admit the next request.

Batches execute in order on one compute stream, so each batch sees the effects of every earlier
batch; `log` records each batch's request range so the whole run can be replayed elsewhere.
"""
from __future__ import annotations

import collections
import time

import numpy as np
import torch

from .batched import BatchedRunner
from .flix import OP_INSERT, Index


class Server:
    """queue_depth: batches of at most QUEUE_BATCH_MAX ops go through the persistent kernel, that many
    per launch (1: each as it is dispatched; 0: every batch through the size-class graphs)."""

    def __init__(self, idx: Index, max_batch: int = 1 << 22, depth: int = 2, min_log: int = 8,
                 free_nodes_min: int = 1 << 20, queue_depth: int = 1):
        self.idx = idx
        self.max_batch = max_batch
        self.depth = depth
        self.runner = BatchedRunner(idx, max_batch=max_batch, min_log=min_log, range_per_op=1,
                                    free_nodes_min=free_nodes_min, check_every=1 << 30, queue_depth=queue_depth)
        self.compute = self.runner.stream
        self.copy = torch.cuda.Stream(device=idx.device)
        dev, dt = idx.device, idx.tdtype
        self.slots = []
        for _ in range(depth):
            self.slots.append(dict(
                ops=torch.empty(max_batch, dtype=torch.uint8, device=dev),
                keys=torch.empty(max_batch, dtype=dt, device=dev),
                aux=torch.empty(max_batch, dtype=dt, device=dev),
                dvals=torch.empty(max_batch, dtype=dt, device=dev),
                dfound=torch.empty(max_batch, dtype=torch.uint8, device=dev),
                vals=torch.empty(max_batch, dtype=dt).pin_memory(),
                found=torch.empty(max_batch, dtype=torch.uint8).pin_memory(),
                dstatus=torch.zeros(4, dtype=torch.int64, device=dev),
                status=torch.zeros(4, dtype=torch.int64).pin_memory(),
                consumed=torch.cuda.Event()))
        self.per_insert = 1 if idx.node_size >= 4 else 2
        self.budget = self._free_nodes()
        self.warmup()

    def warmup(self):
        """Capture every size class's graph now, so that no request waits for a capture."""
        for s in self.runner.sizes:
            self.runner.graph_for(s)
        self.compute.synchronize()

    def _free_nodes(self) -> int:
        self.runner.check()
        return self.idx.stats(stream=self.compute)["nodes_free"]

    def serve(self, arrival_s, req_off, ops, keys, aux, collect: bool = False):
        """Run a request schedule.  ops/keys/aux: flat host arrays in request order (CSR by req_off).
        Returns dict(latency_s per request, log of (first request, end request) per batch, wall_s,
        and, if collect, the per-op vals/found results)."""
        idx = self.idx
        R = len(arrival_s)
        ops_h = torch.from_numpy(np.ascontiguousarray(ops)).pin_memory()
        keys_h = torch.from_numpy(np.ascontiguousarray(keys).view(np.int32 if idx.kw == 32 else np.int64)).pin_memory()
        aux_h = torch.from_numpy(np.ascontiguousarray(aux).view(np.int32 if idx.kw == 32 else np.int64)).pin_memory()
        ins_cum = np.concatenate([[0], np.cumsum(ops == OP_INSERT)])
        req_off = np.asarray(req_off, dtype=np.int64)
        arrival_s = np.asarray(arrival_s, dtype=np.float64)
        lat = np.full(R, np.nan)
        res_vals = np.empty(len(keys), dtype=np.uint32 if idx.kw == 32 else np.uint64) if collect else None
        res_found = np.empty(len(keys), dtype=np.uint8) if collect else None
        inflight = collections.deque()
        log = []
        nxt = 0
        nb = 0
        t0 = time.perf_counter()
        while nxt < R or inflight:
            # retire finished batches
            while inflight and inflight[0][5].query():
                slot, a, b, lo, hi, _, charged = inflight.popleft()
                t = time.perf_counter() - t0
                lat[a:b] = t - arrival_s[a:b]
                st = slot["status"].numpy()
                if st[0] == 0:                       # admitted: return the nodes it did not need
                    self.budget += charged - int(st[2])
                if collect:
                    n = hi - lo
                    res_vals[lo:hi] = slot["vals"][:n].numpy().view(res_vals.dtype)
                    res_found[lo:hi] = slot["found"][:n].numpy()
            if nxt >= R or len(inflight) >= self.depth:
                continue
            now = time.perf_counter() - t0
            arrived = int(np.searchsorted(arrival_s, now, side="right"))
            if arrived <= nxt:
                if not inflight:
                    while time.perf_counter() - t0 < arrival_s[nxt]:
                        pass
                continue
            # coalesce arrived requests: op cap and free-node budget
            lo = int(req_off[nxt])
            b = int(np.searchsorted(req_off, lo + self.max_batch, side="right")) - 1
            b = max(min(b, arrived), nxt + 1)
            need = (ins_cum[req_off[b]] - ins_cum[lo]) * self.per_insert
            if need > self.budget:
                self.budget = self._free_nodes()       # waits for the batches in flight
                while b > nxt + 1 and (ins_cum[req_off[b]] - ins_cum[lo]) * self.per_insert > self.budget:
                    b -= 1
                need = (ins_cum[req_off[b]] - ins_cum[lo]) * self.per_insert
                if need > self.budget:                 # even one request does not fit: grow the pool
                    self.idx.reserve(self.max_batch, need + self.budget + (1 << 20), stream=self.compute)
                    self.runner.invalidate()
                    self.warmup()
                    self.budget = self._free_nodes()
            hi = int(req_off[b])
            n = hi - lo
            self.budget -= need
            slot = self.slots[nb % self.depth]
            # host -> device on the copy stream, once the slot's previous batch has consumed its inputs
            self.copy.wait_event(slot["consumed"])
            with torch.cuda.stream(self.copy):
                slot["ops"][:n].copy_(ops_h[lo:hi], non_blocking=True)
                slot["keys"][:n].copy_(keys_h[lo:hi], non_blocking=True)
                slot["aux"][:n].copy_(aux_h[lo:hi], non_blocking=True)
                ready = torch.cuda.Event()
                ready.record(self.copy)
            self.compute.wait_event(ready)
            r = self.runner.run(slot["ops"][:n], slot["keys"][:n], slot["aux"][:n])
            # results leave the runner's shared buffers at once (device to device, on the compute
            # stream), then go to the host on the copy stream while the next batch computes
            with torch.cuda.stream(self.compute):
                slot["dvals"][:n].copy_(r["vals"], non_blocking=True)
                slot["dfound"][:n].copy_(r["found"], non_blocking=True)
                slot["dstatus"].copy_(r["status"], non_blocking=True)
            slot["consumed"].record(self.compute)
            self.copy.wait_event(slot["consumed"])
            with torch.cuda.stream(self.copy):
                slot["vals"][:n].copy_(slot["dvals"][:n], non_blocking=True)
                slot["found"][:n].copy_(slot["dfound"][:n], non_blocking=True)
                slot["status"].copy_(slot["dstatus"], non_blocking=True)
                done = torch.cuda.Event()
                done.record(self.copy)
            inflight.append((slot, nxt, b, lo, hi, done, need))
            log.append((nxt, b))
            nxt = b
            nb += 1
        wall = time.perf_counter() - t0
        self.runner.check()
        out = dict(latency_s=lat, log=log, wall_s=wall, batches=nb, ops=int(req_off[-1]))
        if collect:
            out["vals"] = res_vals
            out["found"] = res_found
        return out


def plain_serve(idx: Index, arrival_s, req_off, ops, keys, aux, max_requests: int | None = None):
    """Baseline without coalescing: every request is its own flix_apply call, in arrival order."""
    R = len(arrival_s) if max_requests is None else min(max_requests, len(arrival_s))
    lat = np.empty(R)
    t0 = time.perf_counter()
    for i in range(R):
        while time.perf_counter() - t0 < arrival_s[i]:
            pass
        a, b = int(req_off[i]), int(req_off[i + 1])
        r = idx.apply(ops[a:b], keys[a:b], aux[a:b], range_capacity=1)
        r["vals"].cpu()
        lat[i] = time.perf_counter() - t0 - arrival_s[i]
    wall = time.perf_counter() - t0
    return dict(latency_s=lat, wall_s=wall, ops=int(req_off[R]))
