"""Autotuner of the batched form: node size, sort variant and threads per bucket.

For every candidate it builds an index on a held-out sample (its own seed, scaled-down preload),
runs the sample's batch stream through the batched runner, and keeps the configuration with the
highest Mops/s.  Results are cached as JSON keyed by the workload signature, so a later run with the
same signature reuses the choice.

The paper's own sweep (Sec. 5.3.3) covers node sizes {8, 14, 16, 32} and threads per block, and its
Sec. 5.3.6 finds single-thread kernels best for light rounds and tiled ones for heavy rounds.  On
this design threads per block are fixed by the kernels' occupancy; the threads that apply one
bucket's updates are the knob that remains: `bucket_threads` 0 (one thread for a light one-node
bucket, a warp otherwise) or 32 (a warp for every bucket).  The searched knobs are the node size
{16, 32, 64, 128}, the radix-sort variant (one-sweep or reduce-then-scan) and bucket_threads.
"""
from __future__ import annotations

import hashlib
import json
import os
import time

import torch

from .batched import BatchedRunner
from .flix import Index

NODE_SIZES = (16, 32, 64, 128)
SORT_VARIANTS = (1, 2)   # FLIX_SORT_ONESWEEP, FLIX_SORT_REDUCE_SCAN
BUCKET_THREADS = (0, 32)


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "flix_gb300", "tune.json")


def signature(key_bits: int, n_preload: int, batch_sizes, mix) -> str:
    h = hashlib.sha256(json.dumps([key_bits, n_preload, sorted(int(b) for b in batch_sizes), list(mix)]).encode())
    return h.hexdigest()[:16]


def _measure(key_bits, NS, sv, bt, preload_keys, preload_vals, batches, max_batch, range_per_op):
    idx = Index(key_bits=key_bits, node_size=NS, sort_variant=sv, bucket_threads=bt)
    idx.bulk_load(preload_keys, preload_vals)
    run = BatchedRunner(idx, max_batch=max_batch, min_log=8, range_per_op=range_per_op,
                        free_nodes_min=sum(int(k.numel()) for _, k, _ in batches))
    for ops, keys, aux in batches[:2]:                      # capture the graphs of the first classes
        run.run(ops, keys, aux)
    run.synchronize()
    for ops, keys, aux in batches:                          # capture every class used
        run.graph_for(run.size_for(int(keys.numel())))
    t0 = time.perf_counter()
    for ops, keys, aux in batches:
        run.run(ops, keys, aux)
    run.synchronize()
    dt = time.perf_counter() - t0
    n = sum(int(k.numel()) for _, k, _ in batches)
    idx.close()
    return n / dt / 1e6


def autotune(key_bits, preload_keys, preload_vals, batches, range_per_op=64, node_sizes=NODE_SIZES,
             sort_variants=SORT_VARIANTS, bucket_threads=BUCKET_THREADS, cache_path=None, sig=None, log=None):
    """batches: list of (ops, keys, aux) device tensors from a held-out seed.  Returns
    dict(node_size, sort_variant, bucket_threads, mops, table)."""
    cache_path = cache_path or default_cache_path()
    if sig is not None and os.path.exists(cache_path):
        try:
            cached = json.load(open(cache_path)).get(sig)
            if cached:
                return cached
        except (OSError, ValueError):
            pass
    max_batch = max(int(k.numel()) for _, k, _ in batches)
    table = []
    for NS in node_sizes:
        for sv in sort_variants:
            for bt in bucket_threads:
                mops = _measure(key_bits, NS, sv, bt, preload_keys, preload_vals, batches, max_batch, range_per_op)
                table.append(dict(node_size=NS, sort_variant=sv, bucket_threads=bt, mops=mops))
                if log:
                    log("tune NS=%d sort=%d bucket_threads=%d: %.1f Mops/s" % (NS, sv, bt, mops))
                torch.cuda.synchronize()
    best = max(table, key=lambda r: r["mops"])
    res = dict(node_size=best["node_size"], sort_variant=best["sort_variant"], bucket_threads=best["bucket_threads"],
               mops=best["mops"], table=table)
    if sig is not None:
        try:
            os.makedirs(os.path.dirname(cache_path), exist_ok=True)
            data = json.load(open(cache_path)) if os.path.exists(cache_path) else {}
            data[sig] = res
            with open(cache_path, "w") as f:
                json.dump(data, f, indent=1)
        except (OSError, ValueError):
            pass
    return res
