"""The single-thread path of the update kernels (one thread applies the updates of a bucket whose
chain is one node and that receives at most 8 updates which still fit the node: the paper's
single-thread kernels, Sec. 4.2) against the warp path and the structural model.

Every bucket of the batch receives its own number of updates (1 to 12) of every kind (fresh
inserts, deletes, upserts, inserts of present keys, deletes of absent keys), so that runs that fit
the node take the one-thread path and the others (more updates, or a merged run longer than the
node) take the warp path inside the same launch.  The layout (MKBA, chain lengths, node sizes,
maxKeys, keys and values in chain order) must equal the model's after each batch, with the
one-thread path enabled (bucket_threads 0) and disabled (32)."""
import numpy as np
import pytest
import torch

import oracle
import workload as W
from tests.gpu_util import compare_contents, compare_layout, oracle_pair

pytestmark = pytest.mark.gpu


MASK = (1 << 62) - 1


def light_batch(load, NS, rng, nbuckets):
    """Updates for the first nbuckets buckets of a build of `load` (sorted, p = NS/2 keys each):
    bucket i gets 1 + i % 12 updates drawn from its own key range."""
    p = NS // 2
    nbuckets = min(nbuckets, len(load) // p - 1)
    keys, ops, vals = [], [], []
    for i in range(nbuckets):
        lo = int(load[i * p]) if i > 0 else 0
        hi = int(load[i * p + p - 1])
        present = [int(x) for x in load[i * p:i * p + p]]
        for u in range(1 + i % 12):
            kind = rng.integers(0, 5)
            if kind == 0 or kind == 4:                    # fresh insert inside the bucket's range
                k = int(rng.integers(lo + 1, hi, dtype=np.uint64)) if hi - lo > 2 else lo + 1
                keys.append(k); ops.append(W.OP_INSERT); vals.append((k * 3 + 1) & MASK)
            elif kind == 1:                               # delete of a present key
                k = present[int(rng.integers(0, p))]
                keys.append(k); ops.append(W.OP_DELETE); vals.append(0)
            elif kind == 2:                               # upsert: delete then insert the same key
                k = present[int(rng.integers(0, p))]
                keys += [k, k]; ops += [W.OP_DELETE, W.OP_INSERT]; vals += [0, (k * 5 + 2) & MASK]
            else:                                         # insert of a present key (no-op)
                k = present[int(rng.integers(0, p))]
                keys.append(k); ops.append(W.OP_INSERT); vals.append(7)
    perm = rng.permutation(len(keys))
    return (np.array(ops, np.uint8)[perm], np.array(keys, np.uint64)[perm], np.array(vals, np.uint64)[perm])


@pytest.mark.parametrize("kw,NS", [(32, 8), (64, 16), (32, 32), (64, 64)])
@pytest.mark.parametrize("bucket_threads", [0, 32])
def test_light_buckets_every_update_kind(kw, NS, bucket_threads):
    import paper_2604_16725_gb300 as fx
    rng = np.random.default_rng(NS * 7 + kw + bucket_threads)
    load = np.sort(W.universe(kw, 31, 0, 1 << 14).astype(np.uint64))
    vals = W.values_for(kw, load)
    dt = np.uint32 if kw == 32 else np.uint64
    idx = fx.Index(key_bits=kw, node_size=NS, bucket_threads=bucket_threads)
    idx.bulk_load(load.astype(dt), vals)
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    for rnd in range(3):
        ops, keys, aux = light_batch(load, NS, rng, 1500)
        aux = aux & np.uint64((1 << kw) - 2)
        r = idx.apply(ops, keys.astype(dt), aux.astype(dt))
        mp.update(ops, keys, aux)
        md.update(ops, keys, aux)
        compare_layout(idx, md)
        assert md.check() == 0
        load = np.sort(mp.export()[0])[: (len(load) // (NS // 2)) * (NS // 2)]
    compare_contents(idx, mp, kw)
    idx.close()
