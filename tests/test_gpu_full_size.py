"""Update-heavy batches at full size (uint32 keys, node size 32, 64 insert batches of 2^20, then 32
delete batches of a seeded 50%), with the benchmark's restructure policy: checked through a property
that holds at any size.  After insert-only batches the stored pairs are the distinct inserted keys,
each with the value of its first insert (an insert of a present key changes nothing, Sec. 3.2);
after the deletes, those minus the deleted keys.  Both expected sets come from numpy on the batches
alone."""
import numpy as np
import pytest
import torch

import workload as W
from tests.gpu_util import np_of, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


def _first_values(keys, vals):
    u, first = np.unique(keys, return_index=True)
    return u, vals[first]


@pytest.mark.parametrize("dist", ["uniform", "zipf", "sequential"])
def test_update_heavy_full_size(fx, dist):
    ins, deletes = W.update_heavy(dist, seed=3000, n_batches=64, batch=1 << 20)
    idx = fx.Index(key_bits=32, node_size=32)
    st = torch.cuda.Stream()
    restructures = 0
    for k, v in ins:
        idx.insert(torch.from_numpy(k.view(np.int32)).cuda(), torch.from_numpy(v.view(np.int32)).cuda(), stream=st)
        s = idx.stats(stream=st)
        if s["nodes_used"] > 2 * s["buckets"] or s["max_chain"] > 64:
            idx.restructure(stream=st)
            restructures += 1
    all_k = np.concatenate([k for k, _ in ins]).astype(np.uint64)
    all_v = np.concatenate([v for _, v in ins]).astype(np.uint64)
    ek, ev = _first_values(all_k, all_v)
    gk, gv = idx.export(stream=st)
    same(np_of(gk, 32), ek, "%s inserts: keys" % dist)
    same(np_of(gv, 32), ev, "%s inserts: values" % dist)
    assert idx.stats(stream=st)["live_keys"] == ek.size
    dels = deletes(ek.astype(np.uint32))
    for d in dels:
        idx.delete(torch.from_numpy(d.view(np.int32)).cuda(), stream=st)
    gone = np.concatenate(dels).astype(np.uint64)
    keep = ~np.isin(ek, gone)
    gk, gv = idx.export(stream=st)
    same(np_of(gk, 32), ek[keep], "%s deletes: keys" % dist)
    same(np_of(gv, 32), ev[keep], "%s deletes: values" % dist)
    idx.restructure(stream=st)
    s = idx.stats(stream=st)
    assert s["live_keys"] == int(keep.sum()) and s["max_chain"] == 1
    gk, _ = idx.export(stream=st)
    same(np_of(gk, 32), ek[keep], "%s restructure: keys" % dist)
    idx.close()
