"""Serving form (continuous batching) against the oracle.

* Every op of every request, served under a Poisson schedule, equals the oracle replaying the same
  batch composition (the server logs which requests formed each batch).
* A request's results are the same when it is served alone and when it is served inside a mix of
  other requests whose keys are disjoint from its own (tolerance 0: all results are integers).
"""
import numpy as np
import pytest
import torch

import oracle
import workload as W
from tests.gpu_util import same

pytestmark = pytest.mark.gpu


def _preload(kw, bits, seed):
    k = W.universe(kw, seed, 0, 1 << bits)
    return k, W.values_for(kw, k)


def test_served_stream_matches_oracle_replay():
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.serve import Server
    kw, seed = 64, 5100
    req = W.serving_requests(seed=seed, kw=kw, universe_bits=17, preload_bits=16, offered_ops_per_s=2e7,
                             n_requests=3000)
    pk, pv = _preload(kw, 16, seed)
    idx = fx.Index(key_bits=kw, node_size=32)
    idx.bulk_load(pk, pv)
    srv = Server(idx, max_batch=1 << 16, depth=2, min_log=6, free_nodes_min=1 << 16)
    out = srv.serve(req["arrival_s"], req["req_off"], req["ops"], req["keys"], req["aux"], collect=True)
    assert out["batches"] > 1 and not np.isnan(out["latency_s"]).any()
    mp = oracle.Map(kw)
    mp.bulk_load(pk, pv)
    off = req["req_off"]
    for a, b in out["log"]:
        lo, hi = int(off[a]), int(off[b])
        e, st = mp.apply(req["ops"][lo:hi], req["keys"][lo:hi], req["aux"][lo:hi])
        assert st == 0
        same(out["vals"][lo:hi], e["vals"], "requests %d..%d vals" % (a, b))
        same(out["found"][lo:hi], e["found"], "requests %d..%d found" % (a, b))
    k, v = idx.export()
    ek, ev = mp.export()
    same(k.cpu().numpy().view(np.uint64), ek, "final keys")
    same(v.cpu().numpy().view(np.uint64), ev, "final vals")


def test_request_alone_equals_request_in_mix():
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.serve import Server
    kw, seed = 64, 5200
    pk, pv = _preload(kw, 15, seed)
    # the request under test: lookups, inserts and deletes on universe keys 0..511 and fresh keys
    rng = np.random.default_rng(3)
    n_a = 600
    own = np.concatenate([pk[:512], W.universe(kw, seed, 1 << 20, (1 << 20) + 256)])
    ka = own[rng.integers(0, own.size, n_a)]
    oa = rng.choice([W.OP_LOOKUP, W.OP_LOOKUP, W.OP_SUCC, W.OP_INSERT, W.OP_DELETE], n_a).astype(np.uint8)
    aa = np.where(oa == W.OP_INSERT, W.values_for(kw, ka, salt=5), 0).astype(np.uint64)
    # other requests: keys from a disjoint part of the universe (preload counters >= 1024 and fresh keys)
    others = np.concatenate([pk[1024:], W.universe(kw, seed, 1 << 21, (1 << 21) + 4096)])
    n_req, per = 200, 64
    ko = others[rng.integers(0, others.size, n_req * per)]
    oo = rng.choice([W.OP_LOOKUP, W.OP_INSERT, W.OP_DELETE], n_req * per).astype(np.uint8)
    ao = np.where(oo == W.OP_INSERT, W.values_for(kw, ko, salt=6), 0).astype(np.uint64)
    # successor queries of the request under test must not reach the other requests' keys: use lookups
    # only for keys whose successor could cross into them
    oa[oa == W.OP_SUCC] = W.OP_LOOKUP

    def serve(schedule):
        idx = fx.Index(key_bits=kw, node_size=32)
        idx.bulk_load(pk, pv)
        srv = Server(idx, max_batch=1 << 15, depth=2, min_log=6, free_nodes_min=1 << 14)
        arr, offs, ops, keys, aux = schedule
        return srv.serve(arr, offs, ops, keys, aux, collect=True)

    alone = serve((np.array([0.0]), np.array([0, n_a]), oa, ka, aa))
    # mix: the request sits in the middle of a burst of other requests arriving together
    pos = n_req // 2
    ops = np.concatenate([oo[:pos * per], oa, oo[pos * per:]])
    keys = np.concatenate([ko[:pos * per], ka, ko[pos * per:]])
    aux = np.concatenate([ao[:pos * per], aa, ao[pos * per:]])
    sizes = np.array([per] * pos + [n_a] + [per] * (n_req - pos))
    offs = np.concatenate([[0], np.cumsum(sizes)])
    arr = np.linspace(0.0, 2e-3, sizes.size)
    mix = serve((arr, offs, ops, keys, aux))
    batches_with_a = [(a, b) for a, b in mix["log"] if a <= pos < b]
    assert len(batches_with_a) == 1 and batches_with_a[0][1] - batches_with_a[0][0] > 1   # really mixed
    lo, hi = int(offs[pos]), int(offs[pos + 1])
    same(mix["vals"][lo:hi], alone["vals"], "vals alone vs in the mix")
    same(mix["found"][lo:hi], alone["found"], "found alone vs in the mix")
