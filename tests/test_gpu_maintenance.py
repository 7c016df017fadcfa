"""GPU parity of chain maintenance: the elastic bucket split (Sec. 3.4) and the underfull-neighbour
merge (named for deletion in Sec. 5.4.1), run by the batch policy and by explicit calls, against
the structural model with the same readings.  Every comparison is of the full layout (MKBA, chain
lengths, node sizes and maxKeys, pairs in chain order) and the contents, bit-exact."""
import numpy as np
import pytest
import torch

import workload as W
from tests.gpu_util import apply_both, compare_contents, compare_layout, np_of, oracle_pair, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


def _pair(fx, kw, NS, load, split=0, merge=False, pool_nodes=0):
    dt = np.uint32 if kw == 32 else np.uint64
    vals = (load * 3 + 1).astype(dt)
    idx = fx.Index(key_bits=kw, node_size=NS, split_chains_over=split, merge_underfull=merge, pool_nodes=pool_nodes)
    idx.bulk_load(load.astype(dt), vals)
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    md.set_policy(split, merge)
    return idx, mp, md


@pytest.mark.parametrize("kw,NS,split,merge", [(64, 8, 2, True), (32, 16, 4, False), (64, 4, 1, True),
                                               (32, 8, 0, True), (64, 32, 3, True)])
def test_policy_sequences(fx, kw, NS, split, merge):
    """Hot-range and uniform batches, inserts first then deletes, through the synchronous calls and
    mixed batches; the layout is compared after every batch."""
    rng = np.random.default_rng(7 * NS + split)
    dt = np.uint32 if kw == 32 else np.uint64
    dom = 1 << 20
    load = np.unique(rng.integers(0, dom, 4000)).astype(np.uint64)
    idx, mp, md = _pair(fx, kw, NS, load, split, merge)
    for step in range(24):
        n = int(rng.integers(50, 3000))
        lo = int(rng.integers(0, dom - 5000))
        keys = (rng.integers(lo, lo + 5000, n) if step % 2 else rng.integers(0, dom, n)).astype(np.uint64)
        if step % 3 == 2:
            ops = rng.choice([W.OP_LOOKUP, W.OP_SUCC, W.OP_PRED, W.OP_INSERT, W.OP_DELETE], n).astype(np.uint8)
            apply_both(idx, mp, md, ops, keys.astype(dt), rng.integers(0, 1 << 30, n).astype(dt), kw)
        elif step < 14:
            v = (keys * 5).astype(dt)
            idx.insert(keys.astype(dt), v)
            mp.update(np.full(n, W.OP_INSERT, np.uint8), keys, v)
            md.update(np.full(n, W.OP_INSERT, np.uint8), keys, v)
        else:
            ex, _ = mp.export()
            dk = ex[rng.integers(0, ex.size, n)] if ex.size else keys
            idx.delete(dk.astype(dt))
            mp.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
            md.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
        compare_layout(idx, md)
        st = idx.stats()
        assert st["nodes_used"] == md.stats()["nodes"]
        if split:
            assert st["max_chain"] <= split
    compare_contents(idx, mp, kw)
    q = np.concatenate([mp.export()[0], rng.integers(0, dom, 2000).astype(np.uint64)])
    for op, fn in ((W.OP_SUCC, idx.successor), (W.OP_PRED, idx.predecessor)):
        k, v = fn(q.astype(dt))
        e = mp.read(np.full(q.size, op, np.uint8), q)
        same(np_of(k, kw), e["keys"], "keys")
        same(np_of(v, kw), e["vals"], "vals")
    idx.close()


@pytest.mark.parametrize("kw,NS", [(64, 8), (32, 16)])
def test_explicit_split_and_merge(fx, kw, NS):
    """flix_split_chains and flix_merge_underfull on a structure with long chains and underfull
    nodes: the counts they return and the layouts they leave match the model."""
    rng = np.random.default_rng(11)
    dt = np.uint32 if kw == 32 else np.uint64
    load = np.unique(rng.integers(0, 1 << 24, 20000)).astype(np.uint64)
    idx, mp, md = _pair(fx, kw, NS, load)
    ins = np.unique(rng.integers(1 << 20, (1 << 20) + 200000, 30000)).astype(np.uint64)   # hot range
    idx.insert(ins.astype(dt), ins.astype(dt))
    mp.update(np.full(ins.size, W.OP_INSERT, np.uint8), ins, ins)
    md.update(np.full(ins.size, W.OP_INSERT, np.uint8), ins, ins)
    dk = ins[rng.random(ins.size) < 0.8]
    idx.delete(dk.astype(dt))
    mp.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    md.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    compare_layout(idx, md)
    assert idx.stats()["max_chain"] > 8
    freed = idx.merge_underfull()
    assert freed > 0 and freed == md.merge_underfull_all()
    compare_layout(idx, md)
    assert idx.merge_underfull() == 0 == md.merge_underfull_all()      # a second pass finds nothing
    for T in (8, 3, 1):
        added = idx.split_chains(T)
        assert added == md.split_chains(T)
        compare_layout(idx, md)
        assert idx.stats()["max_chain"] <= T
    assert idx.split_chains(1) == 0
    # the split structure takes further batches, a restructure and more batches
    more = np.unique(rng.integers(0, 1 << 24, 5000)).astype(np.uint64)
    idx.insert(more.astype(dt), more.astype(dt))
    mp.update(np.full(more.size, W.OP_INSERT, np.uint8), more, more)
    md.update(np.full(more.size, W.OP_INSERT, np.uint8), more, more)
    compare_layout(idx, md)
    idx.restructure()
    md.restructure()
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    idx.close()


def test_split_policy_on_dense_range_rounds(fx):
    """X = 3%, Y = 90% insert rounds (Sec. 5.2.1) with chains split past 4 nodes, then the delete
    rounds with the merge on; layout after every round, reads at the end."""
    kw, NS, build = 64, 16, 1 << 13
    w = W.xy_rounds(0.03, 0.9, build, 3 * build, 8, seed=21, kw=kw)
    idx = fx.Index(key_bits=kw, node_size=NS, split_chains_over=4, merge_underfull=True)
    idx.bulk_load(w["build_keys"], w["build_vals"])
    mp, md = oracle_pair(kw, NS, 50, w["build_keys"], w["build_vals"])
    md.set_policy(4, True)
    for k, v in w["insert"]:
        idx.insert(k, v)
        mp.update(np.full(k.size, W.OP_INSERT, np.uint8), k, v)
        md.update(np.full(k.size, W.OP_INSERT, np.uint8), k, v)
        compare_layout(idx, md)
        assert idx.stats()["max_chain"] <= 4
    for k in w["delete"]:
        idx.delete(k)
        mp.update(np.full(k.size, W.OP_DELETE, np.uint8), k)
        md.update(np.full(k.size, W.OP_DELETE, np.uint8), k)
        compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    q = np.concatenate([w["build_keys"], w["insert"][0][0]]).astype(np.uint64)
    v, f = idx.lookup(q)
    e = mp.read(np.full(q.size, W.OP_LOOKUP, np.uint8), q)
    same(np_of(v, kw), e["vals"], "lookup.vals")
    idx.close()


def test_split_with_pool_growth(fx):
    """A small initial pool grows during the rounds; the split's second bucket arrays follow the pool."""
    rng = np.random.default_rng(3)
    kw, NS = 32, 8
    load = np.unique(rng.integers(0, 1 << 30, 2000)).astype(np.uint64)
    idx, mp, md = _pair(fx, kw, NS, load, split=2, merge=True, pool_nodes=600)
    for r in range(6):
        lo = int(rng.integers(0, (1 << 30) - (1 << 22)))
        k = np.unique(rng.integers(lo, lo + (1 << 22), 4000)).astype(np.uint64)
        idx.insert(k.astype(np.uint32), k.astype(np.uint32))
        mp.update(np.full(k.size, W.OP_INSERT, np.uint8), k, k)
        md.update(np.full(k.size, W.OP_INSERT, np.uint8), k, k)
        compare_layout(idx, md)
    assert idx.stats()["pool_nodes"] > 600
    compare_contents(idx, mp, kw)
    idx.close()


@pytest.mark.parametrize("kw", [32, 64])
def test_policy_with_heavy_nodes(fx, kw):
    """Batches with more than 2048 updates to one node (merged by all blocks) while the merge and
    the split run after every batch: the maintenance sees the heavy node's final pieces."""
    rng = np.random.default_rng(90 + kw)
    dt = np.uint32 if kw == 32 else np.uint64
    load = np.unique(rng.integers(0, 1 << 24, 2000)).astype(np.uint64)
    idx, mp, md = _pair(fx, kw, 16, load, split=4, merge=True)
    hi = np.arange((1 << 25) + 1, (1 << 25) + 1 + 3 * 15000, 3, dtype=np.uint64)    # above every key
    for b in range(3):
        # 5000 keys above everything stored: the last bucket's node takes them all (heavy)
        keys = np.concatenate([hi[b * 5000:(b + 1) * 5000], load[rng.integers(0, load.size, 300)]])
        ops = np.concatenate([np.full(keys.size - 300, W.OP_INSERT, np.uint8),
                              np.full(300, W.OP_DELETE, np.uint8)])
        aux = rng.integers(1, 1 << 30, keys.size).astype(np.uint64)
        p = rng.permutation(keys.size)
        apply_both(idx, mp, md, ops[p], keys[p].astype(dt), aux[p].astype(dt), kw)
        compare_layout(idx, md)
        assert idx.stats()["max_chain"] <= 4
    # delete most of the inserted keys in one batch: heavy deletes, then merges
    gone = hi[rng.random(hi.size) < 0.9]
    idx.delete(gone.astype(dt))
    mp.update(np.full(gone.size, W.OP_DELETE, np.uint8), gone)
    md.update(np.full(gone.size, W.OP_DELETE, np.uint8), gone)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    idx.close()
