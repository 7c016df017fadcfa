"""GPU parity: the CUDA path against the CPU oracle, element by element, on seeded inputs.

All results are integers, so the bar is bit-exact equality of every output array and of the
bucket/node layout (MKBA, chain lengths, node sizes, maxKeys, keys and values in chain order).
Sizes span several sort tiles (4096 items), partition tiles (2048 merged items) and ragged tails.
"""
import numpy as np
import pytest
import torch

import oracle
import workload as W
from tests.gpu_util import (apply_both, compare_contents, compare_layout, np_of, oracle_pair, policy_restructure,
                            same)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


@pytest.mark.parametrize("sort_variant", [1, 2])
def test_config1_mixed_batch(fx, sort_variant):
    c = W.config1(seed=0)
    kw = c["kw"]
    idx = fx.Index(key_bits=kw, node_size=32, sort_variant=sort_variant)
    idx.bulk_load(c["load_keys"], c["load_vals"])
    mp, md = oracle_pair(kw, 32, 50, c["load_keys"], c["load_vals"])
    compare_layout(idx, md)
    apply_both(idx, mp, md, c["ops"], c["keys"], c["aux"], kw)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)


def test_config1_homogeneous_batches(fx):
    c = W.config1(seed=0)
    kw = c["kw"]
    idx = fx.Index(key_bits=kw, node_size=32)
    idx.bulk_load(c["load_keys"], c["load_vals"])
    mp, md = oracle_pair(kw, 32, 50, c["load_keys"], c["load_vals"])
    ops, keys, aux = c["ops"], c["keys"], c["aux"]
    lk = keys[ops == W.OP_LOOKUP]
    v, f = idx.lookup(lk)
    e = mp.read(np.full(lk.size, W.OP_LOOKUP), lk)
    same(np_of(v, kw), e["vals"], "lookup.vals")
    same(f.cpu().numpy(), e["found"], "lookup.found")
    ik, iv = keys[ops == W.OP_INSERT], aux[ops == W.OP_INSERT]
    idx.insert(ik, iv)
    mp.update(np.full(ik.size, W.OP_INSERT), ik, iv)
    md.update(np.full(ik.size, W.OP_INSERT), ik, iv)
    compare_layout(idx, md)
    dk = keys[ops == W.OP_DELETE]
    idx.delete(dk)
    mp.update(np.full(dk.size, W.OP_DELETE), dk)
    md.update(np.full(dk.size, W.OP_DELETE), dk)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    sk, sv = idx.successor(lk)
    e = mp.read(np.full(lk.size, W.OP_SUCC), lk)
    same(np_of(sk, kw), e["keys"], "succ.keys")
    same(np_of(sv, kw), e["vals"], "succ.vals")


@pytest.mark.parametrize("kw,NS", [(32, 2), (64, 4), (32, 8), (64, 16), (32, 32), (64, 64), (32, 128), (64, 128)])
def test_random_mixed_sequences(fx, kw, NS):
    _random_mixed_sequence(fx, kw, NS, one_pass=True)


@pytest.mark.parametrize("kw,NS", [(32, 8), (64, 64)])
def test_random_mixed_sequences_two_pass_restructure(fx, kw, NS):
    """The same sequences with the restructure that gathers to scratch, then cuts."""
    _random_mixed_sequence(fx, kw, NS, one_pass=False)


def _random_mixed_sequence(fx, kw, NS, one_pass):
    rng = np.random.default_rng(NS * 7 + kw)
    dom = 1 << 16 if kw == 32 else 1 << 40
    load = np.unique(rng.integers(0, dom, 3000, dtype=np.uint64))
    load = load[rng.permutation(load.size)].astype(np.uint64)
    fill = 50 if NS > 2 else 100
    idx = fx.Index(key_bits=kw, node_size=NS, fill_pct=fill, restructure_in_one_pass=one_pass)
    idx.bulk_load(load.astype(np.uint32 if kw == 32 else np.uint64), (load * 3 + 1).astype(np.uint32 if kw == 32 else np.uint64))
    mp, md = oracle_pair(kw, NS, fill, load, load * 3 + 1)
    compare_layout(idx, md)
    dt = np.uint32 if kw == 32 else np.uint64
    for b in range(14):
        n = int(rng.integers(0, 9000))
        center = int(rng.integers(0, dom))
        width = dom if b % 3 else max(dom // 200, 64)
        keys = ((center + rng.integers(0, width, n)) % dom).astype(np.uint64)
        ops = rng.choice([W.OP_LOOKUP, W.OP_SUCC, W.OP_PRED, W.OP_RANGE, W.OP_INSERT, W.OP_INSERT, W.OP_DELETE,
                          W.OP_DELETE, W.OP_NOP], n).astype(np.uint8)
        # some deletes and lookups of stored keys, some repeated keys inside the batch
        kk, _ = mp.export()
        if kk.size and n:
            pick = rng.random(n) < 0.4
            keys[pick] = kk[rng.integers(0, kk.size, int(pick.sum()))]
            rep = rng.random(n) < 0.05
            keys[rep] = keys[0]
        aux = np.where(ops == W.OP_RANGE, np.minimum(keys + rng.integers(0, dom // 500 + 2, n).astype(np.uint64),
                                                     np.uint64(dom)),
                       rng.integers(0, 1 << 30, n).astype(np.uint64))
        aux[(ops == W.OP_RANGE) & (rng.random(n) < 0.05)] = 0          # some lo > hi
        apply_both(idx, mp, md, ops, keys.astype(dt), aux.astype(dt), kw)
        compare_layout(idx, md)
        if b % 5 == 4:
            idx.restructure()
            md.restructure()
            compare_layout(idx, md)
    compare_contents(idx, mp, kw)


def test_read_scale_small(fx):
    kw = 64
    c = W.read_scale(seed=2000, n_load=1 << 18, batch=(1 << 16) + 37, n_range=(1 << 12) + 5, max_len=1000)
    idx = fx.Index(key_bits=kw, node_size=64)
    idx.bulk_load(c["load_keys"], c["load_vals"])
    mp = oracle.Map(kw)
    mp.bulk_load(c["load_keys"], c["load_vals"])
    q = c["queries"]
    v, f = idx.lookup(q)
    e = mp.read(np.full(q.size, W.OP_LOOKUP), q)
    same(np_of(v, kw), e["vals"], "lookup.vals")
    same(f.cpu().numpy(), e["found"], "lookup.found")
    assert abs(e["found"].mean() - 0.7) < 0.01
    sk, sv = idx.successor(q)
    e = mp.read(np.full(q.size, W.OP_SUCC), q)
    same(np_of(sk, kw), e["keys"], "succ.keys")
    same(np_of(sv, kw), e["vals"], "succ.vals")
    lo, hi = c["range_lo"], c["range_hi"]
    off, rk, rv = idx.range(lo, hi)
    e = mp.read(np.full(lo.size, W.OP_RANGE), lo, hi)
    same(off.cpu().numpy().view(np.uint64), e["range_off"], "range.off")
    same(np_of(rk, kw), e["range_keys"], "range.keys")
    same(np_of(rv, kw), e["range_vals"], "range.vals")


@pytest.mark.parametrize("dist", ["uniform", "zipf", "zipf_dense", "sequential"])
def test_update_heavy_small(fx, dist):
    kw, NS = 32, 32
    ins, deletes = W.update_heavy(dist, seed=3000, n_batches=10, batch=(1 << 13) + 3, n_del_batches=4)
    idx = fx.Index(key_bits=kw, node_size=NS)
    mp, md = oracle_pair(kw, NS, 50, np.zeros(0, np.uint32), np.zeros(0, np.uint32))
    compare_layout(idx, md)
    for k, v in ins:
        idx.insert(k, v)
        mp.update(np.full(k.size, W.OP_INSERT), k, v)
        md.update(np.full(k.size, W.OP_INSERT), k, v)
        compare_layout(idx, md)
        policy_restructure(idx, md)
        compare_layout(idx, md)
    stored, _ = mp.export()
    for d in deletes(stored.astype(np.uint32)):
        idx.delete(d)
        mp.update(np.full(d.size, W.OP_DELETE), d)
        md.update(np.full(d.size, W.OP_DELETE), d)
        compare_layout(idx, md)
    idx.restructure()
    md.restructure()
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)


def test_edge_cases(fx):
    for kw in (32, 64):
        dt = np.uint32 if kw == 32 else np.uint64
        km = (1 << kw) - 1
        idx = fx.Index(key_bits=kw, node_size=8)
        # empty index
        v, f = idx.lookup(np.array([0, 5, km], dt))
        assert np_of(v, kw).tolist() == [km] * 3 and f.cpu().tolist() == [0, 0, 0]
        sk, sv = idx.successor(np.array([0, km], dt))
        assert np_of(sk, kw).tolist() == [km, km]
        off, rk, rv = idx.range(np.array([0], dt), np.array([km], dt))
        assert off.cpu().tolist() == [0, 0]
        # empty batches
        idx.insert(np.zeros(0, dt), np.zeros(0, dt))
        idx.delete(np.zeros(0, dt))
        v, f = idx.lookup(np.zeros(0, dt))
        assert v.numel() == 0
        # reserved key rejected, structure unchanged
        idx.insert(np.array([1, 2, 3], dt), np.array([10, 20, 30], dt))
        before = idx.dump_layout()
        with pytest.raises(fx.FlixError) as ei:
            idx.insert(np.array([4, km], dt), np.array([1, 1], dt))
        assert ei.value.code == -1
        with pytest.raises(fx.FlixError):
            idx.bulk_load(np.array([km], dt), np.array([0], dt))
        after = idx.dump_layout()
        for fld in before:
            same(before[fld], after[fld], "unchanged." + fld)
        # duplicates in a bulk load keep the first pair
        idx.bulk_load(np.array([9, 7, 9, 7], dt), np.array([1, 2, 3, 4], dt))
        k, vv = idx.export()
        assert np_of(k, kw).tolist() == [7, 9] and np_of(vv, kw).tolist() == [2, 1]
        # lookup / delete of KEY_MAX is a miss / no-op
        idx.delete(np.array([km], dt))
        v, f = idx.lookup(np.array([km], dt))
        assert f.cpu().tolist() == [0]
        # range capacity too small
        L = fx.load()
        import ctypes
        lo = torch.tensor([0], dtype=idx.tdtype, device="cuda")
        hi = torch.tensor([-1], dtype=idx.tdtype, device="cuda")
        offs = torch.empty(2, dtype=torch.int64, device="cuda")
        rk = torch.empty(1, dtype=idx.tdtype, device="cuda")
        tot = ctypes.c_uint64(0)
        code = L.flix_range(idx._h, ctypes.c_void_p(lo.data_ptr()), ctypes.c_void_p(hi.data_ptr()), 1,
                            ctypes.c_void_p(offs.data_ptr()), ctypes.c_void_p(rk.data_ptr()),
                            ctypes.c_void_p(rk.data_ptr()), 1, ctypes.byref(tot), None)
        torch.cuda.synchronize()
        assert code == -2 and tot.value == 2


def test_pool_exhaustion_leaves_structure_unchanged(fx):
    kw = 32
    dt = np.uint32
    idx = fx.Index(key_bits=kw, node_size=4, pool_nodes=8, grow=False)
    idx.bulk_load(np.arange(1, 9, dtype=dt), np.arange(1, 9, dtype=dt))     # 4 buckets of 2 keys
    before = idx.dump_layout()
    with pytest.raises(fx.FlixError) as ei:
        idx.insert(np.arange(100, 140, dtype=dt), np.arange(40, dtype=dt))
    assert ei.value.code == -2
    after = idx.dump_layout()
    for fld in before:
        same(before[fld], after[fld], "unchanged." + fld)
    # with growth on, the same batch succeeds and matches the model
    idx2 = fx.Index(key_bits=kw, node_size=4, pool_nodes=8, grow=True)
    idx2.bulk_load(np.arange(1, 9, dtype=dt), np.arange(1, 9, dtype=dt))
    md = oracle.Model(kw, 4, 50)
    md.bulk_load(np.arange(1, 9), np.arange(1, 9))
    idx2.insert(np.arange(100, 140, dtype=dt), np.arange(40, dtype=dt))
    md.update(np.full(40, W.OP_INSERT), np.arange(100, 140), np.arange(40))
    compare_layout(idx2, md)
    assert idx2.stats()["pool_nodes"] > 8


@pytest.mark.slow
def test_read_scale_full_size_sampled(fx):
    """The read-scale workload at full size (2^26 u64 keys, NS = 64, 2^24 queries, 2^18 ranges) in
    the launch configuration the benchmark times; sampled outputs checked against the oracle's
    definitions over the sorted stored set."""
    kw = 64
    c = W.read_scale(seed=2000)
    idx = fx.Index(key_bits=kw, node_size=64)
    keys_d = torch.from_numpy(c["load_keys"].view(np.int64)).cuda()
    vals_d = torch.from_numpy(c["load_vals"].view(np.int64)).cuda()
    idx.bulk_load(keys_d, vals_d)
    order = np.argsort(c["load_keys"])
    sk_all, sv_all = c["load_keys"][order], c["load_vals"][order]
    s = idx.stats()
    assert s["buckets"] == (1 << 26) // 32 and s["live_keys"] == 1 << 26 and s["max_chain"] == 1
    q = c["queries"]
    qd = torch.from_numpy(q.view(np.int64)).cuda()
    v, f = idx.lookup(qd)
    sk, sv = idx.successor(qd)
    rng = np.random.default_rng(1)
    samp = np.concatenate([rng.integers(0, q.size, 200000), np.arange(4096), np.arange(q.size - 4096, q.size)])
    ev, ef = oracle.sorted_lookup(sk_all, sv_all, q[samp], kw)
    same(np_of(v, kw)[samp], ev, "lookup.vals")
    same(f.cpu().numpy()[samp], ef, "lookup.found")
    esk, esv, _ = oracle.sorted_successor(sk_all, sv_all, q[samp], kw)
    same(np_of(sk, kw)[samp], esk, "succ.keys")
    same(np_of(sv, kw)[samp], esv, "succ.vals")
    pk, pv = idx.predecessor(qd)
    epk, epv, _ = oracle.sorted_predecessor(sk_all, sv_all, q[samp], kw)
    same(np_of(pk, kw)[samp], epk, "pred.keys")
    same(np_of(pv, kw)[samp], epv, "pred.vals")
    lo, hi = c["range_lo"], c["range_hi"]
    off, rk, rv = idx.range(lo, hi)
    offn = off.cpu().numpy().view(np.uint64)
    same(np.diff(offn), oracle.sorted_range_counts(sk_all, lo, hi), "range.counts")
    rkn, rvn = np_of(rk, kw), np_of(rv, kw)
    for i in rng.integers(0, lo.size, 2000):
        a = np.searchsorted(sk_all, lo[i], "left")
        b = np.searchsorted(sk_all, hi[i], "right")
        same(rkn[offn[i]:offn[i + 1]], sk_all[a:b], "range.keys")
        same(rvn[offn[i]:offn[i + 1]], sv_all[a:b], "range.vals")


def test_large_read_batches_every_output(fx):
    """2^24 lookups and successors on a small index: the results exceed L2, so they are delivered
    through input-position windows; every output is checked, not a sample."""
    kw = 64
    rng = np.random.default_rng(9)
    load = np.unique(rng.integers(0, 1 << 40, 1 << 16, dtype=np.uint64))
    vals = load * np.uint64(7) + np.uint64(3)
    idx = fx.Index(key_bits=kw, node_size=32)
    idx.bulk_load(load, vals)
    q = np.concatenate([load[rng.integers(0, load.size, 1 << 23)],
                        rng.integers(0, 1 << 41, 1 << 23, dtype=np.uint64)])[rng.permutation(1 << 24)]
    qd = torch.from_numpy(q.view(np.int64)).cuda()
    v, f = idx.lookup(qd)
    ev, ef = oracle.sorted_lookup(load, vals, q, kw)
    same(np_of(v, kw), ev, "lookup.vals")
    same(f.cpu().numpy(), ef, "lookup.found")
    sk, sv = idx.successor(qd)
    esk, esv, _ = oracle.sorted_successor(load, vals, q, kw)
    same(np_of(sk, kw), esk, "succ.keys")
    same(np_of(sv, kw), esv, "succ.vals")
    pk, pv = idx.predecessor(qd)
    epk, epv, _ = oracle.sorted_predecessor(load, vals, q, kw)
    same(np_of(pk, kw), epk, "pred.keys")
    same(np_of(pv, kw), epv, "pred.vals")


@pytest.mark.parametrize("one_pass", [True, False])
def test_long_chain_paths(fx, one_pass):
    """A bucket whose chain is far longer than the chain-walk bound (64 nodes): stats, export and
    restructure then put the nodes in chain order by their maxKeys instead of walking the chain."""
    kw, NS = 32, 4
    load = np.arange(10, 2000, 10, dtype=np.uint64)
    vals = load * np.uint64(3)
    idx = fx.Index(key_bits=kw, node_size=NS, restructure_in_one_pass=one_pass)
    idx.bulk_load(load.astype(np.uint32), vals.astype(np.uint32))
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    # 600 keys above every stored key all land in the last bucket: a chain of ~300 nodes
    ins = np.arange(5000, 5600, dtype=np.uint64)
    iv = ins + np.uint64(1)
    for o, k, v in ((W.OP_INSERT, ins, iv), (W.OP_DELETE, ins[::7], None)):
        ops = np.full(k.size, o, np.uint8)
        if o == W.OP_INSERT:
            idx.insert(k.astype(np.uint32), v.astype(np.uint32))
        else:
            idx.delete(k.astype(np.uint32))
        mp.update(ops, k, v)
        md.update(ops, k, v)
        compare_layout(idx, md)
    s, e = idx.stats(), md.stats()
    assert s["max_chain"] > 64
    assert (s["max_chain"], s["live_keys"], s["nodes_used"]) == (e["max_chain"], e["keys"], e["nodes"])
    compare_contents(idx, mp, kw)
    idx.restructure()
    md.restructure()
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    assert idx.stats()["max_chain"] == 1


@pytest.mark.parametrize("kw,NS", [(32, 16), (64, 64), (32, 128)])
def test_heavy_node_batches(fx, kw, NS):
    """More than 2048 updates routed to one node (keys above every stored key land in the last
    bucket): the node is merged by a block of its own.  Mixed ops: inserts of present and absent
    keys, deletes of present and absent keys, upserts (delete then insert) of both."""
    rng = np.random.default_rng(NS + kw)
    dt = np.uint32 if kw == 32 else np.uint64
    load = np.arange(10, 4000, 10, dtype=np.uint64)
    vals = load * np.uint64(3)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(load.astype(dt), vals.astype(dt))
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    hi_keys = np.arange(100000, 100000 + 20000, 2, dtype=np.uint64)          # above every stored key
    for b in range(3):
        keys = rng.choice(hi_keys, 6000)
        ops = rng.choice([W.OP_INSERT, W.OP_INSERT, W.OP_DELETE], keys.size).astype(np.uint8)
        aux = rng.integers(1, 1 << 30, keys.size).astype(np.uint64)
        apply_both(idx, mp, md, ops, keys.astype(dt), aux.astype(dt), kw)
        compare_layout(idx, md)
        if b == 1:
            idx.restructure()
            md.restructure()
            compare_layout(idx, md)
    # homogeneous heavy batches too
    ins = np.arange(200001, 200001 + 2 * 5000, 2, dtype=np.uint64)
    idx.insert(ins.astype(dt), (ins * np.uint64(5)).astype(dt))
    mp.update(np.full(ins.size, W.OP_INSERT, np.uint8), ins, ins * np.uint64(5))
    md.update(np.full(ins.size, W.OP_INSERT, np.uint8), ins, ins * np.uint64(5))
    compare_layout(idx, md)
    dk = ins[::3]
    idx.delete(dk.astype(dt))
    mp.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    md.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)


@pytest.mark.parametrize("kw,NS", [(32, 2), (64, 8)])
def test_predecessor_edges(fx, kw, NS):
    """Predecessor below every key, at every stored key, between keys, and across buckets emptied by
    deletes (their only node stays empty, so the walk continues into earlier buckets)."""
    dt = np.uint32 if kw == 32 else np.uint64
    load = np.arange(100, 100 + 10 * 400, 10, dtype=np.uint64)
    vals = load + np.uint64(7)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(load.astype(dt), vals.astype(dt))
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    # empty a run of buckets in the middle and some single keys elsewhere
    dk = np.concatenate([load[100:260], load[::37]])
    idx.delete(dk.astype(dt))
    mp.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    md.update(np.full(dk.size, W.OP_DELETE, np.uint8), dk)
    compare_layout(idx, md)
    q = np.concatenate([np.arange(0, 4200, 3, dtype=np.uint64), load, np.array([0, 99, 100, 101], np.uint64)])
    pk, pv = idx.predecessor(q.astype(dt))
    e = mp.read(np.full(q.size, W.OP_PRED, np.uint8), q)
    same(np_of(pk, kw), e["keys"], "pred.keys")
    same(np_of(pv, kw), e["vals"], "pred.vals")
    em = md.read(np.full(q.size, W.OP_PRED, np.uint8), q)
    same(em["keys"], e["keys"], "model.pred.keys")


@pytest.mark.parametrize("kw", [32, 64])
def test_heavy_nodes_across_chunks(fx, kw):
    """Heavy nodes are merged in chunks of 2048 updates spread over blocks.  A node of 20 keys gets
    9000 updates: node keys sit exactly on the first chunk boundary (one deleted, one upserted),
    between two chunks, below and above every update, and one is inserted again while present.
    Then two heavy nodes in one chain, then a heavy node that only deletes (it empties and leaves
    the chain)."""
    rng = np.random.default_rng(40 + kw)
    dt = np.uint32 if kw == 32 else np.uint64
    NS = 64
    top = (1 << 31) if kw == 32 else (1 << 40)
    u = np.unique(rng.integers(1 << 20, top, 12000, dtype=np.uint64))[:9000]
    while u[4096] - u[4095] < 2:
        u[4096:] += np.uint64(2)
    extra = np.setdiff1d(np.unique(rng.integers(1 << 20, top, 40, dtype=np.uint64)), u)[:15]
    load = np.unique(np.concatenate([[5, u[2047], u[2048], u[4095] + 1, u[6000], u[-1] + 100], extra])).astype(np.uint64)
    vals = (load * np.uint64(7)).astype(dt).astype(np.uint64)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(load.astype(dt), vals.astype(dt))
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    assert idx.stats()["buckets"] == 1
    ops = np.full(u.size, W.OP_INSERT, np.uint8)
    ops[2047] = W.OP_DELETE
    keys = u.copy()
    aux = rng.integers(1, 1 << 30, u.size).astype(np.uint64)
    # upsert of u[2048] (present): delete then insert; deletes of absent keys above every update key,
    # so that u[i] stays the i-th update of the node and u[2047] / u[2048] end / start a chunk
    absent = u[-1] + np.uint64(200) + np.arange(0, 900, 3, dtype=np.uint64)
    keys = np.concatenate([keys, u[2048:2049], absent])
    ops = np.concatenate([ops, np.array([W.OP_INSERT], np.uint8), np.full(absent.size, W.OP_DELETE, np.uint8)])
    ops[2048] = W.OP_DELETE
    aux = np.concatenate([aux, np.array([12345], np.uint64), np.zeros(absent.size, np.uint64)])
    p = rng.permutation(keys.size)
    apply_both(idx, mp, md, ops[p], keys[p].astype(dt), aux[p].astype(dt), kw)
    compare_layout(idx, md)
    d = md.dump()
    # two heavy nodes in one chain: 3000 keys inside the range of the chain's 100th node, 3000 above all
    lo_b, hi_b = int(d["node_bound"][99]), int(d["node_bound"][100])
    inside = np.unique(rng.integers(lo_b + 1, hi_b, 6000, dtype=np.uint64))
    inside = np.setdiff1d(inside, mp.export()[0])[:3000]
    above = np.arange(int(u[-1]) + 1000, int(u[-1]) + 1000 + 3000 * 3, 3, dtype=np.uint64)
    node100 = d["keys"][int(d["node_size"][:100].sum()):int(d["node_size"][:101].sum())]
    k2 = np.concatenate([inside, above, node100[::2]])
    o2 = np.concatenate([np.full(inside.size + above.size, W.OP_INSERT, np.uint8),
                         np.full(node100[::2].size, W.OP_DELETE, np.uint8)])
    a2 = rng.integers(1, 1 << 30, k2.size).astype(np.uint64)
    p = rng.permutation(k2.size)
    apply_both(idx, mp, md, o2[p], k2[p].astype(dt), a2[p].astype(dt), kw)
    compare_layout(idx, md)
    # a heavy node that only deletes: all keys of the chain's 50th node and 3000 absent keys in its range
    d = md.dump()
    lo_b, hi_b = int(d["node_bound"][49]), int(d["node_bound"][50])
    node50 = d["keys"][int(d["node_size"][:50].sum()):int(d["node_size"][:51].sum())]
    stored = mp.export()[0]
    gone = np.setdiff1d(np.unique(rng.integers(lo_b + 1, hi_b + 1, 8000, dtype=np.uint64)), stored)[:3000]
    k3 = np.concatenate([node50, gone])
    assert gone.size > 2048
    idx.delete(k3.astype(dt))
    mp.update(np.full(k3.size, W.OP_DELETE, np.uint8), k3)
    md.update(np.full(k3.size, W.OP_DELETE, np.uint8), k3)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    idx.close()


def test_torch_caching_allocator(fx):
    """Every device buffer of the index comes from PyTorch's caching allocator: it shows in
    torch.cuda.memory_allocated, survives pool growth, the restructure's and the split's second
    arrays and mixed batches (results against the oracle), and goes back on close."""
    rng = np.random.default_rng(77)
    kw, NS = 64, 16
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    load = np.unique(rng.integers(0, 1 << 40, 5000, dtype=np.uint64))
    vals = load * np.uint64(3)
    idx = fx.Index(key_bits=kw, node_size=NS, pool_nodes=700, allocator="torch")
    idx.bulk_load(load, vals)
    assert torch.cuda.memory_allocated() > before
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    for b in range(6):
        n = 4000
        keys = np.concatenate([rng.integers(0, 1 << 40, n // 2, dtype=np.uint64),
                               rng.integers(1 << 30, (1 << 30) + 100000, n // 2, dtype=np.uint64)])
        ops = rng.choice([W.OP_LOOKUP, W.OP_SUCC, W.OP_PRED, W.OP_INSERT, W.OP_INSERT, W.OP_DELETE], n).astype(np.uint8)
        aux = rng.integers(1, 1 << 30, n).astype(np.uint64)
        apply_both(idx, mp, md, ops, keys, aux, kw)
        compare_layout(idx, md)
        if b == 2:
            idx.restructure()
            md.restructure()
            compare_layout(idx, md)
        if b == 4:
            assert idx.split_chains(2) == md.split_chains(2)
            compare_layout(idx, md)
    assert idx.stats()["pool_nodes"] > 700
    compare_contents(idx, mp, kw)
    idx.close()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


@pytest.mark.parametrize("kw,NS", [(32, 2), (64, 8), (32, 32), (64, 64), (64, 128)])
def test_point_reads_on_chains_every_density(fx, kw, NS):
    """Lookup, successor and predecessor batches of 1/2, 4 and 64 queries per node on an index whose
    buckets are chains (after skewed inserts and some deletes): the fused read stages the nodes of a
    warp's queries in shared memory in one or two rounds, or searches them in global memory when
    the queries hit many nodes; every output against the ordered map."""
    rng = np.random.default_rng(NS + kw)
    load = W.universe(kw, 21, 0, 6000).astype(np.uint64)
    idx = fx.Index(key_bits=kw, node_size=NS)
    vals = W.values_for(kw, load)
    idx.bulk_load(load.astype(np.uint32 if kw == 32 else np.uint64), vals)
    mp = oracle.Map(kw)
    mp.bulk_load(load, vals)
    lo = int(np.sort(load)[1000])
    ins = np.unique(lo + rng.integers(1, 1 << 24, 8000).astype(np.uint64))          # a dense range: chains
    ins = ins[~np.isin(ins, load)]
    ins = np.concatenate([ins, W.universe(kw, 21, 6000, 9000).astype(np.uint64)])
    iv = W.values_for(kw, ins, salt=3)
    dt = np.uint32 if kw == 32 else np.uint64
    idx.insert(ins.astype(dt), iv)
    mp.update(np.full(ins.size, W.OP_INSERT, np.uint8), ins, iv)
    dels = ins[rng.integers(0, ins.size, 2000)]
    idx.delete(dels.astype(dt))
    mp.update(np.full(dels.size, W.OP_DELETE, np.uint8), dels)
    assert idx.stats()["max_chain"] > 1
    sk_, sv_ = mp.export()
    nodes = idx.stats()["nodes_used"]
    for per_node in (0.5, 4, 64):
        m = max(1, int(per_node * nodes))
        q = np.concatenate([sk_[rng.integers(0, sk_.size, m // 2)],
                            rng.integers(0, (1 << kw) - 1, m - m // 2, dtype=np.uint64)])
        q = q[rng.permutation(q.size)].astype(dt)
        v, f = idx.lookup(q)
        e = mp.read(np.full(q.size, W.OP_LOOKUP, np.uint8), q)
        same(np_of(v, kw), e["vals"], "lookup.vals %s" % per_node)
        same(f.cpu().numpy(), e["found"], "lookup.found %s" % per_node)
        k2, v2 = idx.successor(q)
        e = mp.read(np.full(q.size, W.OP_SUCC, np.uint8), q)
        same(np_of(k2, kw), e["keys"], "succ.keys %s" % per_node)
        same(np_of(v2, kw), e["vals"], "succ.vals %s" % per_node)
        k3, v3 = idx.predecessor(q)
        e = mp.read(np.full(q.size, W.OP_PRED, np.uint8), q)
        same(np_of(k3, kw), e["keys"], "pred.keys %s" % per_node)
        same(np_of(v3, kw), e["vals"], "pred.vals %s" % per_node)
    idx.close()
