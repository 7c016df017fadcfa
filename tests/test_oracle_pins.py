"""Pins of the CPU oracle against what the paper fixes: its worked examples and closed forms.

* Tab. 2 (Sec. 4.3.2): TL-Bulk insertion, merged node and the split into halves.
* Tab. 3 (Sec. 4.4): TL-Bulk deletion, the deletion mask, the shift-left distances and the result.
* Sec. 3.2: the initial build cuts the sorted keys into groups of p = nodesize/2; every p-th key is
  the bucket's maxBucket.
* The canonical split rule's closed form (t <= NS: one node; else floor(t/s) pieces).
"""
import numpy as np
import pytest

import oracle
from tests.conftest import read_golden


def ints(s):
    return [int(x) for x in s.split()]


def test_tab2_merge_insert_row():
    g = read_golden("tab2_tl_bulk_insert.txt")
    node, sub = ints(g["node"]), ints(g["sublist"])
    # step 3 of Tab. 2: 15, 17 and 39 are merged; 65 waits for the split
    merged = oracle.merge_insert(node, sub[:3])
    assert merged.tolist() == ints(g["step3"])
    # a key already present is not inserted a second time
    assert oracle.merge_insert(node, [25, 30]).tolist() == node


def test_tab2_split_through_model():
    g = read_golden("tab2_tl_bulk_insert.txt")
    NS = int(g["node_size"])
    m = oracle.Model(32, NS, fill_pct=100)        # p = NS: the five keys form one node
    node = ints(g["node"])
    assert m.bulk_load(node, [k + 1000 for k in node]) == 0
    sub = ints(g["sublist"])
    assert m.update([oracle.OP_INSERT] * len(sub), sub, [k + 1000 for k in sub]) == 0
    d = m.dump()
    assert d["chain_len"].tolist() == [2]
    first, second = ints(g["split_first"]), ints(g["split_second"])
    assert d["node_size"].tolist() == [len(first), len(second)]
    assert d["keys"].tolist() == first + second
    assert d["vals"].tolist() == [k + 1000 for k in first + second]
    # the first half's maxKey is its largest key; the last node keeps the old maxKey (= maxBucket)
    assert d["node_bound"].tolist() == [first[-1], oracle.key_max(32)]
    assert m.check() == 0


def test_tab3_delete_compaction():
    g = read_golden("tab3_tl_bulk_delete.txt")
    node, dels = ints(g["node"]), ints(g["delete"])
    out, shift = oracle.delete_compact(node, dels)
    assert out.tolist() == ints(g["final"])
    assert shift.tolist() == ints(g["shift"])
    assert [1 if s < 0 else 0 for s in shift.tolist()] == ints(g["mask"])


def test_tab3_through_model():
    g = read_golden("tab3_tl_bulk_delete.txt")
    NS = int(g["node_size"])
    m = oracle.Model(64, NS, fill_pct=100)
    node = ints(g["node"])
    m.bulk_load(node, [3 * k for k in node])
    dels = ints(g["delete"])
    m.update([oracle.OP_DELETE] * len(dels), dels)
    d = m.dump()
    assert d["keys"].tolist() == ints(g["final"])
    assert d["vals"].tolist() == [3 * k for k in ints(g["final"])]
    assert d["node_size"].tolist() == [len(ints(g["final"]))]
    assert m.check() == 0


def test_build_example_sec32():
    g = read_golden("build_sec32.txt")
    NS, fill = int(g["node_size"]), int(g["fill_pct"])
    keys = ints(g["keys"])
    for kw in (32, 64):
        m = oracle.Model(kw, NS, fill)
        m.bulk_load(keys, keys)
        d = m.dump()
        km = oracle.key_max(kw)
        exp_mkba = [km if x == "KEY_MAX" else int(x) for x in g["mkba"].split()]
        assert d["mkba"].tolist() == exp_mkba
        groups = [ints(x) for x in g["sorted_groups"].split("|")]
        assert d["node_size"].tolist() == [len(x) for x in groups]
        assert d["keys"].tolist() == sum(groups, [])
        assert d["node_bound"].tolist() == exp_mkba           # one node per bucket after a build
        assert d["chain_len"].tolist() == [1] * len(groups)
        assert m.check(build_shape=True) == 0


@pytest.mark.parametrize("NS", [2, 4, 8, 16, 32, 64, 128])
def test_canonical_layout_closed_form(NS):
    s = NS // 2
    assert oracle.canonical_layout(0, NS) == []
    for t in range(1, 5 * NS + 3):
        ps = oracle.canonical_layout(t, NS)
        assert sum(ps) == t
        if t <= NS:
            assert ps == [t]
        else:
            q = t // s
            assert len(ps) == q
            assert ps[:-1] == [s] * (q - 1)
            assert s <= ps[-1] < NS or (NS == 2 and ps[-1] == 1)


def test_empty_build_and_reserved_key():
    for kw in (32, 64):
        m = oracle.Model(kw, 8)
        assert m.bulk_load([], []) == 0
        d = m.dump()
        assert d["mkba"].tolist() == [oracle.key_max(kw)]
        assert d["chain_len"].tolist() == [1] and d["node_size"].tolist() == [0]
        assert m.check() == 0
        # KEY_MAX is reserved: rejected by the build and by inserts, state unchanged
        assert m.bulk_load([1, oracle.key_max(kw)], [1, 2]) == -1
        assert m.update([oracle.OP_INSERT], [oracle.key_max(kw)], [5]) == -1
        mp = oracle.Map(kw)
        assert mp.bulk_load([oracle.key_max(kw)], [0]) == -1
        assert mp.update([oracle.OP_INSERT], [oracle.key_max(kw)], [5]) == -1
        assert len(mp) == 0


def test_bulk_load_duplicates_keep_first():
    for kw in (32, 64):
        mp = oracle.Map(kw)
        mp.bulk_load([5, 3, 5, 9, 3], [50, 30, 51, 90, 31])
        k, v = mp.export()
        assert k.tolist() == [3, 5, 9] and v.tolist() == [30, 50, 90]
        m = oracle.Model(kw, 4)
        m.bulk_load([5, 3, 5, 9, 3], [50, 30, 51, 90, 31])
        d = m.dump()
        assert d["keys"].tolist() == [3, 5, 9] and d["vals"].tolist() == [30, 50, 90]


def test_successor_is_greater_or_equal():
    # Sec. 6.5 defines successor as the smallest stored key k' >= k
    mp = oracle.Map(32)
    mp.bulk_load([10, 20, 30], [1, 2, 3])
    r = mp.read([oracle.OP_SUCC] * 5, [5, 10, 11, 30, 31])
    km = oracle.key_max(32)
    assert r["keys"].tolist() == [10, 10, 20, 30, km]
    assert r["vals"].tolist() == [1, 1, 2, 3, km]
    assert r["found"].tolist() == [1, 1, 1, 1, 0]


def test_range_inclusive_and_empty():
    mp = oracle.Map(64)
    mp.bulk_load([10, 20, 30, 40], [1, 2, 3, 4])
    ops = [oracle.OP_RANGE] * 4
    r = mp.read(ops, [10, 11, 41, 30], [30, 19, 50, 20])
    assert r["range_off"].tolist() == [0, 3, 3, 3, 3]
    assert r["range_keys"].tolist() == [10, 20, 30]
    assert r["range_vals"].tolist() == [1, 2, 3]


def test_mixed_batch_snapshot_reads():
    # reads see the state before the batch, whatever their position in it
    mp = oracle.Map(32)
    mp.bulk_load([10], [100])
    ops = [oracle.OP_DELETE, oracle.OP_LOOKUP, oracle.OP_INSERT, oracle.OP_LOOKUP]
    r, st = mp.apply(ops, [10, 10, 20, 20], [0, 0, 200, 0])
    assert st == 0
    assert r["vals"].tolist()[1] == 100 and r["found"].tolist() == [0, 1, 0, 0]
    k, v = mp.export()
    assert k.tolist() == [20] and v.tolist() == [200]


def test_model_keeps_first_node_when_bucket_empties():
    # Worked by hand from Sec. 3.2 (build), the split rule and Sec. 4.4 (an emptied node leaves the
    # chain, unless the bucket would have no node left).  NS 4, p 2: buckets [10 20] [30 40] [50 60],
    # maxBucket 20, 40, KEY_MAX; nodes 0, 1, 2.
    km = oracle.key_max(32)
    m = oracle.Model(32, 4, 50)
    m.bulk_load([10, 20, 30, 40, 50, 60], [1, 2, 3, 4, 5, 6])
    assert m.stats()["nodes"] == 3
    # bucket 1 takes 31..35: merged run 30 31 32 33 34 35 40 (t = 7 > 4) becomes floor(7/2) = 3
    # pieces of 2, 2 and 3 keys, maxKeys 31, 33 and the old 40; two nodes come from the pool
    m.update([oracle.OP_INSERT] * 5, [31, 32, 33, 34, 35], [31, 32, 33, 34, 35])
    d0 = m.dump()
    assert d0["chain_len"].tolist() == [1, 3, 1]
    assert d0["node_size"].tolist() == [2, 2, 2, 3, 2]
    assert d0["node_bound"].tolist() == [20, 31, 33, 40, km]
    assert m.stats()["nodes"] == 5
    # every key of bucket 1 leaves: the chain's first node stays, empty, as the bucket's only node,
    # with maxKey = maxBucket 40; the other two go back to the free stack
    m.update([oracle.OP_DELETE] * 7, [30, 31, 32, 33, 34, 35, 40])
    d = m.dump()
    assert d["chain_len"].tolist() == [1, 1, 1]
    assert d["node_size"].tolist() == [2, 0, 2]
    assert d["node_bound"].tolist() == [20, 40, km]
    assert d["mkba"].tolist() == [20, 40, km]
    assert m.stats()["nodes"] == 3 and m.stats()["max_chain"] == 1
    assert m.check() == 0
    # the emptied bucket still routes its range: successor of 25 is in bucket 2, an insert lands in
    # the kept node, and the freed nodes are reused before the pool grows
    r = m.read([oracle.OP_SUCC, oracle.OP_LOOKUP], [25, 40])
    assert r["keys"].tolist()[0] == 50 and r["found"].tolist() == [1, 0]
    m.update([oracle.OP_INSERT] * 3, [36, 37, 38], [36, 37, 38])
    d1 = m.dump()
    assert d1["chain_len"].tolist() == [1, 1, 1] and d1["node_size"].tolist() == [2, 3, 2]
    m.update([oracle.OP_INSERT] * 3, [11, 12, 13], [11, 12, 13])   # 10 11 12 13 20: pieces 2 and 3
    assert m.dump()["chain_len"].tolist() == [2, 1, 1] and m.stats()["nodes"] == 4
    assert m.check() == 0
    # the last bucket: its chain's last node leaves, maxBucket passes to the new last node
    m2 = oracle.Model(32, 4, 100)
    m2.bulk_load([10, 20, 30, 40], [0] * 4)
    m2.update([oracle.OP_INSERT] * 4, [11, 12, 13, 14], [0] * 4)   # 8 keys -> pieces 2,2,... split
    d2 = m2.dump()
    assert d2["chain_len"].tolist()[0] > 1
    last = d2["keys"].tolist()[-d2["node_size"].tolist()[-1]:]
    m2.update([oracle.OP_DELETE] * len(last), last)
    d3 = m2.dump()
    assert d3["node_bound"].tolist()[-1] == oracle.key_max(32)
    assert m2.check() == 0
