"""Structural invariants and cross-checks of the oracle at moderate sizes (CPU only).

* The semantic map and the structural model reach the same contents after every batch.
* The model's invariants hold after every batch (key order across buckets and chains, keys inside
  (previous maxKey, maxKey], node fill bounds, no lost or duplicated keys, node accounting).
* Restructuring leaves one half-full node per bucket and the same contents (Sec. 3.5, Sec. 6.6).
* Successor and range results agree with a linear scan over the sorted live set.
"""
import numpy as np
import pytest

import oracle
import workload as W


def test_config1_recipe_map_vs_model():
    c = W.config1(seed=0)
    kw = c["kw"]
    mp = oracle.Map(kw)
    md = oracle.Model(kw, 32, 50)
    assert mp.bulk_load(c["load_keys"], c["load_vals"]) == 0
    assert md.bulk_load(c["load_keys"], c["load_vals"]) == 0
    assert md.check(build_shape=True) == 0
    st = md.stats()
    assert st["buckets"] == (1 << 16) // 16 and st["keys"] == 1 << 16
    r, s = mp.apply(c["ops"], c["keys"], c["aux"])
    assert s == 0
    rm = md.read(c["ops"], c["keys"])
    lk = c["ops"] == W.OP_LOOKUP
    assert np.array_equal(r["vals"][lk], rm["vals"][lk])
    assert int(r["found"][lk].sum()) == 4096            # half of the 8192 lookups hit
    md.update(c["ops"], c["keys"], c["aux"])
    assert md.check() == 0
    k, v = mp.export()
    d = md.dump()
    assert np.array_equal(k, d["keys"]) and np.array_equal(v, d["vals"])
    # 4096 fresh inserts, deletes of loaded keys (some drawn twice)
    ndel = np.unique(c["keys"][c["ops"] == W.OP_DELETE]).size
    assert len(mp) == (1 << 16) + 4096 - ndel


@pytest.mark.parametrize("NS,kw", [(16, 32), (32, 32), (64, 64), (128, 64)])
def test_update_rounds_with_skew_and_restructure(NS, kw):
    rng = np.random.default_rng(NS)
    load = W.universe(kw, 1, 0, 20000)
    mp, md = oracle.Map(kw), oracle.Model(kw, NS, 50)
    mp.bulk_load(load, W.values_for(kw, load))
    md.bulk_load(load, W.values_for(kw, load))
    fresh = 20000
    for rnd in range(6):
        # inserts concentrated on a few buckets (dense range) plus uniform, then deletes
        n = 3000
        base = np.sort(load)[rng.integers(0, 19000)]
        dense = (np.uint64(base) + rng.integers(1, 5000, n // 2).astype(np.uint64)).astype(np.uint64)
        if kw == 32:
            dense = np.minimum(dense, np.uint64(2**32 - 2))
        uni = W.universe(kw, 1, fresh, fresh + n // 2).astype(np.uint64)
        fresh += n // 2
        keys = np.concatenate([dense, uni])
        k_now, _ = mp.export()
        dels = k_now[rng.integers(0, k_now.size, n)]
        ops = np.concatenate([np.full(n, W.OP_INSERT), np.full(n, W.OP_DELETE)]).astype(np.uint8)
        allk = np.concatenate([keys, dels])
        aux = np.concatenate([W.values_for(64, keys, salt=rnd).astype(np.uint64) >> np.uint64(64 - kw + 1),
                              np.zeros(n, np.uint64)])
        perm = rng.permutation(2 * n)
        ops, allk, aux = ops[perm], allk[perm], aux[perm]
        assert mp.update(ops, allk, aux) == 0
        assert md.update(ops, allk, aux) == 0
        assert md.check() == 0
        k, v = mp.export()
        d = md.dump()
        assert np.array_equal(k, d["keys"]) and np.array_equal(v, d["vals"])
        if rnd == 3:
            before = md.stats()
            rec = md.restructure()
            after = md.stats()
            assert rec == before["nodes"] - after["nodes"]
            assert after["max_chain"] == 1
            assert md.check(build_shape=True) == 0
            d2 = md.dump()
            assert np.array_equal(k, d2["keys"]) and np.array_equal(v, d2["vals"])


def test_successor_predecessor_and_range_vs_linear_scan():
    rng = np.random.default_rng(7)
    for kw in (32, 64):
        keys = np.unique(rng.integers(0, 5000, 700).astype(np.uint64))
        vals = keys * np.uint64(3) + np.uint64(1)
        mp = oracle.Map(kw)
        mp.bulk_load(keys, vals)
        q = rng.integers(0, 5100, 400).astype(np.uint64)
        hi = q + rng.integers(0, 200, 400).astype(np.uint64)
        hi[::7] = q[::7] - np.minimum(q[::7], np.uint64(1))          # some lo > hi
        r = mp.read(np.full(400, W.OP_SUCC, np.uint8), q)
        rr = mp.read(np.full(400, W.OP_RANGE, np.uint8), q, hi)
        km = (1 << kw) - 1
        allk, allv = keys.tolist(), vals.tolist()
        for i in range(400):
            succ = [j for j, x in enumerate(allk) if x >= q[i]]
            if succ:
                assert int(r["keys"][i]) == allk[succ[0]] and int(r["vals"][i]) == allv[succ[0]]
            else:
                assert int(r["keys"][i]) == km and int(r["vals"][i]) == km
            inr = [x for x in allk if q[i] <= x <= hi[i]]
            a, b = int(rr["range_off"][i]), int(rr["range_off"][i + 1])
            assert rr["range_keys"][a:b].tolist() == inr
        # predecessor: the largest stored key <= q, by a linear scan
        rp = mp.read(np.full(400, W.OP_PRED, np.uint8), q)
        for i in range(400):
            pred = [j for j, x in enumerate(allk) if x <= q[i]]
            if pred:
                assert int(rp["keys"][i]) == allk[pred[-1]] and int(rp["vals"][i]) == allv[pred[-1]]
                assert rp["found"][i] == 1
            else:
                assert int(rp["keys"][i]) == km and int(rp["vals"][i]) == km and rp["found"][i] == 0
        # the numpy sampled helpers agree with the map (they serve the full-size sampled checks)
        sk, sv, sf = oracle.sorted_successor(keys, vals, q, kw)
        assert np.array_equal(sk, r["keys"]) and np.array_equal(sv, r["vals"]) and np.array_equal(sf, r["found"])
        pk, pv, pf = oracle.sorted_predecessor(keys, vals, q, kw)
        assert np.array_equal(pk, rp["keys"]) and np.array_equal(pv, rp["vals"]) and np.array_equal(pf, rp["found"])
        cnt = oracle.sorted_range_counts(keys, q, hi)
        assert np.array_equal(cnt, np.diff(rr["range_off"]))


def _scan_lookup(allk, allv, x, km):
    """Lookup by a linear scan of the stored pairs: the definition, written out."""
    for k, v in zip(allk, allv):
        if k == x:
            return v, 1
    return km, 0


@pytest.mark.parametrize("kw", [32, 64])
def test_sorted_lookup_vs_map_and_linear_scan(kw):
    # sorted_lookup checks the full-size sampled and the every-output GPU lookups; here it is
    # compared with the ordered map and with a linear scan: hits, misses, the keys next to the
    # reserved KEY_MAX, the smallest key, and an empty key set
    km = (1 << kw) - 1
    rng = np.random.default_rng(11 + kw)
    keys = np.unique(np.concatenate([rng.integers(0, 3000, 300).astype(np.uint64),
                                     np.array([0, km - 1, km - 2], np.uint64)]))
    vals = (keys * np.uint64(7) + np.uint64(3)) & np.uint64(km - 1)
    q = np.concatenate([keys[rng.integers(0, keys.size, 200)], rng.integers(0, 3100, 200).astype(np.uint64),
                        np.array([0, 1, km - 1, km - 2, km - 3, km], np.uint64)])
    allk, allv = keys.tolist(), vals.tolist()
    for sk, sv in ((keys, vals), (np.zeros(0, np.uint64), np.zeros(0, np.uint64))):
        lv, lf = oracle.sorted_lookup(sk, sv, q, kw)
        mp = oracle.Map(kw)
        mp.bulk_load(sk, sv)
        r = mp.read(np.full(q.size, W.OP_LOOKUP, np.uint8), q)
        assert np.array_equal(lv, r["vals"]) and np.array_equal(lf, r["found"])
        for i in range(q.size):
            v, f = _scan_lookup(sk.tolist(), sv.tolist(), int(q[i]), km)
            assert int(lv[i]) == v and int(lf[i]) == f
        if sk.size:
            assert int(lf.sum()) >= 200                       # every drawn stored key is a hit
            assert int(lv[-1]) == km and lf[-1] == 0          # KEY_MAX itself is never stored
            assert int(lv[-4]) == allv[allk.index(km - 1)] and lf[-4] == 1
        else:
            assert not lf.any() and (lv == np.uint64(km)).all()
    # the successor and predecessor helpers on an empty set and next to KEY_MAX
    for fn in (oracle.sorted_successor, oracle.sorted_predecessor):
        ek, ev, ef = fn(np.zeros(0, np.uint64), np.zeros(0, np.uint64), q, kw)
        assert not ef.any() and (ek == np.uint64(km)).all() and (ev == np.uint64(km)).all()
    sk_, sv_, sf_ = oracle.sorted_successor(keys, vals, np.array([km - 1, km], np.uint64), kw)
    assert sk_.tolist() == [km - 1, km] and sf_.tolist() == [1, 0]
    pk_, pv_, pf_ = oracle.sorted_predecessor(keys, vals, np.array([km, 0], np.uint64), kw)
    assert pk_.tolist() == [km - 1, 0] and pf_.tolist() == [1, 1]


def test_generators_are_deterministic_and_distinct():
    a = W.universe(64, 5, 0, 10000)
    b = W.universe(64, 5, 0, 10000)
    assert np.array_equal(a, b) and np.unique(a).size == a.size
    c = W.universe(64, 5, 10000, 20000)
    assert np.intersect1d(a, c).size == 0
    a32 = W.universe(32, 5, 0, 1 << 18)
    assert np.unique(a32).size == a32.size and (a32 != np.uint32(0xFFFFFFFF)).all()
    z = W.zipf(1, 2, 200000, 0.99, 1 << 30)
    assert z.min() >= 1 and z.max() <= 1 << 30
    # Zipf(0.99): rank 1 is about twice as frequent as rank 2
    f1, f2 = (z == 1).sum(), (z == 2).sum()
    assert 1.6 < f1 / f2 < 2.4
    s = W.scramble30(np.arange(1 << 16))
    assert np.unique(s).size == 1 << 16 and s.max() < 1 << 30
