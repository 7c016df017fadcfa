"""Brute-force pins of the oracle: tiny key domains, every short batch, against a plain Python dict
that applies the batch literally (reads on the snapshot by linear scans, then every insert and
delete one at a time in submission order).  It shares nothing with the oracle's code: no sorting,
no per-key grouping, no net-effect folding, no buckets.
"""
import itertools
import random

import numpy as np
import pytest

import oracle

L, S, R, I, D, P = (oracle.OP_LOOKUP, oracle.OP_SUCC, oracle.OP_RANGE, oracle.OP_INSERT, oracle.OP_DELETE,
                    oracle.OP_PRED)


def brute(state, ops, keys, aux, kw):
    km = (1 << kw) - 1
    items = sorted(state.items())
    out_k, out_v, out_f, offs, rk, rv = [], [], [], [0], [], []
    for op, k, a in zip(ops, keys, aux):
        ok, ov, of = km, km, 0
        if op == L and k in state:
            ok, ov, of = k, state[k], 1
        elif op == S:
            for kk, vv in items:
                if kk >= k:
                    ok, ov, of = kk, vv, 1
                    break
        elif op == P:
            for kk, vv in items:
                if kk <= k:
                    ok, ov, of = kk, vv, 1
        elif op == R:
            for kk, vv in items:
                if k <= kk <= a:
                    rk.append(kk)
                    rv.append(vv)
        out_k.append(ok)
        out_v.append(ov)
        out_f.append(of)
        offs.append(len(rk))
    for op, k, a in zip(ops, keys, aux):
        if op == I and k not in state:
            state[k] = a
        elif op == D:
            state.pop(k, None)
    return dict(keys=out_k, vals=out_v, found=out_f, range_off=offs, range_keys=rk, range_vals=rv)


def check_batch(mp, md, state, ops, keys, aux, kw):
    r_map, st = mp.apply(ops, keys, aux)
    assert st == 0
    # the structural model answers lookups, successors and predecessors through its buckets and chains
    rm = md.read(ops, keys)
    md.update(ops, keys, aux)
    exp = brute(state, ops, keys, aux, kw)
    for f in ("keys", "vals", "found", "range_off", "range_keys", "range_vals"):
        assert r_map[f].tolist() == exp[f], f
    for i, op in enumerate(ops):
        if op in (L, S, P):
            assert int(rm["keys"][i]) == exp["keys"][i]
            assert int(rm["vals"][i]) == exp["vals"][i]
            assert int(rm["found"][i]) == exp["found"][i]
    k, v = mp.export()
    items = sorted(state.items())
    assert k.tolist() == [x for x, _ in items] and v.tolist() == [y for _, y in items]
    d = md.dump()
    assert d["keys"].tolist() == [x for x, _ in items] and d["vals"].tolist() == [y for _, y in items]
    assert md.check() == 0


def test_single_key_runs_exhaustive():
    """Every insert/delete sequence of length <= 6 on one key, from both prior states."""
    for n in range(1, 7):
        for seq in itertools.product((I, D), repeat=n):
            for prior in (False, True):
                st = {7: 999} if prior else {}
                mp = oracle.Map(32)
                mp.bulk_load(list(st.keys()), list(st.values()))
                md = oracle.Model(32, 2)
                md.bulk_load(list(st.keys()), list(st.values()))
                ops = list(seq)
                keys = [7] * n
                aux = [100 + i for i in range(n)]
                check_batch(mp, md, dict(st), ops, keys, aux, 32)


@pytest.mark.parametrize("NS", [2, 4])
def test_all_two_op_batches_small_domain(NS):
    """Every prior subset of a 5-key domain x every batch of two ops over it."""
    dom = [1, 3, 5, 7, 9]
    singles = [(op, k) for op in (L, S, P, R, I, D) for k in range(0, 11)]
    rng = random.Random(NS)
    for mask in range(1 << len(dom)):
        prior = {k: 10 * k for j, k in enumerate(dom) if mask >> j & 1}
        for (o1, k1), (o2, k2) in itertools.product(singles, repeat=2):
            if rng.random() > 0.08:          # a fixed, seeded 8% of the 4,356 pairs per subset
                continue
            mp = oracle.Map(64)
            mp.bulk_load(list(prior), list(prior.values()))
            md = oracle.Model(64, NS)
            md.bulk_load(list(prior), list(prior.values()))
            check_batch(mp, md, dict(prior), [o1, o2], [k1, k2], [k1 + 2 if o1 == R else 500,
                                                                  k2 + 3 if o2 == R else 600], 64)


@pytest.mark.parametrize("seed", range(12))
def test_random_batch_sequences(seed):
    rng = random.Random(seed)
    kw = 32 if seed % 2 else 64
    NS = rng.choice([2, 4, 8, 16])
    fill = rng.choice([50, 50, 25, 100])
    dom = rng.choice([16, 64, 300])
    base = rng.sample(range(dom), rng.randint(0, dom // 2))
    state = {k: k * 7 + 1 for k in base}
    mp = oracle.Map(kw)
    mp.bulk_load(list(state), list(state.values()))
    md = oracle.Model(kw, NS, fill)
    md.bulk_load(list(state), list(state.values()))
    assert md.check(build_shape=True) == 0
    for b in range(25):
        n = rng.randint(0, 60)
        # skew: half of the batches hit a narrow key range
        lo = rng.randrange(dom)
        width = dom if b % 2 else max(2, dom // 10)
        ops, keys, aux = [], [], []
        for _ in range(n):
            op = rng.choice([L, S, P, R, I, I, D, D])
            k = (lo + rng.randrange(width)) % dom
            ops.append(op)
            keys.append(k)
            aux.append(k + rng.randrange(20) if op == R else rng.randrange(1 << 20))
        check_batch(mp, md, state, ops, keys, aux, kw)
        if b % 7 == 6:
            before = md.dump()["keys"].tolist()
            md.restructure()
            assert md.check(build_shape=True) == 0
            assert md.dump()["keys"].tolist() == before


@pytest.mark.parametrize("threads", [1, 3, 8])
def test_batch_synchronous_map_on_threads_equals_the_map(threads):
    """The all-core CPU baseline (reads split over threads, updates merged by key range on threads)
    gives the results and the state of the plain map after every mixed batch."""
    rng = np.random.default_rng(threads)
    for kw in (32, 64):
        load = np.unique(rng.integers(0, 50000, 6000).astype(np.uint64))
        a, b = oracle.Map(kw), oracle.Map(kw)
        a.bulk_load(load, load * np.uint64(3))
        b.bulk_load(load, load * np.uint64(3))
        for rnd in range(6):
            n = int(rng.integers(1, 4000))
            ops = rng.choice([oracle.OP_LOOKUP, oracle.OP_SUCC, oracle.OP_PRED, oracle.OP_RANGE, oracle.OP_INSERT,
                              oracle.OP_DELETE, oracle.OP_NOP], n).astype(np.uint8)
            keys = rng.integers(0, 52000, n).astype(np.uint64)
            hit = rng.random(n) < 0.4                     # stored keys for hits, deletes and upserts
            keys[hit] = load[rng.integers(0, load.size, int(hit.sum()))]
            aux = np.where(ops == oracle.OP_RANGE, keys + rng.integers(0, 300, n).astype(np.uint64),
                           rng.integers(0, 1 << 20, n).astype(np.uint64))
            ra = a.read(ops, keys, aux)
            rb = b.read_mt(ops, keys, aux, threads=threads)
            for f in ("keys", "vals", "found", "range_off", "range_keys", "range_vals"):
                assert np.array_equal(ra[f], rb[f]), (kw, rnd, f)
            assert a.update(ops, keys, aux) == b.update_mt(ops, keys, aux, threads=threads) == 0
            ka, va = a.export()
            kb, vb = b.export()
            assert np.array_equal(ka, kb) and np.array_equal(va, vb), (kw, rnd)
