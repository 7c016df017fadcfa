"""Helpers shared by the GPU parity tests: run a batch through the CUDA path and through the oracle,
and compare results element by element (all integer: bit-exact)."""
import numpy as np

import oracle


def np_of(t, kw):
    a = t.detach().cpu().numpy()
    return a.view(np.uint32 if kw == 32 else np.uint64).astype(np.uint64)


def same(a, b, what):
    a = np.asarray(a).astype(np.uint64)
    b = np.asarray(b).astype(np.uint64)
    assert a.shape == b.shape, "%s: shape %s vs %s" % (what, a.shape, b.shape)
    bad = np.nonzero(a != b)[0]
    assert bad.size == 0, "%s: %d mismatches, first at %d: %s vs %s" % (what, bad.size, bad[0], a[bad[0]], b[bad[0]])


def compare_layout(idx, model):
    d = idx.dump_layout()
    m = model.dump()
    for f in ("mkba", "chain_len", "node_size", "node_bound", "keys", "vals"):
        same(d[f], m[f], "layout." + f)


def compare_contents(idx, mp, kw):
    k, v = idx.export()
    ek, ev = mp.export()
    same(np_of(k, kw), ek, "export.keys")
    same(np_of(v, kw), ev, "export.vals")


def apply_both(idx, mp, model, ops, keys, aux, kw):
    """One mixed batch on the GPU, on the semantic map and on the structural model; compare."""
    r = idx.apply(ops, keys, aux)
    e, st = mp.apply(ops, keys, aux)
    assert st == 0
    if model is not None:
        assert model.update(ops, keys, aux) == 0
    same(np_of(r["keys"], kw), e["keys"], "apply.keys")
    same(np_of(r["vals"], kw), e["vals"], "apply.vals")
    same(r["found"].cpu().numpy(), e["found"], "apply.found")
    same(r["range_off"].cpu().numpy().view(np.uint64), e["range_off"], "apply.range_off")
    same(np_of(r["range_keys"], kw), e["range_keys"], "apply.range_keys")
    same(np_of(r["range_vals"], kw), e["range_vals"], "apply.range_vals")
    return r


def policy_restructure(idx, model=None):
    """Deterministic restructure policy: restructure when nodes > 2 * buckets or a chain > 64."""
    s = idx.stats()
    if s["nodes_used"] > 2 * s["buckets"] or s["max_chain"] > 64:
        idx.restructure()
        if model is not None:
            model.restructure()
        return True
    return False


def oracle_pair(kw, NS, fill, keys, vals):
    mp = oracle.Map(kw)
    md = oracle.Model(kw, NS, fill)
    assert mp.bulk_load(keys, vals) == 0
    assert md.bulk_load(keys, vals) == 0
    return mp, md
