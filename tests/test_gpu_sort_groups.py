"""GPU parity of batches built to reach every path of the batch sort.

The sort skips digits that are the same in every key; it may stop after the highest few varying
digits and then sorts each group of keys with an equal prefix in place (in shared memory for up to
8 items, one block with a bitonic network for up to 4096, a chunked radix sort of the remaining
digits beyond that); and it sorts by every varying digit when every prefix digit has a heavy bin.
Each case runs mixed batches through the CUDA path and through the oracle and compares every result
and the final layout bit-exactly.  A mis-sorted batch routes operations to the wrong buckets or
folds one key's operations in the wrong order (the groups below hold repeated keys with inserts,
deletes and reads interleaved), and shows up in those comparisons.
"""
import numpy as np
import pytest
import torch

import workload as W
from tests.gpu_util import apply_both, compare_contents, compare_layout, oracle_pair

pytestmark = pytest.mark.gpu

MIX = np.array([W.OP_LOOKUP, W.OP_SUCC, W.OP_INSERT, W.OP_DELETE], dtype=np.uint8)


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


def _group(rng, kw, prefix_bits, size, distinct):
    """`size` keys sharing their top `prefix_bits` bits, drawn (with repeats) from `distinct` values."""
    low_bits = kw - prefix_bits
    top = int(rng.integers(1, 1 << prefix_bits - 1)) << low_bits
    low = rng.integers(0, 1 << low_bits, distinct, dtype=np.uint64)
    return (np.uint64(top) | low[rng.integers(0, distinct, size)]).astype(np.uint64)


def _batch(rng, kw, base, groups, loaded):
    """Mixed ops over uniform `base` keys plus the group keys, shuffled; a third of the group keys
    are taken from the loaded keys so that deletes and lookups hit."""
    g = np.concatenate(groups) if groups else np.zeros(0, np.uint64)
    hit = rng.random(g.size) < 0.3
    g = g.copy()
    g[hit] = loaded[rng.integers(0, loaded.size, int(hit.sum()))]
    keys = np.concatenate([base, g]).astype(np.uint64)
    kmax = (1 << kw) - 1
    keys[keys == kmax] = kmax - 1                       # the reserved key is not a valid operand
    ops = MIX[rng.integers(0, MIX.size, keys.size)]
    aux = rng.integers(0, 1 << min(kw, 63), keys.size, dtype=np.uint64)
    p = rng.permutation(keys.size)
    dt = np.uint32 if kw == 32 else np.uint64
    return ops[p], keys[p].astype(dt), aux[p].astype(dt)


def _run(fx, kw, NS, load, batches, sort_variant=1):
    dt = np.uint32 if kw == 32 else np.uint64
    load = load.astype(dt)
    vals = (load * dt(3) + dt(1)).astype(dt)
    idx = fx.Index(key_bits=kw, node_size=NS, sort_variant=sort_variant)
    idx.bulk_load(load, vals)
    mp, md = oracle_pair(kw, NS, 50, load, vals)
    for ops, keys, aux in batches:
        apply_both(idx, mp, md, ops, keys, aux, kw)
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    idx.close()


def _uniform(rng, kw, n):
    return rng.integers(0, (1 << kw) - 1, n, dtype=np.uint64)


@pytest.mark.parametrize("sort_variant", [1, 2])
def test_prefix_groups_of_every_length(fx, sort_variant):
    """2^22 ops of 64-bit keys: the plan sorts the top 3 digits and finishes the groups: a group of
    about 5600 ops (chunked radix sort), one of about 500 (bitonic), and 200 of 1..8 (one thread)."""
    rng = np.random.default_rng(1)
    kw, n = 64, 1 << 22
    load = np.unique(_uniform(rng, kw, 1 << 16))
    groups = [_group(rng, kw, 24, 8000, 2000), _group(rng, kw, 24, 700, 300)]
    groups += [_group(rng, kw, 24, int(rng.integers(2, 9)), 4) for _ in range(200)]
    load = np.unique(np.concatenate([load, groups[0][:700], groups[1][:100]]))
    base = _uniform(rng, kw, n - sum(g.size for g in groups))
    _run(fx, kw, 64, load, [_batch(rng, kw, base, groups, load)], sort_variant)


def test_heavy_key_sorts_every_digit(fx):
    """A tenth of the batch is one key: every digit has a heavy bin and the plan sorts every digit."""
    rng = np.random.default_rng(2)
    kw, n = 64, 1 << 20
    load = np.unique(_uniform(rng, kw, 1 << 15))
    hot = np.full(n // 10, load[7], dtype=np.uint64)
    base = _uniform(rng, kw, n - hot.size)
    batches = [_batch(rng, kw, base, [hot], load) for _ in range(2)]
    _run(fx, kw, 32, load, batches)


def test_constant_high_digits_are_skipped(fx):
    """Keys in one window of 2^20 values above 2^50: the five high digits are equal everywhere."""
    rng = np.random.default_rng(3)
    kw = 64
    lo = (5 << 50) + (3 << 36)
    load = np.unique(rng.integers(lo, lo + (1 << 20), 1 << 14, dtype=np.uint64))
    base = rng.integers(lo, lo + (1 << 20), 1 << 18, dtype=np.uint64)
    _run(fx, kw, 16, load, [_batch(rng, kw, base, [], load)])


def test_all_keys_equal(fx):
    """Every op of the batch has the same key: no digit varies and one stable pass copies the batch."""
    rng = np.random.default_rng(4)
    kw = 64
    load = np.unique(_uniform(rng, kw, 5000))
    for key in (load[100], np.uint64(12345)):
        ops = MIX[rng.integers(0, MIX.size, 9000)]
        keys = np.full(9000, key, dtype=np.uint64)
        aux = rng.integers(0, 1 << 40, 9000, dtype=np.uint64)
        _run(fx, kw, 8, load, [(ops, keys, aux)])


def test_prefix_groups_32bit_keys(fx):
    """2^16 ops of 32-bit keys: the plan sorts the top 2 digits; a group of about 600 ops (bitonic)
    and 100 groups of 2..8."""
    rng = np.random.default_rng(5)
    kw, n = 32, 1 << 16
    load = np.unique(_uniform(rng, kw, 1 << 14))
    groups = [_group(rng, kw, 24, 600, 150)] + [_group(rng, kw, 24, int(rng.integers(2, 9)), 3) for _ in range(100)]
    base = _uniform(rng, kw, n - sum(g.size for g in groups))
    _run(fx, kw, 32, load, [_batch(rng, kw, base, groups, load) for _ in range(2)])


def test_dense_range_keeps_prefix_plan(fx):
    """A quarter of 2^21 ops in 2% of the key range (the top digit alone is heavy: the plan keeps
    the prefix passes and the finish), with repeated keys and groups of equal prefix inside it."""
    rng = np.random.default_rng(6)
    kw, n = 64, 1 << 21
    lo = int(0.4 * 2 ** 64)
    width = int(0.02 * 2 ** 64)
    load = np.unique(np.concatenate([_uniform(rng, kw, 1 << 15),
                                     rng.integers(lo, lo + width, 1 << 14, dtype=np.uint64)]))
    hot = rng.integers(lo, lo + width, n // 4, dtype=np.uint64)
    hot[: 3000] = hot[3000:6000] & ~np.uint64((1 << 24) - 1)        # groups sharing a 40-bit prefix
    groups = [hot, np.full(500, hot[10], dtype=np.uint64)]
    base = _uniform(rng, kw, n - sum(g.size for g in groups))
    _run(fx, kw, 32, load, [_batch(rng, kw, base, groups, load) for _ in range(2)])
