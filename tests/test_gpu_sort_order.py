"""The batch sort (Sec. 3.3; Tab. 1 times it) on its own, through the flix_sort_pairs test hook:
keys ascending and, for equal keys, input order (a stable sort, which the same-key fold of an update
batch relies on), compared element by element with a stable argsort of the same keys.

The cases reach every plan the sort takes: the prefix plan with the in-tile finish of short groups
(uniform keys), groups too long for it (17..4096 items: bitonic in one block; more: the chunked
radix sort of the lower digits), repeated keys (the finish must keep their input order), heavy keys
(every digit sorted), constant digits (skipped), ragged tile tails, and both key widths."""
import numpy as np
import pytest
import torch

import workload as W
from tests.gpu_util import same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


def check_sort(fx, keys, kw):
    idx = fx.Index(key_bits=kw, node_size=32)
    k, p = idx.sort_pairs(keys)
    exp = np.argsort(keys, kind="stable")
    got_p = p.cpu().numpy().view(np.uint32).astype(np.int64)
    got_k = k.cpu().numpy().view(np.uint32 if kw == 32 else np.uint64)
    same(got_p, exp, "positions (n=%d)" % keys.size)
    same(got_k, keys[exp], "keys (n=%d)" % keys.size)
    idx.close()


def rng_keys(kw, n, seed):
    r = np.random.default_rng(seed)
    hi = (1 << kw) - 1
    return r.integers(0, hi, n, dtype=np.uint64 if kw == 64 else np.uint32, endpoint=False)


@pytest.mark.parametrize("n", [1, 2, 31, 4095, 4096, 4097, 12345, 1 << 20, (1 << 22) + 77, 1 << 24])
def test_uniform_u64_prefix_plan(fx, n):
    check_sort(fx, rng_keys(64, n, n), 64)


@pytest.mark.parametrize("n", [1, 4097, 1 << 20, (1 << 22) + 5])
def test_uniform_u32(fx, n):
    check_sort(fx, rng_keys(32, n, 7 + n), 32)


def test_groups_past_the_in_tile_finish(fx):
    """2^21 keys whose top 24 bits take few values: groups of equal prefix from 2 to ~40000 items
    (one block's bitonic sort up to 4096, the chunked radix sort beyond), with repeated full keys."""
    r = np.random.default_rng(3)
    n = 1 << 21
    sizes = np.concatenate([r.integers(2, 17, 3000), r.integers(17, 4097, 300), [5000, 17000, 40000]])
    prefixes = r.choice(1 << 24, sizes.size, replace=False).astype(np.uint64)
    pre = np.repeat(prefixes, sizes)
    pre = np.concatenate([pre, r.integers(0, 1 << 24, n - pre.size).astype(np.uint64)])
    low = r.integers(0, 1 << 40, n, dtype=np.uint64)
    low[r.random(n) < 0.2] = 12345                       # many exact duplicates inside groups
    keys = (pre << np.uint64(40)) | low
    keys = keys[r.permutation(n)]
    check_sort(fx, keys, 64)


def test_heavy_repeated_keys(fx):
    """Zipf-distributed keys (the served form's hot keys): tens of thousands of copies of the hottest
    keys, whose input order the sort must keep."""
    z = W.zipf(5, 1, 1 << 21, 0.99, 1 << 20).astype(np.uint64)
    keys = W.mix64(z) >> np.uint64(1)
    check_sort(fx, keys, 64)
    check_sort(fx, (keys & np.uint64(0xFFFFFFF0)).astype(np.uint32), 32)


def test_constant_and_dense_digits(fx):
    r = np.random.default_rng(9)
    n = 1 << 20
    check_sort(fx, r.integers(0, 1 << 20, n, dtype=np.uint64), 64)                  # top 5 digits constant
    check_sort(fx, (np.uint64(0xABCD) << np.uint64(48)) | r.integers(0, 1 << 16, n, dtype=np.uint64), 64)
    check_sort(fx, np.full(n, 42, np.uint64), 64)                                    # one key repeated
    check_sort(fx, np.arange(n, 0, -1, dtype=np.uint64) * np.uint64(1 << 30), 64)    # descending, distinct


def test_passes_past_the_prefix(fx):
    """Plans with more passes than the prefix digits, which run in one cooperative launch with a grid
    barrier between passes: one extra pass (three top digits of 64 values each: not heavy, but a
    random item would share its 3-digit prefix with about 4 others, so a fourth digit is taken), and
    every digit sorted (Zipf keys make every prefix digit heavy), both with ragged last tiles."""
    r = np.random.default_rng(21)
    n = (1 << 20) + 123
    top = [r.integers(0, 64, n, dtype=np.uint64) for _ in range(3)]
    keys = (top[0] << np.uint64(56)) | (top[1] << np.uint64(48)) | (top[2] << np.uint64(40)) | \
        r.integers(0, 1 << 40, n, dtype=np.uint64)
    check_sort(fx, keys, 64)
    z = W.zipf(11, 1, (1 << 21) + 1001, 0.99, 1 << 20).astype(np.uint64)
    keys = W.mix64(z) >> np.uint64(1)
    check_sort(fx, keys, 64)
    check_sort(fx, (keys & np.uint64(0xFFFFFFF0)).astype(np.uint32), 32)
