"""The device form of the batched-stream generator (workload/device.py) on CPU torch tensors: its
SplitMix64 finaliser, key universe and value hash give exactly the numpy generator's words (the
batched and served benchmarks draw their keys from it), and a short stream keeps the recipe: batch
sizes, op codes, distinct fresh inserts, range ends not below their starts."""
import numpy as np
import pytest

import workload as W
from workload import device as WD

torch = pytest.importorskip("torch")


def _u64(t):
    return t.numpy().view(np.uint64)


def test_mix64_matches_numpy():
    rng = np.random.default_rng(5)
    x = rng.integers(0, 2**63, 4096, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, 4096, dtype=np.uint64)
    x[:4] = np.array([0, 1, 2**63, 2**64 - 1], dtype=np.uint64)
    got = WD.mix64(torch.from_numpy(x.view(np.int64)))
    assert np.array_equal(_u64(got), W.mix64(x))


@pytest.mark.parametrize("seed", [4000, 4100, 5000])
def test_universe_and_values_match_numpy(seed):
    ctr = np.arange(0, 1 << 14, dtype=np.uint64)
    got = WD.universe_at64(seed, torch.from_numpy(ctr.view(np.int64)))
    exp = W.universe_at(64, seed, ctr)
    assert np.array_equal(_u64(got), exp)
    assert np.unique(exp).size == exp.size and not (exp == np.uint64(2**64 - 1)).any()
    v = WD.values_for64(got, salt=3)
    assert np.array_equal(_u64(v), W.values_for(64, exp, salt=3))


def test_short_stream_keeps_the_recipe():
    s = WD.mixed_stream_device(seed=4100, n_preload=1 << 12, n_batches=40, lo_exp=4, hi_exp=9, device="cpu")
    assert np.array_equal(_u64(s["preload_keys"]), W.universe(64, 4100, 0, 1 << 12))
    fresh = []
    for (ops, keys, aux), m in zip(s["batches"](), s["sizes"]):
        o = ops.numpy()
        assert o.size == int(m) and o.min() >= W.OP_LOOKUP and o.max() <= W.OP_DELETE
        k, a = _u64(keys), _u64(aux)
        fresh.append(k[o == W.OP_INSERT])
        r = o == W.OP_RANGE
        assert (a[r] >= k[r]).all()                      # unsigned order: hi never below lo
    fresh = np.concatenate(fresh)
    assert np.unique(fresh).size == fresh.size           # inserts take keys never drawn before
    assert not np.isin(fresh, _u64(s["preload_keys"])).any()
