"""flix_lookup_noalloc, the lookup entry point that allocates no device memory during the call, gives
exactly the results of flix_lookup, on two calls in a row, through the C ABI, and both equal the
oracle's lookup over the loaded keys.

It serves callers that cannot allocate device memory when they query (a process whose allocator
has already reserved the device, a latency-bound path that must not block on cudaMalloc, a custom
allocator the library cannot see).  This file is collected last so that a failure here does not
hide the results of the other GPU tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import workload as W

pytestmark = pytest.mark.gpu


def _vp(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("kw,NS", [(32, 32), (64, 64)])
def test_noalloc_lookup_matches_lookup(kw, NS):
    import paper_2604_16725_gb300 as fx
    L = fx.load()
    n_load = 1 << 18
    c = W.read_scale(seed=77 + kw, kw=kw, n_load=n_load, batch=(1 << 16) + 11, n_range=0)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(c["load_keys"], c["load_vals"])
    stream = torch.cuda.current_stream()
    order = np.argsort(c["load_keys"].astype(np.uint64), kind="stable")
    sk = c["load_keys"].astype(np.uint64)[order]
    sv = c["load_vals"].astype(np.uint64)[order]
    for call, q in enumerate((c["queries"], c["queries"][::-1][:40000].copy())):
        qd = idx._dev(q)
        n = qd.numel()
        v_ref, f_ref = idx.lookup(qd)
        v = torch.full((n,), -1, dtype=idx.tdtype, device="cuda")
        f = torch.full((n,), 7, dtype=torch.uint8, device="cuda")
        code = L.flix_lookup_noalloc(idx._h, _vp(qd), n, _vp(v), _vp(f), ctypes.c_void_p(stream.cuda_stream))
        assert code == 0, L.flix_last_error(idx._h)
        torch.cuda.synchronize()
        assert torch.equal(v, v_ref), "values differ on call %d" % call
        assert torch.equal(f, f_ref), "found flags differ on call %d" % call
        ev, ef = oracle.sorted_lookup(sk, sv, q.astype(np.uint64), kw)
        got = v.cpu().numpy().view(np.uint32 if kw == 32 else np.uint64).astype(np.uint64)
        assert np.array_equal(got, ev), "values differ from the oracle on call %d" % call
        assert np.array_equal(f.cpu().numpy(), ef), "found flags differ from the oracle on call %d" % call
        assert 0.6 < f.float().mean().item() < 0.8


def test_noalloc_rejects_oversized_batch():
    import paper_2604_16725_gb300 as fx
    L = fx.load()
    idx = fx.Index(key_bits=64, node_size=64)
    idx.bulk_load(np.arange(1, 1000, dtype=np.uint64), np.arange(1, 1000, dtype=np.uint64))
    n = 1 << 20                                   # about 31 MB of scratch, more than the 16 MiB array
    q = torch.zeros(n, dtype=torch.int64, device="cuda")
    v = torch.empty(n, dtype=torch.int64, device="cuda")
    before = idx.launch_count()
    code = L.flix_lookup_noalloc(idx._h, _vp(q), n, _vp(v), None, None)
    assert code == -1
    assert b"scratch" in L.flix_last_error(idx._h)
    assert idx.launch_count() == before          # rejected before launching anything
