"""Batched form (captured CUDA graphs, device-side admission) against the oracle: every output of
every batch of an uneven mixed stream, bit-exact, across a restructure that forces re-capture."""
import numpy as np
import pytest
import torch

import oracle
import workload as W
from tests.gpu_util import np_of, same

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kw,NS", [(64, 64), (32, 16)])
def test_batched_stream_matches_oracle(kw, NS):
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.batched import BatchedRunner
    s = W.mixed_stream(seed=4100 + kw, kw=kw, n_preload=1 << 15, n_batches=40, lo_exp=2, hi_exp=12, max_len=200)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(s["preload_keys"], s["preload_vals"])
    mp = oracle.Map(kw)
    mp.bulk_load(s["preload_keys"], s["preload_vals"])
    run = BatchedRunner(idx, max_batch=1 << 12, min_log=4, range_per_op=256, free_nodes_min=1 << 14)
    for b, (ops, keys, aux) in enumerate(s["batches"]()):
        r = run.run(idx._dev(ops, torch.uint8), idx._dev(keys), idx._dev(aux))
        with torch.cuda.stream(run.stream):
            got = {k: v.clone() for k, v in r.items()}
        run.check()
        e, st = mp.apply(ops, keys, aux)
        assert st == 0
        assert int(got["status"][0]) == 0
        same(np_of(got["keys"], kw), e["keys"], "batch %d keys" % b)
        same(np_of(got["vals"], kw), e["vals"], "batch %d vals" % b)
        same(got["found"].cpu().numpy(), e["found"], "batch %d found" % b)
        off = got["range_off"].cpu().numpy().view(np.uint64)
        same(off, e["range_off"], "batch %d range_off" % b)
        t = int(off[-1])
        same(np_of(got["range_keys"][:t], kw), e["range_keys"], "batch %d range_keys" % b)
        same(np_of(got["range_vals"][:t], kw), e["range_vals"], "batch %d range_vals" % b)
        if b == 20:
            idx.restructure(stream=run.stream)
            idx.reserve(1 << 12, 1 << 14, stream=run.stream)
            run.invalidate()
    k, v = idx.export()
    ek, ev = mp.export()
    same(np_of(k, kw), ek, "final keys")
    same(np_of(v, kw), ev, "final vals")


def test_batched_stream_with_merge_and_split():
    """The merge runs inside the captured graphs after every admitted batch; the elastic split runs
    between replays (graphs re-captured).  Results and layout against the map and the model."""
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.batched import BatchedRunner
    from tests.gpu_util import compare_layout
    kw, NS = 64, 8
    s = W.mixed_stream(seed=4300, kw=kw, n_preload=1 << 13, n_batches=40, lo_exp=4, hi_exp=12, max_len=50,
                       mix=(0.3, 0.1, 0.05, 0.3, 0.25))
    idx = fx.Index(key_bits=kw, node_size=NS, merge_underfull=True)
    idx.bulk_load(s["preload_keys"], s["preload_vals"])
    mp = oracle.Map(kw)
    mp.bulk_load(s["preload_keys"], s["preload_vals"])
    md = oracle.Model(kw, NS, 50)
    md.bulk_load(s["preload_keys"], s["preload_vals"])
    md.set_policy(0, True)
    run = BatchedRunner(idx, max_batch=1 << 12, min_log=4, range_per_op=64, free_nodes_min=1 << 14)
    added = 0
    for b, (ops, keys, aux) in enumerate(s["batches"]()):
        r = run.run(idx._dev(ops, torch.uint8), idx._dev(keys), idx._dev(aux))
        with torch.cuda.stream(run.stream):
            got = {k: v.clone() for k, v in r.items()}
        run.check()
        e, st = mp.apply(ops, keys, aux)
        assert st == 0 and md.update(ops, keys, aux) == 0
        same(np_of(got["keys"], kw), e["keys"], "batch %d keys" % b)
        same(np_of(got["vals"], kw), e["vals"], "batch %d vals" % b)
        if b % 8 == 7:
            a = run.split_chains(2)
            assert a == md.split_chains(2)
            added += a
            compare_layout(idx, md)
    assert added > 0
    compare_layout(idx, md)
    k, v = idx.export()
    ek, ev = mp.export()
    same(np_of(k, kw), ek, "final keys")
    same(np_of(v, kw), ev, "final vals")


def test_async_admission_rejects_without_changes():
    """A batch the node pool cannot hold is rejected on the device and leaves the index unchanged."""
    import paper_2604_16725_gb300 as fx
    kw = 32
    idx = fx.Index(key_bits=kw, node_size=4, pool_nodes=8, grow=False)
    idx.bulk_load(np.arange(1, 9, dtype=np.uint32), np.arange(1, 9, dtype=np.uint32))
    idx.reserve(64, 0)
    before = idx.dump_layout()
    n = 40
    ops = torch.full((n,), fx.OP_INSERT, dtype=torch.uint8, device="cuda")
    keys = torch.arange(100, 100 + n, dtype=torch.int32, device="cuda")
    aux = torch.arange(n, dtype=torch.int32, device="cuda")
    out = dict(keys=torch.empty(n, dtype=torch.int32, device="cuda"), vals=torch.empty(n, dtype=torch.int32, device="cuda"),
               found=torch.empty(n, dtype=torch.uint8, device="cuda"),
               range_off=torch.empty(n + 1, dtype=torch.int64, device="cuda"),
               range_keys=torch.empty(1, dtype=torch.int32, device="cuda"),
               range_vals=torch.empty(1, dtype=torch.int32, device="cuda"),
               status=torch.zeros(4, dtype=torch.int64, device="cuda"))
    idx.apply_async(ops, keys, aux, out)
    torch.cuda.synchronize()
    st = out["status"].cpu().tolist()
    assert st[0] == 2 and st[2] > st[3]           # node pool short: need > free
    after = idx.dump_layout()
    for f in before:
        same(before[f], after[f], "unchanged " + f)
    # a reserved key in an insert is rejected the same way
    keys2 = torch.tensor([5, -1], dtype=torch.int32, device="cuda")
    ops2 = torch.full((2,), fx.OP_INSERT, dtype=torch.uint8, device="cuda")
    out2 = {k: (v[:3] if k == "range_off" else v[:2] if k in ("keys", "vals", "found") else v) for k, v in out.items()}
    idx.apply_async(ops2, keys2, aux[:2], out2)
    torch.cuda.synchronize()
    assert out2["status"].cpu().tolist()[0] == 1
    after2 = idx.dump_layout()
    for f in before:
        same(before[f], after2[f], "unchanged " + f)


@pytest.mark.parametrize("kw,NS", [(64, 16), (32, 32)])
def test_batched_persistent_queue_matches_oracle(kw, NS):
    """The runner's persistent path: batches of at most 2048 ops queue up and run by one launch of the
    persistent kernel per 8 batches; larger ones flush the queue and take the graph path.  Every
    output of every batch and the final contents against the oracle, across a restructure."""
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.batched import BatchedRunner
    depth = 8
    s = W.mixed_stream(seed=4700 + kw, kw=kw, n_preload=1 << 15, n_batches=48, lo_exp=3, hi_exp=12.5, max_len=100)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(s["preload_keys"], s["preload_vals"])
    mp = oracle.Map(kw)
    mp.bulk_load(s["preload_keys"], s["preload_vals"])
    run = BatchedRunner(idx, max_batch=1 << 13, min_log=4, range_per_op=128, free_nodes_min=1 << 15,
                        queue_depth=depth)
    batches = list(s["batches"]())
    assert any(k.size > 2048 for _, k, _ in batches) and any(k.size <= 2048 for _, k, _ in batches)
    for g0 in range(0, len(batches), depth):
        group = batches[g0:g0 + depth]
        views = []
        for ops, keys, aux in group:
            r = run.run(idx._dev(ops, torch.uint8), idx._dev(keys), idx._dev(aux))
            if keys.size > 2048:            # graph path: its views are reused by the next graph batch
                with torch.cuda.stream(run.stream):
                    r = {k: v.clone() for k, v in r.items()}
            views.append(r)
        run.check()
        for b, ((ops, keys, aux), got) in enumerate(zip(group, views)):
            e, st = mp.apply(ops, keys, aux)
            assert st == 0 and int(got["status"][0]) == 0
            tag = "batch %d" % (g0 + b)
            same(np_of(got["keys"], kw), e["keys"], tag + " keys")
            same(np_of(got["vals"], kw), e["vals"], tag + " vals")
            same(got["found"].cpu().numpy(), e["found"], tag + " found")
            off = got["range_off"].cpu().numpy().view(np.uint64)
            same(off, e["range_off"], tag + " range_off")
            t = int(off[-1])
            same(np_of(got["range_keys"][:t], kw), e["range_keys"], tag + " range_keys")
        if g0 == 24:
            run.restructure_if_needed(max_nodes_per_bucket=0.0)        # forces a restructure
    assert run.queues > 0
    k, v = idx.export()
    ek, ev = mp.export()
    same(np_of(k, kw), ek, "final keys")
    same(np_of(v, kw), ev, "final vals")
