"""The batched form's persistent kernel (flix_apply_queue): queues of small uneven mixed batches run
by one cooperative launch each, against the oracle -- every output of every batch, bit-exact, and
the bucket/node layout against the structural model after every queue; device-side admission that
rejects a batch without changing anything; and a bounded wait that gives up (a ready word that
nothing sets) and is reported as FLIX_ETIMEDOUT with the context still usable."""
import numpy as np
import pytest
import torch

import oracle
import workload as W
from tests.gpu_util import compare_layout, np_of, oracle_pair, same

pytestmark = pytest.mark.gpu


def outputs(idx, n, range_cap):
    return dict(keys_out=idx._empty(max(n, 1)), vals_out=idx._empty(max(n, 1)),
                found=idx._empty(max(n, 1), torch.uint8), range_off=idx._empty(n + 1, torch.int64),
                range_keys=idx._empty(max(range_cap, 1)), range_vals=idx._empty(max(range_cap, 1)),
                status=torch.full((4,), -1, dtype=torch.int64, device="cuda"))


def check_batch(got, e, kw, tag):
    n = e["keys"].size
    same(np_of(got["keys_out"][:n], kw), e["keys"], tag + " keys")
    same(np_of(got["vals_out"][:n], kw), e["vals"], tag + " vals")
    same(got["found"][:n].cpu().numpy(), e["found"], tag + " found")
    off = got["range_off"].cpu().numpy().view(np.uint64)
    same(off, e["range_off"], tag + " range_off")
    t = int(off[-1])
    same(np_of(got["range_keys"][:t], kw), e["range_keys"], tag + " range_keys")
    same(np_of(got["range_vals"][:t], kw), e["range_vals"], tag + " range_vals")


@pytest.mark.parametrize("kw,NS,per_queue", [(64, 8, 20), (32, 32, 7), (64, 64, 1)])
def test_queue_stream_matches_oracle(kw, NS, per_queue):
    import paper_2604_16725_gb300 as fx
    s = W.mixed_stream(seed=4500 + NS, kw=kw, n_preload=1 << 14, n_batches=60, lo_exp=0, hi_exp=11, max_len=40,
                       mix=(0.35, 0.15, 0.1, 0.25, 0.15))
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(s["preload_keys"], s["preload_vals"])
    mp, md = oracle_pair(kw, NS, 50, s["preload_keys"], s["preload_vals"])
    batches = list(s["batches"]())
    # predecessor ops too: every 9th op of each batch reads its predecessor
    for ops, _, _ in batches:
        ops[::9] = np.where(ops[::9] <= W.OP_RANGE, W.OP_PRED, ops[::9])
    for q0 in range(0, len(batches), per_queue):
        group = batches[q0:q0 + per_queue]
        qs = []
        for ops, keys, aux in group:
            b = outputs(idx, ops.size, 64 * ops.size)
            b.update(ops=idx._dev(ops, torch.uint8), keys=idx._dev(keys), aux=idx._dev(aux))
            qs.append(b)
        idx.apply_queue(qs)
        torch.cuda.synchronize()
        for i, ((ops, keys, aux), got) in enumerate(zip(group, qs)):
            e, st = mp.apply(ops, keys, aux)
            assert st == 0
            assert md.update(ops, keys, aux) == 0
            assert got["status"].tolist()[0] == 0, got["status"].tolist()
            check_batch(got, e, kw, "batch %d" % (q0 + i))
        compare_layout(idx, md)
        assert md.check() == 0
    s_ = idx.stats()
    assert s_["live_keys"] == len(mp)
    k, v = idx.export()
    ek, ev = mp.export()
    same(np_of(k, kw), ek, "final keys")
    same(np_of(v, kw), ev, "final vals")
    idx.close()


def test_queue_admission_rejects_without_changes():
    """In one queue: a batch the node pool cannot hold, one whose range pairs exceed its capacity and
    one with the reserved key are rejected on the device and change nothing; the batches around them
    are applied."""
    import paper_2604_16725_gb300 as fx
    kw, NS = 32, 4
    idx = fx.Index(key_bits=kw, node_size=NS, pool_nodes=16, grow=False)
    load = np.arange(10, 90, 10, dtype=np.uint32)
    idx.bulk_load(load, load + 1)
    mp, md = oracle_pair(kw, NS, 50, load.astype(np.uint64), (load + 1).astype(np.uint64))
    plan = [
        (np.array([W.OP_INSERT, W.OP_LOOKUP], np.uint8), np.array([15, 20], np.uint32), np.array([7, 0], np.uint32), 8, 0),
        (np.full(40, W.OP_INSERT, np.uint8), np.arange(100, 140, dtype=np.uint32), np.arange(40, dtype=np.uint32), 8, 2),
        (np.array([W.OP_RANGE, W.OP_DELETE], np.uint8), np.array([0, 30], np.uint32), np.array([80, 0], np.uint32), 2, 4),
        (np.array([W.OP_INSERT, W.OP_DELETE], np.uint8), np.array([0xFFFFFFFF, 40], np.uint32), np.array([1, 0], np.uint32), 8, 1),
        (np.array([W.OP_DELETE, W.OP_SUCC], np.uint8), np.array([50, 51], np.uint32), np.array([0, 0], np.uint32), 8, 0),
    ]
    qs = []
    for ops, keys, aux, cap, _ in plan:
        b = outputs(idx, ops.size, cap)
        b.update(ops=idx._dev(ops, torch.uint8), keys=idx._dev(keys), aux=idx._dev(aux))
        qs.append(b)
    idx.apply_queue(qs)
    torch.cuda.synchronize()
    for (ops, keys, aux, cap, flag), got in zip(plan, qs):
        assert got["status"].tolist()[0] == flag
        e = mp.read(ops, keys.astype(np.uint64), aux.astype(np.uint64))
        lookups = ops != W.OP_RANGE
        same(np_of(got["keys_out"][:ops.size], kw)[lookups], e["keys"][lookups], "reads")
        if flag == 0:
            mp.update(ops, keys.astype(np.uint64), aux.astype(np.uint64))
            md.update(ops, keys.astype(np.uint64), aux.astype(np.uint64))
    compare_layout(idx, md)
    idx.close()


def test_queue_wait_gives_up_and_reports_timeout():
    """The second batch's ready word is never set: the kernel's bounded wait gives up, the queue
    stops there (the first batch applied, the others marked not run), the next synchronising call
    returns FLIX_ETIMEDOUT, and the index and the context keep working."""
    import paper_2604_16725_gb300 as fx
    kw, NS = 64, 16
    idx = fx.Index(key_bits=kw, node_size=NS)
    load = np.arange(1, 2001, dtype=np.uint64) * np.uint64(1000)
    idx.bulk_load(load, load + np.uint64(5))
    mp, md = oracle_pair(kw, NS, 50, load, load + np.uint64(5))
    never = torch.zeros(1, dtype=torch.int32, device="cuda")
    set_ = torch.ones(1, dtype=torch.int32, device="cuda")
    qs = []
    for i in range(3):
        ops = np.full(64, W.OP_INSERT, np.uint8)
        keys = load[:64] + np.uint64(1 + i)
        b = outputs(idx, 64, 64)
        b.update(ops=idx._dev(ops, torch.uint8), keys=idx._dev(keys), aux=idx._dev(keys * np.uint64(2)),
                 ready=set_ if i != 1 else never)
        qs.append((b, ops, keys))
    idx.apply_queue([b for b, _, _ in qs], wait_us=20000)
    torch.cuda.synchronize()
    assert [b["status"].tolist()[0] for b, _, _ in qs] == [0, 8, 8]
    with pytest.raises(fx.FlixError) as ei:
        idx.stats()
    assert ei.value.code == -5
    mp.update(qs[0][1], qs[0][2], qs[0][2] * np.uint64(2))
    md.update(qs[0][1], qs[0][2], qs[0][2] * np.uint64(2))
    compare_layout(idx, md)
    # the handle and the context still work: the same queue with every word set runs through
    set_all = [dict(b, ready=set_) for b, _, _ in qs[1:]]
    idx.apply_queue(set_all)
    torch.cuda.synchronize()
    assert [b["status"].tolist()[0] for b in set_all] == [0, 0]
    for _, ops, keys in qs[1:]:
        md.update(ops, keys, keys * np.uint64(2))
    compare_layout(idx, md)
    idx.close()
