"""GPU parity on the dense-range (X/Y) update rounds of Sec. 5.2.1 and the restructure accounting of
Sec. 6.6 (Tab. 2): a uniform build, insert rounds that send the fraction Y of their keys into a hot
interval covering the fraction X of the key range, delete rounds that remove them again, then a
restructure.  The layout is compared with the structural model after every round, and the number of
nodes the restructure recovers is compared exactly."""
import numpy as np
import pytest
import torch

import workload as W
from tests.gpu_util import compare_contents, compare_layout, np_of, oracle_pair, same

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fx():
    import paper_2604_16725_gb300 as fx
    fx.load()
    assert torch.cuda.is_available()
    return fx


@pytest.mark.parametrize("X,Y,kw,NS", [(0.25, 0.9, 64, 32), (0.9, 0.9, 64, 32), (0.03, 0.9, 64, 16),
                                       (0.12, 0.9, 32, 8)])
def test_xy_rounds_and_restructure_accounting(fx, X, Y, kw, NS):
    build = 1 << 14
    w = W.xy_rounds(X, Y, build, 3 * build, 8, seed=11, kw=kw)
    idx = fx.Index(key_bits=kw, node_size=NS)
    idx.bulk_load(w["build_keys"], w["build_vals"])
    mp, md = oracle_pair(kw, NS, 50, w["build_keys"], w["build_vals"])
    for k, v in w["insert"]:
        idx.insert(k, v)
        mp.update(np.full(k.size, W.OP_INSERT, np.uint8), k, v)
        md.update(np.full(k.size, W.OP_INSERT, np.uint8), k, v)
        compare_layout(idx, md)
    assert idx.stats()["live_keys"] == 4 * build
    for k in w["delete"]:
        idx.delete(k)
        mp.update(np.full(k.size, W.OP_DELETE, np.uint8), k)
        md.update(np.full(k.size, W.OP_DELETE, np.uint8), k)
        compare_layout(idx, md)
    before = idx.stats()["nodes_used"]
    assert before == md.stats()["nodes"]
    idx.restructure()
    md.restructure()
    compare_layout(idx, md)
    compare_contents(idx, mp, kw)
    after = idx.stats()["nodes_used"]
    assert after == md.stats()["nodes"]
    assert 0 < after < before
    # reads over the hot interval after the rounds: every stored key and its neighbours
    q = np.concatenate([w["build_keys"].astype(np.uint64), w["build_keys"].astype(np.uint64) + 1])
    q = q[q < (1 << kw) - 1].astype(w["build_keys"].dtype)
    sk, sv = idx.successor(q)
    e = mp.read(np.full(q.size, W.OP_SUCC, np.uint8), q)
    same(np_of(sk, kw), e["keys"], "succ.keys")
    idx.close()
