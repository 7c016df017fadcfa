"""The dense-range (X/Y) update workload of Sec. 5.2.1: properties the generator must have before any
result measured on it means what the paper's workloads mean."""
import numpy as np
import pytest

import workload as W


@pytest.mark.parametrize("kw", [32, 64])
@pytest.mark.parametrize("X,Y", [(0.9, 0.9), (0.25, 0.9), (0.03, 0.9), (0.5, 0.5)])
def test_xy_rounds_shape(kw, X, Y):
    build, inserts, rounds = 3000, 9001, 8
    w = W.xy_rounds(X, Y, build, inserts, rounds, seed=7, kw=kw)
    kmax = (1 << kw) - 1
    lo, hi = w["hot"]
    assert 0 <= lo < hi <= kmax
    assert abs((hi - lo) / kmax - X) < 1e-6                              # the hot interval spans X
    ins = [k.astype(np.uint64) for k, _ in w["insert"]]
    assert [k.size for k in ins] == [inserts // rounds] * (rounds - 1) + [inserts - (rounds - 1) * (inserts // rounds)]
    allk = np.concatenate([w["build_keys"].astype(np.uint64)] + ins)
    assert np.unique(allk).size == allk.size                             # distinct by construction
    assert allk.max() < kmax                                             # never the reserved key
    assert np.all(w["build_keys"] % 2 == 0) and all(np.all(k % 2 == 1) for k in ins)
    for k in ins:                                                        # Y of every round is hot
        assert int(((k >= lo) & (k < hi)).sum()) == int(round(Y * k.size))
    for k, d in zip(ins, w["delete"]):                                   # deletes undo the rounds
        assert np.array_equal(k, d.astype(np.uint64))
    v = np.concatenate([vv.astype(np.uint64) for _, vv in w["insert"]])
    assert v.max() < kmax


def test_xy_uniform_case_spreads_keys():
    """X = Y = 0.9 is uniform: every tenth of the key range holds about a tenth of the inserts."""
    w = W.xy_rounds(0.9, 0.9, 1000, 200000, 4, seed=3, kw=64)
    k = np.concatenate([kk for kk, _ in w["insert"]]).astype(np.float64) / 2.0 ** 64
    h, _ = np.histogram(k, bins=10, range=(0, 1))
    assert np.all(np.abs(h / k.size - 0.1) < 0.01)


def test_bijection_below_is_a_permutation():
    for size in (1, 2, 3, 1000, 4097):
        p = W.bijection_below(np.arange(size, dtype=np.uint64), size, 9)
        assert np.array_equal(np.sort(p), np.arange(size, dtype=np.uint64))


@pytest.mark.parametrize("share", [0.0, 0.3, 0.653])
def test_xy_delete_share_is_a_subset_of_the_inserts(share):
    w = W.xy_rounds(0.25, 0.9, 2000, 6001, 8, seed=5, kw=64, delete_share=share)
    ins = np.concatenate([k for k, _ in w["insert"]])
    d = np.concatenate(w["delete"])
    assert len(w["delete"]) == 8 and d.size == int(round(share * ins.size))
    assert np.unique(d).size == d.size and np.isin(d, ins).all()
    sizes = [x.size for x in w["delete"]]
    assert max(sizes) - min(sizes) <= 1


def test_tab4_implied_quantities():
    # the printed rows, read with "% recovered" = recovered / nodes before the restructure
    for row in W.TAB4:
        q = W.tab4_implied(row)
        assert abs(q["before"] - q["after"] - row[3]) < 1e-6
        assert 0.0 < q["delete_share"] < 1.0 and row[1] < q["live"] < row[2]
    # the same build at both workloads leaves about the same node count before the restructure
    b = {r[0] + str(r[1]): W.tab4_implied(r)["before"] for r in W.TAB4}
    assert abs(b["X25Y90" + str(1 << 20)] / b["X90Y90" + str(1 << 20)] - 1) < 0.01
