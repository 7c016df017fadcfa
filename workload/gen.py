"""Counter-based, seeded generators for FliX workloads (numpy only).

Every random quantity is a pure function of (seed, stream, counter), so the same arrays come out on
any machine and in any process.  The primitives are:

* ``mix64`` -- the SplitMix64 output finaliser (Steele, Lea and Flood, "Fast splittable pseudorandom
  number generators", OOPSLA 2014).  It is a bijection on 64-bit words, so distinct counters give
  distinct keys, which lets key universes be drawn without de-duplication.
* ``mix32`` -- the MurmurHash3 32-bit finaliser ``fmix32`` (A. Appleby), also a bijection.
* ``zipf`` -- rejection-inversion sampling of a Zipf(s) law on {1..N} (Hoermann and Derflinger,
  "Rejection-inversion to generate variates from monotone discrete distributions", ACM TOMACS 1996).

Key width ``kw`` is 32 or 64.  The all-ones word is reserved (it is the last bucket's bound and the
"none" value), so no generated key or value ever equals it.

Operation codes match the C ABI: NOP=0, LOOKUP=1, SUCC=2, RANGE=3, INSERT=4, DELETE=5.
"""
from __future__ import annotations

import math

import numpy as np

OP_NOP, OP_LOOKUP, OP_SUCC, OP_RANGE, OP_INSERT, OP_DELETE, OP_PRED = 0, 1, 2, 3, 4, 5, 6

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)

__all__ = [
    "OP_NOP", "OP_LOOKUP", "OP_SUCC", "OP_RANGE", "OP_INSERT", "OP_DELETE", "OP_PRED",
    "key_max", "mix64", "mix32", "uniform01", "universe", "values_for", "zipf",
    "scramble30", "scramble_bits", "universe_at", "log_uniform_sizes", "permutation",
    "config1", "read_scale", "update_heavy", "mixed_stream", "serving_requests",
    "bijection_below", "xy_rounds", "TAB4", "tab4_implied",
]


def key_max(kw: int) -> int:
    return (1 << kw) - 1


def mix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser applied element-wise (a bijection on uint64)."""
    z = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def mix32(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 fmix32 applied element-wise (a bijection on uint32)."""
    h = np.asarray(x, dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        h ^= h >> np.uint32(16)
        h *= np.uint32(0x85EBCA6B)
        h ^= h >> np.uint32(13)
        h *= np.uint32(0xC2B2AE35)
        h ^= h >> np.uint32(16)
    return h


def _stream_words(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n pseudo-random 64-bit words for (seed, stream), counter-based SplitMix64."""
    base = mix64(np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1) & 0xFFFFFFFFFFFFFFFF],
                          dtype=np.uint64))[0]
    ctr = np.arange(start + 1, start + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(base + ctr * _GOLDEN)


def uniform01(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n doubles uniform in [0, 1) with 53 random bits each."""
    w = _stream_words(seed, stream, n, start)
    return (w >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def universe(kw: int, seed: int, lo: int, hi: int) -> np.ndarray:
    """Keys number lo..hi-1 of the seeded key universe: distinct across all counters, never KEY_MAX.

    The universe is the bijection mix(counter ^ s) with a seed-dependent mask s, so keys drawn from
    disjoint counter ranges are disjoint sets.  The single counter whose image is the reserved
    all-ones word is redirected to the spare counter 2^kw - 1, which no caller uses.
    """
    assert 0 <= lo <= hi
    assert kw == 64 or hi <= (1 << 32) - 1
    return universe_at(kw, seed, np.arange(lo, hi, dtype=np.uint64))


def universe_at(kw: int, seed: int, ctr: np.ndarray) -> np.ndarray:
    """Keys of the seeded universe at the given counters (see `universe`)."""
    ctr = np.asarray(ctr, dtype=np.uint64)
    if kw == 64:
        s = _stream_words(seed, 0xC0FFEE, 1)[0]
        k = mix64(ctr ^ s)
        bad = k == _M64
        if bad.any():
            k[bad] = mix64(np.array([_M64 ^ s], dtype=np.uint64))[0]
        return k
    assert kw == 32
    s = np.uint32(int(_stream_words(seed, 0xC0FFEE, 1)[0]) & 0xFFFFFFFF)
    k = mix32(ctr.astype(np.uint32) ^ s)
    bad = k == np.uint32(0xFFFFFFFF)
    if bad.any():
        k[bad] = mix32(np.array([0xFFFFFFFF], dtype=np.uint32) ^ s)[0]
    return k


def values_for(kw: int, keys: np.ndarray, salt: int = 0) -> np.ndarray:
    """A value per key (a hash of the key), never the all-ones 'none' value."""
    if kw == 64:
        v = mix64(np.asarray(keys, dtype=np.uint64) ^ np.uint64(0x5DEECE66D + salt))
        return v & np.uint64(0xFFFFFFFFFFFFFFFE)
    v = mix32(np.asarray(keys, dtype=np.uint32) ^ np.uint32((0x2545F491 + salt) & 0xFFFFFFFF))
    return v & np.uint32(0xFFFFFFFE)


def permutation(seed: int, stream: int, n: int) -> np.ndarray:
    """A seeded uniform permutation of range(n) (argsort of random words)."""
    return np.argsort(_stream_words(seed, stream, n), kind="stable")


def scramble30(r: np.ndarray) -> np.ndarray:
    """A fixed bijection of [0, 2^30): odd multiply mod 2^30 and xorshift, twice."""
    m = np.uint64((1 << 30) - 1)
    x = np.asarray(r, dtype=np.uint64) & m
    with np.errstate(over="ignore"):
        x = (x * np.uint64(0x2F0F3A75)) & m
        x ^= x >> np.uint64(15)
        x = (x * np.uint64(0x1B873593)) & m
        x ^= x >> np.uint64(13)
    return x


def zipf(seed: int, stream: int, n: int, s: float, N: int) -> np.ndarray:
    """n ranks in [1, N] drawn from Zipf(s) by rejection-inversion (Hoermann & Derflinger 1996).

    Density h(x) = x^-s on [1, N]; H is its antiderivative, written in the numerically stable
    helper form so that s close to 1 is exact enough.  Accept k = round(x) when k - x <= c
    (the squeeze) or when u >= H(k + 1/2) - h(k).  The two helper functions with their series
    fallbacks and the squeeze constant c follow the form of this method in Apache Commons Math's
    RejectionInversionZipfSampler.
    """
    assert s > 0 and N >= 1
    one_m_s = 1.0 - s

    def helper1(t):  # log1p(t) / t
        t = np.asarray(t, dtype=np.float64)
        out = np.ones_like(t)
        big = np.abs(t) > 1e-8
        out[big] = np.log1p(t[big]) / t[big]
        small = ~big
        out[small] = 1.0 - t[small] * (0.5 - t[small] / 3.0)
        return out

    def helper2(t):  # expm1(t) / t
        t = np.asarray(t, dtype=np.float64)
        out = np.ones_like(t)
        big = np.abs(t) > 1e-8
        out[big] = np.expm1(t[big]) / t[big]
        small = ~big
        out[small] = 1.0 + t[small] * 0.5 * (1.0 + t[small] / 3.0)
        return out

    def H(x):
        lx = np.log(x)
        return helper2(one_m_s * lx) * lx

    def Hinv(y):
        t = np.maximum(y * one_m_s, -1.0)
        return np.exp(helper1(t) * y)

    def h(x):
        return np.exp(-s * np.log(x))

    hx1 = float(H(np.array([1.5]))[0]) - 1.0
    hN = float(H(np.array([N + 0.5]))[0])
    c = 2.0 - float(Hinv(H(np.array([2.5])) - h(np.array([2.0])))[0])

    out = np.empty(n, dtype=np.int64)
    todo = np.arange(n)
    ctr = 0
    while todo.size:
        u01 = uniform01(seed, stream, todo.size, start=ctr)
        ctr += todo.size
        u = hN + u01 * (hx1 - hN)
        x = Hinv(u)
        k = np.clip(np.floor(x + 0.5), 1, N)
        ok = (k - x <= c) | (u >= H(k + 0.5) - h(k))
        out[todo[ok]] = k[ok].astype(np.int64)
        todo = todo[~ok]
    return out


def log_uniform_sizes(seed: int, stream: int, n: int, lo_exp: float, hi_exp: float) -> np.ndarray:
    """n sizes floor(2^U(lo_exp, hi_exp))."""
    u = uniform01(seed, stream, n)
    return np.floor(np.exp2(lo_exp + u * (hi_exp - lo_exp))).astype(np.int64)


def _kdt(kw):
    return np.uint64 if kw == 64 else np.uint32


# ----------------------------------------------------------------------------------------------
# Configurations.  Sizes are parameters so the same recipe runs scaled down in the tests.
# ----------------------------------------------------------------------------------------------

def config1(seed: int = 0, kw: int = 32, n_load: int = 1 << 16, n_ops: int = 1 << 14):
    """Tiny plain case: load n_load distinct uniform keys, then one mixed batch of n_ops.

    Mix: 50% lookups (half hits from the loaded keys, half misses), 25% inserts of fresh keys,
    25% deletes of loaded keys, shuffled by the seed.
    """
    dt = _kdt(kw)
    load = universe(kw, seed, 0, n_load)
    load_v = values_for(kw, load)
    nl = n_ops // 2
    nh = nl // 2
    nm = nl - nh
    ni = n_ops // 4
    nd = n_ops - nl - ni
    w = _stream_words(seed, 11, 4 * n_ops)
    hits = load[(w[:nh] % np.uint64(n_load)).astype(np.int64)]
    misses = universe(kw, seed, n_load, n_load + nm)
    fresh = universe(kw, seed, n_load + nm, n_load + nm + ni)
    dels = load[(w[nh:nh + nd] % np.uint64(n_load)).astype(np.int64)]
    keys = np.concatenate([hits, misses, fresh, dels]).astype(dt)
    ops = np.concatenate([np.full(nl, OP_LOOKUP), np.full(ni, OP_INSERT),
                          np.full(nd, OP_DELETE)]).astype(np.uint8)
    aux = np.zeros(n_ops, dtype=dt)
    aux[nl:nl + ni] = values_for(kw, fresh, salt=1)
    perm = permutation(seed, 12, n_ops)
    return dict(kw=kw, load_keys=load, load_vals=load_v,
                ops=ops[perm], keys=keys[perm], aux=aux[perm])


def read_scale(seed: int = 2000, kw: int = 64, n_load: int = 1 << 26, batch: int = 1 << 24,
               miss_rate: float = 0.3, n_range: int = 1 << 18, max_len: int = 1000):
    """Read-scale case: n_load distinct uniform keys; point/successor batch with a miss rate;
    range batch whose queries span U[1, max_len] consecutive stored keys.

    Range bounds need the sorted stored keys, which the generator computes with numpy's sort (a
    library primitive, not the method).
    """
    dt = _kdt(kw)
    load = universe(kw, seed, 0, n_load)
    load_v = values_for(kw, load)
    nmiss = int(round(batch * miss_rate))
    nhit = batch - nmiss
    w = _stream_words(seed, 21, nhit)
    hits = load[(w % np.uint64(n_load)).astype(np.int64)]
    misses = universe(kw, seed, n_load, n_load + nmiss)
    q = np.concatenate([hits, misses]).astype(dt)
    q = q[permutation(seed, 22, batch)]
    out = dict(kw=kw, load_keys=load, load_vals=load_v, queries=q)
    if n_range:
        sk = np.sort(load)
        wi = _stream_words(seed, 23, n_range)
        wl = _stream_words(seed, 24, n_range)
        i = (wi % np.uint64(n_load)).astype(np.int64)
        ln = (wl % np.uint64(max_len)).astype(np.int64) + 1
        j = np.minimum(i + ln - 1, n_load - 1)
        out["range_lo"] = sk[i].astype(dt)
        out["range_hi"] = sk[j].astype(dt)
    return out


def update_heavy(dist: str, seed: int = 3000, kw: int = 32, n_batches: int = 64,
                 batch: int = 1 << 20, zipf_s: float = 0.99, domain_bits: int = 30,
                 n_del_batches: int = 32):
    """Update-heavy case: insert batches drawn uniform / Zipf / sorted-sequential, then delete
    batches that remove a seeded random 50% of the keys stored after the insert phase.

    Returns the insert batches (keys, values) and a function that, given the stored key set after
    the insert phase (from the oracle), returns the delete batches.
    """
    dt = _kdt(kw)
    ins = []
    for b in range(n_batches):
        if dist == "uniform":
            k = universe(kw, seed + 17 * b, 0, batch)
        elif dist in ("zipf", "zipf_dense"):
            r = zipf(seed, 100 + b, batch, zipf_s, 1 << domain_bits) - 1
            k = (scramble30(r) if dist == "zipf" else r.astype(np.uint64)).astype(dt)
        elif dist == "sequential":
            k = np.arange(b * batch, (b + 1) * batch, dtype=np.uint64).astype(dt)
        else:
            raise ValueError(dist)
        ins.append((k.astype(dt), values_for(kw, k, salt=b + 1)))

    def deletes(stored_keys: np.ndarray):
        n = stored_keys.size
        pick = permutation(seed, 999, n)[: n // 2]
        chosen = stored_keys[pick]
        return [c.astype(dt) for c in np.array_split(chosen, n_del_batches)]

    return ins, deletes


def mixed_stream(seed: int = 4000, kw: int = 64, n_preload: int = 1 << 27, n_batches: int = 10000,
                 lo_exp: float = 8, hi_exp: float = 22, hit_rate: float = 0.7, max_len: int = 1000,
                 mix=(0.60, 0.15, 0.05, 0.10, 0.10)):
    """Batched-form stream: preload, then uneven mixed batches (lookup/succ/range/insert/delete).

    Hits and deletes draw from the preload plus inserts generated earlier in the stream (stale keys
    are allowed: deleting an absent key is a no-op).  Range queries take lo from the universe and
    hi = lo + span where span is 1..max_len times the mean gap between the keys generated so far
    (preload and earlier inserts), so they cover at most about max_len stored keys however far the
    stream has grown the index.
    Yields (ops, keys, aux) per batch; preload arrays come first via the 'preload' entry.
    """
    dt = _kdt(kw)
    pre = universe(kw, seed, 0, n_preload)
    sizes = log_uniform_sizes(seed, 1, n_batches, lo_exp, hi_exp)
    cum = np.cumsum(np.array(mix) / np.sum(mix))

    def batches():
        # the keys inserted so far are universe counters [n_preload, n_preload + n_ins): sampling
        # "preload or earlier insert" is sampling a counter below n_preload + n_ins
        n_ins = 0
        miss_ctr = 0
        for b, m in enumerate(sizes):
            m = int(m)
            u = uniform01(seed, 10 + 3 * b, m)
            ops = np.searchsorted(cum, u, side="right").astype(np.uint8) + 1
            ops = np.minimum(ops, OP_DELETE).astype(np.uint8)
            aux = np.zeros(m, dtype=dt)
            w = _stream_words(seed, 11 + 3 * b, 3 * m)
            src = w[:m] % np.uint64(n_preload + n_ins)
            kk = universe_at(kw, seed, src).astype(np.uint64)
            hit = (w[m:2 * m] >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53)) < hit_rate
            miss_keys = universe(kw, seed ^ 0x5A5A, miss_ctr, miss_ctr + m)
            miss_ctr += m
            kk = np.where(hit, kk, miss_keys.astype(np.uint64))
            is_ins = ops == OP_INSERT
            k_ins = int(is_ins.sum())
            fresh = universe(kw, seed, n_preload + n_ins, n_preload + n_ins + k_ins)
            n_ins += k_ins
            kk[is_ins] = fresh.astype(np.uint64)
            keys = kk.astype(dt)
            aux[is_ins] = values_for(kw, fresh, salt=b + 7)
            is_rng = ops == OP_RANGE
            gap = (1 << kw) // max(n_preload + n_ins, 1)
            span = ((w[2 * m:] % np.uint64(max_len)).astype(np.uint64) + np.uint64(1)) * np.uint64(gap)
            with np.errstate(over="ignore"):
                hi = kk + span
            hi = np.where(hi < kk, np.uint64(key_max(kw) - 1), hi)          # 64-bit wrap
            hi = np.minimum(hi, np.uint64(key_max(kw) - 1))
            aux[is_rng] = hi[is_rng].astype(dt)
            yield ops, keys, aux

    return dict(kw=kw, preload_keys=pre, preload_vals=values_for(kw, pre), sizes=sizes,
                batches=batches)


def scramble_bits(r: np.ndarray, bits: int, seed: int) -> np.ndarray:
    """A seeded bijection of [0, 2^bits): four rounds of odd multiply and xorshift mod 2^bits."""
    m = np.uint64((1 << bits) - 1)
    x = np.asarray(r, dtype=np.uint64) & m
    keys = _stream_words(seed, 77, 4) | np.uint64(1)
    with np.errstate(over="ignore"):
        for k in keys:
            x = (x * k) & m
            x ^= x >> np.uint64(max(bits // 2, 1))
    return x


def serving_requests(seed: int = 5000, kw: int = 64, universe_bits: int = 29, preload_bits: int = 28,
                     offered_ops_per_s: float = 1e8, n_requests: int = 100000, zipf_s: float = 0.9,
                     mix=(0.80, 0.10, 0.10)):
    """Serving-form request schedule: Poisson arrivals of requests of floor(2^U(0,12)) ops,
    80/10/10 lookup/insert/delete over Zipf(0.9) ranks mapped through a seeded bijection of the
    universe's indices (so popular keys are spread over the key space).

    The universe is mix(counter) for counters [0, 2^universe_bits); the first 2^preload_bits of it
    are the preload (`universe(kw, seed, 0, 1 << preload_bits)`).  Returns the preload count and
    per-request (arrival_s, ops, keys, aux) arrays in CSR form (req_off[n_requests + 1]).
    """
    dt = _kdt(kw)
    U = 1 << universe_bits
    sizes = log_uniform_sizes(seed, 1, n_requests, 0, 12)
    total = int(sizes.sum())
    mean_ops = total / n_requests
    rate = offered_ops_per_s / mean_ops
    gaps = -np.log1p(-uniform01(seed, 2, n_requests)) / rate
    arrival = np.cumsum(gaps)
    r = zipf(seed, 3, total, zipf_s, U) - 1
    ctr = scramble_bits(r, universe_bits, seed)
    keys = universe_at(kw, seed, ctr).astype(dt)
    cum = np.cumsum(np.array(mix) / np.sum(mix))
    sel = np.searchsorted(cum, uniform01(seed, 5, total), side="right")
    ops = np.array([OP_LOOKUP, OP_INSERT, OP_DELETE], dtype=np.uint8)[np.minimum(sel, 2)]
    aux = np.where(ops == OP_INSERT, values_for(kw, keys, salt=3), 0).astype(dt)
    off = np.zeros(n_requests + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    return dict(kw=kw, universe_bits=universe_bits, n_preload=1 << preload_bits, arrival_s=arrival,
                req_off=off, ops=ops, keys=keys, aux=aux, mean_ops=mean_ops)


def bijection_below(c: np.ndarray, size: int, seed: int) -> np.ndarray:
    """A seeded bijection of [0, size) applied to counters c < size: `scramble_bits` over the
    smallest power of two >= size, re-applied to any image >= size until it falls below size
    (cycle walking; it terminates because the scramble is a permutation of the power-of-two range)."""
    c = np.asarray(c, dtype=np.uint64)
    if size <= 1:
        return np.zeros(c.shape, dtype=np.uint64)
    bits = max(int(size - 1).bit_length(), 1)
    x = scramble_bits(c, bits, seed)
    out = np.ascontiguousarray(x)
    bad = np.nonzero(out >= np.uint64(size))[0]
    while bad.size:
        out[bad] = scramble_bits(out[bad], bits, seed)
        bad = bad[out[bad] >= np.uint64(size)]
    return out


def xy_rounds(X: float, Y: float, build: int, inserts: int, rounds: int, seed: int = 6000,
              kw: int = 64, delete_share: float = 1.0):
    """Dense-range (X/Y) update workload: a hot interval covering the fraction X of the key range
    receives the fraction Y of every insert round; the rest of the round is spread uniformly over
    the remaining key range.  X = Y = 0.9 is the uniform case.

    Keys are distinct by construction: with V = 2^(kw-1) - 1 values v, build keys are 2v and
    inserted keys 2v + 1 (never KEY_MAX).  Build values v are `bijection_below` of the counters
    0..build-1 over [0, V).  The hot interval is [h0, h0 + H) in v, H = floor(X V), h0 seeded;
    hot inserts take counters 0, 1, ... of a bijection of [0, H) shifted by h0, cold inserts counters
    of a bijection of [0, V - H) with the hot interval skipped.  Each round holds
    round(Y m) hot and m - round(Y m) cold keys (m = inserts / rounds, the last round takes the
    remainder), hot ones first: the keys are distinct and every batch is sorted, so their order
    changes no result.  With delete_share = 1 the delete rounds remove the keys of the insert
    rounds, round by round (the structure returns to its build keys); with delete_share < 1 they
    remove round(delete_share * inserts) of the inserted keys, a seeded choice in seeded order, in
    `rounds` batches of (nearly) equal size.

    Returns dict(build_keys, build_vals, insert=[(keys, vals)], delete=[keys], hot=(lo_key, hi_key)).
    """
    assert 0.0 < X <= 1.0 and 0.0 <= Y <= 1.0 and kw in (32, 64) and 0.0 <= delete_share <= 1.0
    dt = _kdt(kw)
    V = (1 << (kw - 1)) - 1
    H = max(1, min(V - 1, int(X * V)))
    h0 = int(_stream_words(seed, 1, 1)[0] % np.uint64(V - H + 1))
    bk = (bijection_below(np.arange(build, dtype=np.uint64), V, seed ^ 0x11) << np.uint64(1)).astype(dt)
    per = [inserts // rounds] * rounds
    per[-1] += inserts - sum(per)
    n_hot = [int(round(Y * m)) for m in per]
    assert sum(n_hot) <= H and sum(per) - sum(n_hot) <= V - H, "more keys than the interval holds"
    ins, dels = [], []
    ch = cc = 0
    for r, m in enumerate(per):
        kh, kc = n_hot[r], m - n_hot[r]
        vh = bijection_below(np.arange(ch, ch + kh, dtype=np.uint64), H, seed ^ 0x22) + np.uint64(h0)
        ic = bijection_below(np.arange(cc, cc + kc, dtype=np.uint64), V - H, seed ^ 0x33)
        vc = np.where(ic < np.uint64(h0), ic, ic + np.uint64(H))
        ch += kh
        cc += kc
        v = np.concatenate([vh, vc])
        k = ((v << np.uint64(1)) | np.uint64(1)).astype(dt)
        ins.append((k, values_for(kw, k, salt=r + 1)))
        dels.append(k.copy())
    if delete_share < 1.0:
        allk = np.concatenate(dels) if dels else np.zeros(0, dt)
        take = permutation(seed ^ 0x44, 5, allk.size)[:int(round(delete_share * allk.size))]
        dels = [np.ascontiguousarray(d) for d in np.array_split(allk[take], rounds)]
    return dict(kw=kw, build_keys=bk, build_vals=values_for(kw, bk), insert=ins, delete=dels,
                hot=(2 * h0, 2 * (h0 + H)))


# Tab. 4 (Sec. 6.6): nodes recovered by one restructure after 8 insert rounds and 8 delete rounds,
# node size 32.  (workload, build keys, final keys, nodes recovered, % recovered) as printed; "1M"
# and "33M" are read as 2^20 and 2^25 (their final sizes, 4M and 134M, are 4x those), "100M" as
# 10^8 with the printed final size 300M.
TAB4 = (("X25Y90", 1 << 20, 4 << 20, 54623, 29), ("X25Y90", 1 << 25, 4 << 25, 1745428, 29),
        ("X25Y90", 100_000_000, 300_000_000, 3928746, 28), ("X90Y90", 1 << 20, 4 << 20, 81307, 43),
        ("X90Y90", 1 << 25, 4 << 25, 2603137, 43), ("X90Y90", 100_000_000, 300_000_000, 6130104, 46))


def tab4_implied(row, half: int = 16):
    """What one Tab. 4 row implies when "% recovered" is the share of the nodes before the
    restructure: nodes before = recovered / share, nodes after = before - recovered, live keys at
    the restructure = after * half (the restructure cuts half-full nodes), and the share of the
    inserted keys the delete rounds removed = (final - live) / (final - build)."""
    _, build, final, rec, pct = row
    before = rec / (pct / 100.0)
    after = before - rec
    live = after * half
    return dict(before=before, after=after, live=live, delete_share=(final - live) / (final - build))

