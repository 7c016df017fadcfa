// Initial build (Sec. 3.2), restructuring (Sec. 3.5) and the live-pair gather they and the export
// share.
//
// Build: the sorted, de-duplicated pairs are cut into groups of p = fill * NS keys; group i becomes
// node i and bucket i, whose maxBucket is the group's largest key (the last bucket's is KEY_MAX).
// Node ids follow bucket order, and the free stack holds the remaining ids with the smallest on
// top, so nodes allocated later stay near their buckets.
//
// Restructure: every bucket's live count (a walk of its chain), a scan, a gather of the live pairs
// in bucket and chain order (globally sorted), then the same cut.  Chains are walked node by node
// only up to SHORT_CHAIN nodes; when a longer chain exists, the nodes in use (the ids not on the
// free stack) are put in chain order by sorting them by maxKey instead (maxKeys increase strictly
// along a chain and from bucket to bucket), and a scan of their sizes gives each node's first rank.
#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr int BT = 256;

constexpr uint32_t SHORT_CHAIN = 64;

// Live pairs per bucket; a chain longer than SHORT_CHAIN nodes sets *long_flag instead.
template <class K>
__global__ void k_live_count(DevIdx<K> ix, uint64_t* __restrict__ cnt, uint32_t* __restrict__ long_flag)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ix.nb) return;
    uint64_t c = 0;
    uint32_t steps = 0;
    for (uint32_t x = ix.head[b]; x != NIL; x = ix.next[x]) {
        if (++steps > SHORT_CHAIN) { atomicOr(long_flag, 1u); break; }
        c += ix.size[x];
    }
    cnt[b] = c;
}

// ---- nodes in chain order without walking chains ----------------------------------------------

__global__ void k_unmark_free(const uint32_t* __restrict__ free_ids, const DevState* __restrict__ ds,
                              uint8_t* __restrict__ mark)
{
    grid_dep_enter();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ds->free_top) mark[free_ids[i]] = 0;
}

template <class K>
__global__ void k_used_compact(DevIdx<K> ix, const uint8_t* __restrict__ mark, const uint32_t* __restrict__ pos,
                               uint64_t cap, K* __restrict__ ubound, uint32_t* __restrict__ uid)
{
    grid_dep_enter();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= cap || !mark[i]) return;
    ubound[pos[i]] = ix.bound[i];
    uid[pos[i]] = (uint32_t)i;
}

template <class K>
__global__ void k_node_sizes(DevIdx<K> ix, const uint32_t* __restrict__ uid, const uint32_t* __restrict__ perm,
                             uint64_t m, uint32_t* __restrict__ order, uint32_t* __restrict__ osz)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    const uint32_t nd = uid[perm[j]];
    order[j] = nd;
    osz[j] = ix.size[nd];
}

// one warp per node in chain order: its pairs to ranks noff[j] ... (flat, or straight into the
// second node arrays with CUT)
template <class K, bool CUT>
__global__ void k_gather_nodes(DevIdx<K> ix, const uint32_t* __restrict__ order, const uint64_t* __restrict__ noff,
                               uint64_t m, uint32_t p, uint64_t nb_new, K* __restrict__ ok, K* __restrict__ ov);

// chain[b] += 1 for every node of bucket b (bk: bucket of every node in chain order)
__global__ void k_chain_count(const uint32_t* __restrict__ bk, uint64_t m, uint32_t* __restrict__ chain)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j < m) atomicAdd(&chain[bk[j]], 1u);
}

__global__ void k_chain_max(const uint32_t* __restrict__ chain, uint64_t nb, unsigned long long* __restrict__ out)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b < nb) atomicMax(out, (unsigned long long)chain[b]);
}

constexpr uint32_t FULL = 0xFFFFFFFFu;

// One warp per 32 consecutive buckets copies their chains' pairs to out[goff[b] ...].  Lane l
// loads bucket b0 + l's first node and its size and link in parallel; the first nodes of buckets
// whose chains end there are copied together with one independent load per pair (each lane finds
// its pair's bucket by a shuffle search over the prefix of their sizes); the other chains are then
// walked node by node by the whole warp.
template <class K>
__global__ void k_gather(DevIdx<K> ix, const uint64_t* __restrict__ goff, K* __restrict__ ok, K* __restrict__ ov)
{
    grid_dep_enter();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t b0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    if (b0 >= ix.nb) return;
    const uint32_t NS = ix.NS;
    const uint64_t b = b0 + lane;
    uint32_t n_l = NIL, sz_l = 0, nx_l = NIL;
    uint64_t o_l = 0;
    if (b < ix.nb) {
        n_l = ix.head[b];
        o_l = goff[b];
        sz_l = ix.size[n_l];
        nx_l = ix.next[n_l];
    }
    // single-node chains: one flat copy
    const uint32_t cnt = nx_l == NIL ? sz_l : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        uint32_t src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t probe = src + step - 1;
            if (__shfl_sync(FULL, incl, probe) <= t) src += step;
        }
        const uint32_t base = __shfl_sync(FULL, incl - cnt, src);
        const uint32_t sn = __shfl_sync(FULL, n_l, src);
        const uint64_t so = __shfl_sync(FULL, o_l, src);
        if (t < total) {
            const uint32_t k = t - base;
            ok[so + k] = ix.keys[(uint64_t)sn * NS + k];
            ov[so + k] = ix.vals[(uint64_t)sn * NS + k];
        }
    }
    // longer chains, one bucket at a time
    uint32_t rest = __ballot_sync(FULL, nx_l != NIL);
    while (rest) {
        const uint32_t i = __ffs(rest) - 1;
        rest &= rest - 1;
        uint64_t o = __shfl_sync(FULL, o_l, i);
        uint32_t x = __shfl_sync(FULL, n_l, i);
        uint32_t steps = 0;
        while (x != NIL) {
            if (++steps > ix.cap) break;
            const uint32_t sz = ix.size[x];
            for (uint32_t s2 = lane; s2 < sz; s2 += 32) {
                ok[o + s2] = ix.keys[(uint64_t)x * NS + s2];
                ov[o + s2] = ix.vals[(uint64_t)x * NS + s2];
            }
            o += sz;
            x = ix.next[x];
        }
    }
}

// One-pass restructure: like k_gather, but the pair of global rank e goes straight to slot e % p
// of node e / p of the second node arrays (k2, v2); the last pair of every group but the last
// also sets its node's maxKey and its bucket's maxBucket.
template <class K>
__device__ __forceinline__ void put_ranked(DevIdx<K>& ix, K* __restrict__ k2, K* __restrict__ v2, uint64_t e,
                                           uint32_t p, uint64_t nb_new, K key, K val)
{
    const uint64_t node = e < (1ull << 32) ? (uint64_t)((uint32_t)e / p) : e / p;
    const uint32_t slot = (uint32_t)(e - node * p);
    k2[node * ix.NS + slot] = key;
    v2[node * ix.NS + slot] = val;
    if (slot == p - 1 && node + 1 < nb_new) {
        ix.bound[node] = key;
        ix.mkba[node] = key;
    }
}

template <class K>
__global__ void k_gather_cut(DevIdx<K> ix, const uint64_t* __restrict__ goff, uint32_t p, uint64_t nb_new,
                             K* __restrict__ k2, K* __restrict__ v2)
{
    grid_dep_enter();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t b0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 32;
    if (b0 >= ix.nb) return;
    const uint32_t NS = ix.NS;
    const uint64_t b = b0 + lane;
    uint32_t n_l = NIL, sz_l = 0, nx_l = NIL;
    uint64_t o_l = 0;
    if (b < ix.nb) {
        n_l = ix.head[b];
        o_l = goff[b];
        sz_l = ix.size[n_l];
        nx_l = ix.next[n_l];
    }
    const uint32_t cnt = nx_l == NIL ? sz_l : 0u;
    uint32_t incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(FULL, incl, d);
        if (lane >= (uint32_t)d) incl += y;
    }
    const uint32_t total = __shfl_sync(FULL, incl, 31);
    for (uint32_t t0 = 0; t0 < total; t0 += 32) {
        const uint32_t t = t0 + lane;
        uint32_t src = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const uint32_t probe = src + step - 1;
            if (__shfl_sync(FULL, incl, probe) <= t) src += step;
        }
        const uint32_t base = __shfl_sync(FULL, incl - cnt, src);
        const uint32_t sn = __shfl_sync(FULL, n_l, src);
        const uint64_t so = __shfl_sync(FULL, o_l, src);
        if (t < total) {
            const uint32_t k = t - base;
            put_ranked(ix, k2, v2, so + k, p, nb_new, ix.keys[(uint64_t)sn * NS + k], ix.vals[(uint64_t)sn * NS + k]);
        }
    }
    uint32_t rest = __ballot_sync(FULL, nx_l != NIL);
    while (rest) {
        const uint32_t i = __ffs(rest) - 1;
        rest &= rest - 1;
        uint64_t o = __shfl_sync(FULL, o_l, i);
        uint32_t x = __shfl_sync(FULL, n_l, i);
        uint32_t steps = 0;
        while (x != NIL) {
            if (++steps > ix.cap) break;
            const uint32_t sz = ix.size[x];
            for (uint32_t s2 = lane; s2 < sz; s2 += 32)
                put_ranked(ix, k2, v2, o + s2, p, nb_new, ix.keys[(uint64_t)x * NS + s2], ix.vals[(uint64_t)x * NS + s2]);
            o += sz;
            x = ix.next[x];
        }
    }
}

template <class K, bool CUT>
__global__ void k_gather_nodes(DevIdx<K> ix, const uint32_t* __restrict__ order, const uint64_t* __restrict__ noff,
                               uint64_t m, uint32_t p, uint64_t nb_new, K* __restrict__ ok, K* __restrict__ ov)
{
    grid_dep_enter();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t j = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (j >= m) return;
    const uint32_t nd = order[j];
    const uint64_t o = noff[j];
    const uint32_t sz = ix.size[nd];
    for (uint32_t s2 = lane; s2 < sz; s2 += 32) {
        const K key = ix.keys[(uint64_t)nd * ix.NS + s2];
        const K val = ix.vals[(uint64_t)nd * ix.NS + s2];
        if (CUT) {
            put_ranked(ix, ok, ov, o + s2, p, nb_new, key, val);
        } else {
            ok[o + s2] = key;
            ov[o + s2] = val;
        }
    }
}

// one warp per new node: node i takes pairs [i * p, min((i + 1) * p, n))
template <class K>
__global__ void k_cut_keys(DevIdx<K> ix, const K* __restrict__ sk, const K* __restrict__ sv, uint64_t n, uint32_t p)
{
    grid_dep_enter();
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t node = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t lo = node * p;
    if (lo >= n) return;
    const uint32_t cnt = (uint32_t)(n - lo < p ? n - lo : p);
    for (uint32_t s2 = lane; s2 < cnt; s2 += 32) {
        ix.keys[node * ix.NS + s2] = sk[lo + s2];
        ix.vals[node * ix.NS + s2] = sv[lo + s2];
    }
}

template <class K>
__global__ void k_cut_meta(DevIdx<K> ix, const K* __restrict__ sk, uint64_t n, uint32_t p, uint64_t nb_new,
                           uint64_t cap, uint32_t* __restrict__ free_ids)
{
    grid_dep_enter();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nb_new) {
        const uint64_t lo = i * p;
        const uint64_t hi = lo + p < n ? lo + p : n;
        ix.size[i] = (uint32_t)(hi > lo ? hi - lo : 0);
        ix.next[i] = NIL;
        ix.head[i] = (uint32_t)i;
        // sk == nullptr: the one-pass restructure already set every maxKey but the last
        if (sk || i + 1 == nb_new) {
            const K mb = (i + 1 == nb_new) ? key_max<K>() : sk[hi - 1];
            ix.bound[i] = mb;
            ix.mkba[i] = mb;
        }
    }
    // free stack: ids nb_new .. cap-1, smallest id on top
    if (i < cap - nb_new) free_ids[i] = (uint32_t)(cap - 1 - i);
}

// keep the first pair of each run of equal keys: flags, then compaction by a scan
template <class K>
__global__ void k_dedupe_flags(const K* __restrict__ skeys, uint64_t n, uint32_t* __restrict__ head)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    head[j] = (j == 0 || skeys[j] != skeys[j - 1]) ? 1u : 0u;
}

template <class K>
__global__ void k_dedupe_write(const K* __restrict__ skeys, const uint32_t* __restrict__ sidx,
                               const K* __restrict__ vals, uint64_t n, const uint32_t* __restrict__ head,
                               const uint32_t* __restrict__ pos, K* __restrict__ ok, K* __restrict__ ov)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n || !head[j]) return;
    ok[pos[j]] = skeys[j];
    ov[pos[j]] = vals[sidx[j]];
}

// counts[0] = longest chain, counts[1] = live keys, counts[2] = nodes in chains; counts[3] = 1 if a
// chain is longer than SHORT_CHAIN nodes (the other counts are then incomplete)
template <class K>
__global__ void k_stats(DevIdx<K> ix, unsigned long long* __restrict__ out)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ix.nb) return;
    unsigned long long c = 0, k = 0;
    for (uint32_t x = ix.head[b]; x != NIL; x = ix.next[x]) {
        if (c == SHORT_CHAIN) { atomicOr(&out[3], 1ull); break; }
        c++;
        k += ix.size[x];
    }
    atomicMax(&out[0], c);
    atomicAdd(&out[1], k);
    atomicAdd(&out[2], c);
}

// Elastic split, pass 1: per bucket, how many buckets it becomes.
template <class K>
__global__ void k_split_count(DevIdx<K> ix, uint32_t max_chain, const uint32_t* __restrict__ uoff,
                              uint64_t* __restrict__ cnt)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ix.nb) return;
    if (uoff && uoff[b] == uoff[b + 1]) { cnt[b] = 1; return; }
    uint64_t L = 0;
    for (uint32_t x = ix.head[b]; x != NIL; x = ix.next[x]) {
        if (++L > ix.cap) { atomicOr(ix.err, ERR_CHAIN); break; }
    }
    cnt[b] = L > max_chain ? L : 1;
}

// Elastic split, pass 2: the new MKBA and heads.  A split chain's nodes are unlinked and each
// becomes a bucket whose maxBucket is the node's maxKey (the last node's maxKey is the old
// maxBucket); other buckets are copied.
template <class K>
__global__ void k_split_write(DevIdx<K> ix, const uint64_t* __restrict__ cnt, const uint64_t* __restrict__ boff,
                              K* __restrict__ mkba2, uint32_t* __restrict__ head2)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ix.nb) return;
    const uint64_t o = boff[b], L = cnt[b];
    if (L == 1) {
        mkba2[o] = ix.mkba[b];
        head2[o] = ix.head[b];
        return;
    }
    uint32_t x = ix.head[b];
    for (uint64_t i = 0; i < L && x != NIL; i++) {
        const uint32_t nx = ix.next[x];
        head2[o + i] = x;
        mkba2[o + i] = ix.bound[x];
        ix.next[x] = NIL;
        x = nx;
    }
}

// Underfull-neighbour merge: walk the chain; while the current node and the next hold at most NS/2
// pairs together, the next node's pairs are appended to the current one (they are all larger),
// the current node takes its maxKey and node-link, and the next node goes on the free stack.
template <class K>
__global__ void k_merge_underfull(DevIdx<K> ix, const uint32_t* __restrict__ uoff, int gated, DevState* __restrict__ ds,
                                  uint32_t* __restrict__ free_ids, unsigned long long* __restrict__ freed)
{
    grid_dep_enter();
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= ix.nb) return;
    if (gated && !ds->applied) return;   // after a batch: only if the batch was applied
    if (uoff && uoff[b] == uoff[b + 1]) return;
    uint32_t a = ix.head[b];
    if (ix.next[a] == NIL) return;
    const uint32_t half = ix.NS / 2;
    uint32_t sa = ix.size[a];
    uint64_t steps = 0;
    for (uint32_t x = ix.next[a]; x != NIL; x = ix.next[a]) {
        if (++steps > ix.cap) { atomicOr(ix.err, ERR_CHAIN); return; }
        const uint32_t sx = ix.size[x];
        if (sa + sx <= half) {
            K* ak = ix.keys + (uint64_t)a * ix.NS + sa;
            K* av = ix.vals + (uint64_t)a * ix.NS + sa;
            const K* xk = ix.keys + (uint64_t)x * ix.NS;
            const K* xv = ix.vals + (uint64_t)x * ix.NS;
            for (uint32_t i = 0; i < sx; i++) {
                ak[i] = xk[i];
                av[i] = xv[i];
            }
            sa += sx;
            ix.size[a] = sa;
            ix.bound[a] = ix.bound[x];
            ix.next[a] = ix.next[x];
            free_ids[atomicAdd(&ds->free_top, 1ull)] = x;
            if (freed) atomicAdd(freed, 1ull);
        } else {
            a = x;
            sa = sx;
        }
    }
}

}  // namespace

// Forces the module loader to load every kernel of this file now (see preload_kernels).
void preload_build_kernels()
{
    cudaFuncAttributes a;
#define FLIX_TOUCH(...) cudaFuncGetAttributes(&a, __VA_ARGS__)
    FLIX_TOUCH(k_unmark_free);
    FLIX_TOUCH(k_chain_count);
    FLIX_TOUCH(k_chain_max);
#define FLIX_TOUCH_K(K)                      \
    FLIX_TOUCH(k_live_count<K>);             \
    FLIX_TOUCH(k_gather<K>);                 \
    FLIX_TOUCH(k_gather_cut<K>);             \
    FLIX_TOUCH(k_used_compact<K>);           \
    FLIX_TOUCH(k_node_sizes<K>);             \
    FLIX_TOUCH((k_gather_nodes<K, false>));  \
    FLIX_TOUCH((k_gather_nodes<K, true>));   \
    FLIX_TOUCH(k_cut_keys<K>);               \
    FLIX_TOUCH(k_cut_meta<K>);               \
    FLIX_TOUCH(k_dedupe_flags<K>);           \
    FLIX_TOUCH(k_dedupe_write<K>);           \
    FLIX_TOUCH(k_stats<K>);                  \
    FLIX_TOUCH(k_split_count<K>);            \
    FLIX_TOUCH(k_split_write<K>);            \
    FLIX_TOUCH(k_merge_underfull<K>)
    FLIX_TOUCH_K(uint32_t);
    FLIX_TOUCH_K(uint64_t);
#undef FLIX_TOUCH_K
#undef FLIX_TOUCH
}

template <class K>
cudaError_t live_count(Ctx& c, uint64_t* cnt, uint32_t* long_flag)
{
    cudaError_t e = fill_bytes(c, long_flag, 0, 4);
    if (e) return e;
    return launch(c, K_LIVE_COUNT, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_live_count<K>, dev_view<K>(c.h), cnt,
                  long_flag);
}

template <class K>
size_t node_order_scratch_bytes(uint64_t cap)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(cap) + al((cap + 1) * 4) + al(cap * sizeof(K)) * 2 + al(cap * 4) * 4 + al((cap + 1) * 8) +
           sort_scratch_bytes<K>(cap) + scan_scratch_bytes<uint32_t>(cap) + scan_scratch_bytes<uint64_t>(cap) + 4096;
}

template <class K>
int node_order(Ctx& c, NodeOrder<K>& no)
{
    flix_index* h = c.h;
    Arena& A = h->arena;
    const uint64_t cap = h->cap;
    uint8_t* mark = A.take<uint8_t>(cap);
    uint32_t* pos = A.take<uint32_t>(cap + 1);
    K* ubound = A.take<K>(cap);
    uint32_t* uid = A.take<uint32_t>(cap);
    if (!mark || !pos || !ubound || !uid) return FLIX_ENOMEM;
    cudaError_t e = fill_bytes(c, mark, 1, cap);
    if (!e)
        e = launch(c, K_LIVE_COUNT, dim3(div_up(cap, BT)), dim3(BT), 0, k_unmark_free, (const uint32_t*)h->free_ids,
                   (const DevState*)h->dstate, mark);
    if (!e) e = scan_exclusive<uint8_t, uint32_t>(c, mark, pos, cap);
    if (!e)
        e = launch(c, K_LIVE_COUNT, dim3(div_up(cap, BT)), dim3(BT), 0, k_used_compact<K>, dev_view<K>(h),
                   (const uint8_t*)mark, (const uint32_t*)pos, cap, ubound, uid);
    if (e) return FLIX_ECUDA;
    int r = readback_at(h, c.st, 0, {{pos + cap, 4}});
    if (r) return r;
    const uint64_t m = h->hpin[0];
    no.m = m;
    no.bound = A.take<K>(m ? m : 1);
    uint32_t* perm = A.take<uint32_t>(m ? m : 1);
    no.order = A.take<uint32_t>(m ? m : 1);
    uint32_t* osz = A.take<uint32_t>(m ? m : 1);
    no.noff = A.take<uint64_t>(m + 1);
    if (!no.bound || !perm || !no.order || !osz || !no.noff) return FLIX_ENOMEM;
    e = sort_pairs<K>(c, ubound, nullptr, no.bound, perm, m);
    if (!e && m)
        e = launch(c, K_LIVE_COUNT, dim3(div_up(m, BT)), dim3(BT), 0, k_node_sizes<K>, dev_view<K>(h),
                   (const uint32_t*)uid, (const uint32_t*)perm, m, no.order, osz);
    if (!e) e = scan_exclusive<uint32_t, uint64_t>(c, osz, no.noff, m);
    return e ? FLIX_ECUDA : FLIX_OK;
}

template <class K>
cudaError_t gather_nodes(Ctx& c, const NodeOrder<K>& no, K* out_k, K* out_v)
{
    return launch(c, K_GATHER, dim3(div_up(no.m * 32, BT)), dim3(BT), 0, k_gather_nodes<K, false>, dev_view<K>(c.h),
                  (const uint32_t*)no.order, (const uint64_t*)no.noff, no.m, c.h->p, (uint64_t)0, out_k, out_v);
}

template <class K>
cudaError_t gather_nodes_cut(Ctx& c, const NodeOrder<K>& no, uint64_t nb_new, K* k2, K* v2)
{
    return launch(c, K_GATHER, dim3(div_up(no.m * 32, BT)), dim3(BT), 0, k_gather_nodes<K, true>, dev_view<K>(c.h),
                  (const uint32_t*)no.order, (const uint64_t*)no.noff, no.m, c.h->p, nb_new, k2, v2);
}

template <class K>
cudaError_t chain_max_by_nodes(Ctx& c, const NodeOrder<K>& no, uint64_t* out_max)
{
    flix_index* h = c.h;
    Arena& A = h->arena;
    uint32_t* bk = A.take<uint32_t>(no.m ? no.m : 1);
    uint32_t* chain = A.take<uint32_t>(h->nb);
    if (!bk || !chain) return cudaErrorMemoryAllocation;
    cudaError_t e = fill_bytes(c, chain, 0, h->nb * 4);
    if (!e) e = fill_bytes(c, out_max, 0, 8);
    if (!e && no.m) e = partition<K>(c, static_cast<const K*>(h->mkba), h->nb, no.bound, no.m, nullptr, nullptr, bk);
    if (!e && no.m)
        e = launch(c, K_STATS, dim3(div_up(no.m, BT)), dim3(BT), 0, k_chain_count, (const uint32_t*)bk, no.m, chain);
    if (!e)
        e = launch(c, K_STATS, dim3(div_up(h->nb, BT)), dim3(BT), 0, k_chain_max, (const uint32_t*)chain, h->nb,
                   reinterpret_cast<unsigned long long*>(out_max));
    return e;
}

template <class K>
cudaError_t gather_live(Ctx& c, const uint64_t* goff, K* out_k, K* out_v)
{
    return launch(c, K_GATHER, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_gather<K>, dev_view<K>(c.h), goff, out_k,
                  out_v);
}

template <class K>
cudaError_t gather_cut(Ctx& c, const uint64_t* goff, uint64_t n, uint64_t nb_new, K* k2, K* v2)
{
    (void)n;
    return launch(c, K_GATHER, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_gather_cut<K>, dev_view<K>(c.h), goff, c.h->p,
                  nb_new, k2, v2);
}

template <class K>
cudaError_t cut_buckets(Ctx& c, const K* sk, const K* sv, uint64_t n, uint64_t nb_new)
{
    flix_index* h = c.h;
    h->nb = nb_new;
    DevIdx<K> ix = dev_view<K>(h);
    cudaError_t e = cudaSuccess;
    if (sk) {
        e = launch(c, K_CUT_KEYS, dim3(div_up(div_up(n, h->p) * 32ull, BT)), dim3(BT), 0, k_cut_keys<K>, ix, sk, sv, n,
                   h->p);
        if (e) return e;
    }
    const uint64_t work = nb_new > h->cap - nb_new ? nb_new : h->cap - nb_new;
    e = launch(c, K_CUT_META, dim3(div_up(work, BT)), dim3(BT), 0, k_cut_meta<K>, ix, sk, n, h->p, nb_new, h->cap,
               h->free_ids);
    if (e) return e;
    return set_free_top(c, h->cap - nb_new);
}

template <class K>
cudaError_t dedupe_sorted(Ctx& c, const K* skeys, const uint32_t* sidx, const K* vals, uint64_t n, K* ok, K* ov,
                          uint32_t* n_dev)
{
    Arena& A = c.h->arena;
    uint32_t* head = A.take<uint32_t>(n + 1);
    uint32_t* pos = A.take<uint32_t>(n + 1);
    if (!head || !pos) return cudaErrorMemoryAllocation;
    if (n == 0) return fill_bytes(c, n_dev, 0, 4);
    cudaError_t e = launch(c, K_DEDUPE, dim3(div_up(n, BT)), dim3(BT), 0, k_dedupe_flags<K>, skeys, n, head);
    if (e) return e;
    if ((e = scan_exclusive<uint32_t, uint32_t>(c, head, pos, n))) return e;
    if ((e = copy_words(c, n_dev, pos + n, 1))) return e;
    return launch(c, K_DEDUPE, dim3(div_up(n, BT)), dim3(BT), 0, k_dedupe_write<K>, skeys, sidx, vals, n,
                  (const uint32_t*)head, (const uint32_t*)pos, ok, ov);
}

template <class K>
cudaError_t split_count(Ctx& c, uint32_t max_chain, const uint32_t* uoff, uint64_t* cnt)
{
    return launch(c, K_SPLIT, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_split_count<K>, dev_view<K>(c.h), max_chain,
                  uoff, cnt);
}

template <class K>
cudaError_t split_write(Ctx& c, const uint64_t* cnt, const uint64_t* boff, K* mkba2, uint32_t* head2)
{
    return launch(c, K_SPLIT, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_split_write<K>, dev_view<K>(c.h), cnt, boff,
                  mkba2, head2);
}

template <class K>
cudaError_t merge_underfull(Ctx& c, const uint32_t* uoff, int gated, unsigned long long* freed)
{
    return launch(c, K_MERGE, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_merge_underfull<K>, dev_view<K>(c.h), uoff,
                  gated, c.h->dstate, c.h->free_ids, freed);
}

template <class K>
cudaError_t stats_kernel(Ctx& c, uint64_t* out3)
{
    cudaError_t e = fill_bytes(c, out3, 0, 4 * sizeof(uint64_t));
    if (e) return e;
    return launch(c, K_STATS, dim3(div_up(c.h->nb, BT)), dim3(BT), 0, k_stats<K>, dev_view<K>(c.h),
                  reinterpret_cast<unsigned long long*>(out3));
}

#define FLIX_BUILD_INST(K)                                                                                 \
    template cudaError_t live_count<K>(Ctx&, uint64_t*, uint32_t*);                                         \
    template size_t node_order_scratch_bytes<K>(uint64_t);                                                 \
    template int node_order<K>(Ctx&, NodeOrder<K>&);                                                       \
    template cudaError_t gather_nodes<K>(Ctx&, const NodeOrder<K>&, K*, K*);                               \
    template cudaError_t gather_nodes_cut<K>(Ctx&, const NodeOrder<K>&, uint64_t, K*, K*);                 \
    template cudaError_t chain_max_by_nodes<K>(Ctx&, const NodeOrder<K>&, uint64_t*);                      \
    template cudaError_t gather_live<K>(Ctx&, const uint64_t*, K*, K*);                                    \
    template cudaError_t gather_cut<K>(Ctx&, const uint64_t*, uint64_t, uint64_t, K*, K*);                 \
    template cudaError_t cut_buckets<K>(Ctx&, const K*, const K*, uint64_t, uint64_t);                     \
    template cudaError_t dedupe_sorted<K>(Ctx&, const K*, const uint32_t*, const K*, uint64_t, K*, K*,     \
                                          uint32_t*);                                                      \
    template cudaError_t stats_kernel<K>(Ctx&, uint64_t*);                                                 \
    template cudaError_t split_count<K>(Ctx&, uint32_t, const uint32_t*, uint64_t*);                       \
    template cudaError_t split_write<K>(Ctx&, const uint64_t*, const uint64_t*, K*, uint32_t*);            \
    template cudaError_t merge_underfull<K>(Ctx&, const uint32_t*, int, unsigned long long*);

FLIX_BUILD_INST(uint32_t)
FLIX_BUILD_INST(uint64_t)

}  // namespace flix
