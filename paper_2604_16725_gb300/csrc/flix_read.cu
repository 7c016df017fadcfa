// Read path: bucket partition of the sorted batch (Sec. 3.3, Sec. 4.1), point and successor
// queries (Sec. 3.3, Sec. 6.5) and range queries (named in Sec. 2.1; inclusive [lo, hi] here).
//
// Partition.  Bucket i owns the keys in (maxBucket_{i-1}, maxBucket_i]; its sublist starts at the
// first sorted key greater than maxBucket_{i-1}.  The paper finds that start with one binary search
// per bucket.  Here all starts come from one merge-path co-ranking of the sorted MKBA with the
// sorted batch (a key equal to a maxBucket goes before it), which yields the same offsets with
// coalesced reads and one global search per 2048 merged items.  The same merge also tells every
// operation its bucket (the number of maxBucket values below its key), which the read kernels use.
//
// Queries.  One thread per sorted query: it takes its bucket from the partition, walks the
// node-links from the bucket's first node to the first node with key <= maxKey (Sec. 4.1) and
// binary-searches that node.  Consecutive threads hold consecutive keys, so the threads of a warp
// share buckets and nodes and their loads coalesce or hit L1; a bucket that receives many queries
// (skew, or a padded batch's tail) is spread over as many threads as it has queries.
#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr int PT_THREADS = 256;
constexpr int PT_ITEMS = 8;
constexpr int PT_TILE = PT_THREADS * PT_ITEMS;
constexpr int RP_THREADS = 256;

// Smallest a in [max(0, d - nB), min(d, nA)] such that A[a] >= B[d - 1 - a]: the number of A
// items among the first d items of the merge of A and B when B wins ties.
template <class K>
__device__ __forceinline__ uint64_t corank(const K* __restrict__ A, uint64_t nA, const K* __restrict__ B,
                                           uint64_t nB, uint64_t d)
{
    uint64_t lo = d > nB ? d - nB : 0, hi = d < nA ? d : nA;
    while (lo < hi) {
        uint64_t mid = (lo + hi) >> 1;
        if (A[mid] >= B[d - 1 - mid]) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// Merge-path split points: ca[t] = A items among the first min(t * PT_TILE, nA + m) items of the
// merge of A = mkba and B = the sorted batch (B wins ties), for t = 0..ntiles.
template <class K>
__global__ void __launch_bounds__(256) k_corank(const K* __restrict__ mkba, uint64_t nA, const K* __restrict__ skeys,
                                                uint64_t mmax, const uint32_t* __restrict__ m_dev,
                                                uint64_t* __restrict__ ca, uint32_t ntiles)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > ntiles) return;
    const uint64_t m = m_dev ? (uint64_t)*m_dev : mmax;
    const uint64_t L = nA + m;
    const uint64_t d = (uint64_t)t * PT_TILE < L ? (uint64_t)t * PT_TILE : L;
    ca[t] = corank(mkba, nA, skeys, m, d);
}

// First index in s[0..len) whose value is >= q (lower) or > q (upper).
template <class K, bool UPPER>
__device__ __forceinline__ uint32_t smem_bound(const K* s, uint32_t len, K q)
{
    uint32_t base = 0;
    while (len > 0) {
        const uint32_t half = len >> 1;
        const K v = s[base + half];
        if (UPPER ? !(q < v) : (v < q)) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// One merge-path tile of PT_TILE merged items per block: off[i + 1] = number of batch keys <=
// mkba[i] (off may be null); bk[j] = bucket of batch key j = number of mkba entries < key j (bk may
// be null).  Inside the tile each item finds its rank among the other side's tile items by binary
// search in shared memory; items are thread-strided, so the writes coalesce.
template <class K>
__global__ void __launch_bounds__(PT_THREADS) k_partition(const K* __restrict__ mkba, const K* __restrict__ skeys,
                                                          const uint64_t* __restrict__ ca, uint64_t nA, uint64_t mmax,
                                                          const uint32_t* __restrict__ m_dev,
                                                          uint32_t* __restrict__ off, uint32_t* __restrict__ bk)
{
    __shared__ K sA[PT_TILE];
    __shared__ K sB[PT_TILE];
    const uint64_t m = m_dev ? (uint64_t)*m_dev : mmax;
    const uint64_t L = nA + m;
    const uint64_t d0 = (uint64_t)blockIdx.x * PT_TILE;
    if (d0 >= L) return;
    const uint64_t d1 = d0 + PT_TILE < L ? d0 + PT_TILE : L;
    if (off && blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
    const uint64_t a0 = ca[blockIdx.x], a1 = ca[blockIdx.x + 1];
    const uint64_t b0 = d0 - a0, b1 = d1 - a1;
    const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - b0);
    for (uint32_t t = threadIdx.x; t < la; t += PT_THREADS) sA[t] = mkba[a0 + t];
    for (uint32_t t = threadIdx.x; t < lb; t += PT_THREADS) sB[t] = skeys[b0 + t];
    __syncthreads();
    if (bk)
        for (uint32_t t = threadIdx.x; t < lb; t += PT_THREADS)
            bk[b0 + t] = (uint32_t)(a0 + smem_bound<K, false>(sA, la, sB[t]));
    if (off)
        for (uint32_t t = threadIdx.x; t < la; t += PT_THREADS)
            off[a0 + t + 1] = (uint32_t)(b0 + smem_bound<K, true>(sB, lb, sA[t]));
}

// First position in nk[0..sz) whose key is >= q.
template <class K>
__device__ __forceinline__ uint32_t node_lower_bound(const K* __restrict__ nk, uint32_t sz, K q)
{
    uint32_t base = 0, len = sz;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (__ldg(nk + base + half) < q) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// First position in nk[from..sz) whose key is > q.
template <class K>
__device__ __forceinline__ uint32_t node_upper_bound(const K* __restrict__ nk, uint32_t from, uint32_t sz, K q)
{
    uint32_t base = from, len = sz - from;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (!(q < __ldg(nk + base + half))) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// From bucket b's first node, walk node-links to the first node whose maxKey >= q (Sec. 4.1).
template <class K>
__device__ __forceinline__ bool find_node(const DevIdx<K>& ix, uint32_t b, K q, uint32_t& node, uint32_t& sz, K& bd,
                                          uint32_t& nx)
{
    node = __ldg(ix.head + b);
    sz = __ldg(ix.size + node);
    bd = __ldg(ix.bound + node);
    nx = __ldg(ix.next + node);
    uint32_t steps = 0;
    while (q > bd) {
        if (nx == NIL || ++steps > ix.cap) { atomicOr(ix.err, ERR_CHAIN); return false; }
        node = nx;
        sz = __ldg(ix.size + node);
        bd = __ldg(ix.bound + node);
        nx = __ldg(ix.next + node);
    }
    return true;
}

template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_read_point(DevIdx<K> ix, int mode, const K* __restrict__ skeys,
                                                           const uint32_t* __restrict__ sidx, uint64_t m,
                                                           const uint32_t* __restrict__ bk,
                                                           const uint8_t* __restrict__ ops, K* __restrict__ keys_out,
                                                           K* __restrict__ vals_out, uint8_t* __restrict__ found_out)
{
    const uint64_t j = (uint64_t)blockIdx.x * RP_THREADS + threadIdx.x;
    if (j >= m) return;
    const uint32_t idx = sidx[j];
    const int op = mode ? mode : ops[idx];
    const K KM = key_max<K>();
    K rk = KM, rv = KM;
    uint8_t f = 0;
    if (op == FLIX_OP_LOOKUP || op == FLIX_OP_SUCC) {
        const K q = skeys[j];
        const uint32_t b = bk[j];
        const uint32_t NS = ix.NS;
        uint32_t node, sz, nx;
        K bd;
        if (find_node(ix, b, q, node, sz, bd, nx)) {
            const K* nk = ix.keys + (uint64_t)node * NS;
            const uint32_t pos = node_lower_bound(nk, sz, q);
            if (op == FLIX_OP_LOOKUP) {
                if (pos < sz && __ldg(nk + pos) == q) {
                    rk = q;
                    rv = __ldg(ix.vals + (uint64_t)node * NS + pos);
                    f = 1;
                }
            } else if (pos < sz) {
                rk = __ldg(nk + pos);
                rv = __ldg(ix.vals + (uint64_t)node * NS + pos);
                f = 1;
            } else {
                // the smallest key >= q is the first key of the next non-empty node in chain order,
                // continuing into the following buckets
                uint32_t n2 = nx;
                uint64_t bb = b;
                for (uint64_t guard = 0, lim = (uint64_t)ix.cap + ix.nb + 1; guard < lim; guard++) {
                    if (n2 == NIL) {
                        if (++bb >= ix.nb) break;
                        n2 = ix.head[bb];
                        continue;
                    }
                    if (ix.size[n2] > 0) {
                        rk = ix.keys[(uint64_t)n2 * NS];
                        rv = ix.vals[(uint64_t)n2 * NS];
                        f = 1;
                        break;
                    }
                    n2 = ix.next[n2];
                }
            }
        }
    }
    if (keys_out) keys_out[idx] = rk;
    if (vals_out) vals_out[idx] = rv;
    if (found_out) found_out[idx] = f;
}

// Range count: per range query, the start (bucket, node, position) and the number of stored keys
// in [lo, hi].  Nodes whose maxKey <= hi are counted from their size alone.
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_range_count(DevIdx<K> ix, const K* __restrict__ skeys,
                                                            const uint32_t* __restrict__ sidx, uint64_t m,
                                                            const uint32_t* __restrict__ bk,
                                                            const uint8_t* __restrict__ ops, const K* __restrict__ hi_arr,
                                                            uint32_t* __restrict__ start_bucket,
                                                            uint32_t* __restrict__ start_node,
                                                            uint32_t* __restrict__ start_pos, uint64_t* __restrict__ cnt)
{
    const uint64_t j = (uint64_t)blockIdx.x * RP_THREADS + threadIdx.x;
    if (j >= m) return;
    const uint32_t idx = sidx[j];
    if (ops && ops[idx] != FLIX_OP_RANGE) {
        cnt[idx] = 0;
        return;
    }
    const uint32_t NS = ix.NS;
    const K lo = skeys[j];
    const K hi = hi_arr[idx];
    uint32_t bb = bk[j];
    uint32_t node, sz, nx;
    K bd;
    uint64_t c = 0;
    if (!find_node(ix, bb, lo, node, sz, bd, nx)) {
        cnt[idx] = 0;
        start_bucket[j] = bb;
        start_node[j] = ix.head[bb];
        start_pos[j] = 0;
        return;
    }
    uint32_t pos = node_lower_bound(ix.keys + (uint64_t)node * NS, sz, lo);
    start_bucket[j] = bb;
    start_node[j] = node;
    start_pos[j] = pos;
    if (lo <= hi) {
        for (uint64_t guard = 0, lim = (uint64_t)ix.cap + ix.nb + 1; guard < lim; guard++) {
            if (bd <= hi) {
                c += sz - pos;
            } else {
                c += node_upper_bound(ix.keys + (uint64_t)node * NS, pos, sz, hi) - pos;
                break;
            }
            node = nx;
            while (node == NIL) {
                if (++bb >= ix.nb) break;
                node = ix.head[bb];
            }
            if (node == NIL) break;
            sz = ix.size[node];
            bd = ix.bound[node];
            nx = ix.next[node];
            pos = 0;
        }
    }
    cnt[idx] = c;
}

// Range fill: one warp per sorted query copies its pairs node by node (coalesced).
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_range_fill(DevIdx<K> ix, const uint32_t* __restrict__ sidx,
                                                           uint64_t m, const uint8_t* __restrict__ ops,
                                                           const uint32_t* __restrict__ start_bucket,
                                                           const uint32_t* __restrict__ start_node,
                                                           const uint32_t* __restrict__ start_pos,
                                                           const uint64_t* __restrict__ roff, K* __restrict__ rkeys,
                                                           K* __restrict__ rvals, const DevState* __restrict__ ds)
{
    if (ds && !ds->admitted) return;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t j = ((uint64_t)blockIdx.x * RP_THREADS + threadIdx.x) >> 5;
    if (j >= m) return;
    const uint32_t idx = sidx[j];
    if (ops && ops[idx] != FLIX_OP_RANGE) return;
    uint64_t o = roff[idx];
    uint64_t c = roff[idx + 1] - o;
    if (c == 0) return;
    const uint32_t NS = ix.NS;
    uint32_t bb = start_bucket[j];
    uint32_t node = start_node[j];
    uint32_t pos = start_pos[j];
    for (uint64_t guard = 0, lim = (uint64_t)ix.cap + ix.nb + 1; guard < lim && c > 0; guard++) {
        const uint32_t sz = ix.size[node];
        const uint32_t avail = sz > pos ? sz - pos : 0;
        const uint32_t take = (uint64_t)avail < c ? avail : (uint32_t)c;
        const K* nk = ix.keys + (uint64_t)node * NS + pos;
        const K* nv = ix.vals + (uint64_t)node * NS + pos;
        for (uint32_t t = lane; t < take; t += 32) {
            rkeys[o + t] = nk[t];
            rvals[o + t] = nv[t];
        }
        o += take;
        c -= take;
        pos = 0;
        if (c == 0) break;
        node = ix.next[node];
        while (node == NIL) {
            if (++bb >= ix.nb) { if (lane == 0) atomicOr(ix.err, ERR_RANGE); return; }
            node = ix.head[bb];
        }
    }
}

}  // namespace

size_t partition_scratch_bytes(uint64_t nb, uint64_t m)
{
    return ((size_t)(div_up(nb + m, PT_TILE) + 1) * 8 + 255) & ~size_t(255);
}

template <class K>
cudaError_t partition(Ctx& c, const K* mkba, uint64_t nb, const K* skeys, uint64_t m, const uint32_t* m_dev,
                      uint32_t* off, uint32_t* bk)
{
    const uint32_t grid = div_up(nb + m, PT_TILE);
    uint64_t* ca = c.h->arena.take<uint64_t>((size_t)grid + 1);
    if (!ca) return cudaErrorMemoryAllocation;
    cudaError_t e = launch(c, K_PARTITION, dim3(div_up((uint64_t)grid + 1, 256)), dim3(256), 0, k_corank<K>, mkba, nb,
                           skeys, m, m_dev, ca, grid);
    if (e) return e;
    return launch(c, K_PARTITION, dim3(grid), dim3(PT_THREADS), 0, k_partition<K>, mkba, skeys, (const uint64_t*)ca,
                  nb, m, m_dev, off, bk);
}

template <class K>
cudaError_t read_point(Ctx& c, int mode, const K* skeys, const uint32_t* sidx, uint64_t m, const uint32_t* bk,
                       const uint8_t* ops, K* keys_out, K* vals_out, uint8_t* found_out)
{
    if (m == 0) return cudaSuccess;
    return launch(c, K_READ_POINT, dim3(div_up(m, RP_THREADS)), dim3(RP_THREADS), 0, k_read_point<K>,
                  dev_view<K>(c.h), mode, skeys, sidx, m, bk, ops, keys_out, vals_out, found_out);
}

template <class K>
cudaError_t range_count(Ctx& c, const K* skeys, const uint32_t* sidx, uint64_t m, const uint32_t* bk,
                        const uint8_t* ops, const K* hi, uint32_t* start_bucket, uint32_t* start_node,
                        uint32_t* start_pos, uint64_t* cnt)
{
    if (m == 0) return cudaSuccess;
    return launch(c, K_RANGE_COUNT, dim3(div_up(m, RP_THREADS)), dim3(RP_THREADS), 0, k_range_count<K>,
                  dev_view<K>(c.h), skeys, sidx, m, bk, ops, hi, start_bucket, start_node, start_pos, cnt);
}

template <class K>
cudaError_t range_fill(Ctx& c, const uint32_t* sidx, uint64_t m, const uint8_t* ops, const uint32_t* start_bucket,
                       const uint32_t* start_node, const uint32_t* start_pos, const uint64_t* roff, K* rkeys, K* rvals,
                       bool gated)
{
    if (m == 0) return cudaSuccess;
    const uint32_t grid = div_up(m * 32, RP_THREADS);
    return launch(c, K_RANGE_FILL, dim3(grid), dim3(RP_THREADS), 0, k_range_fill<K>, dev_view<K>(c.h), sidx, m, ops,
                  start_bucket, start_node, start_pos, roff, rkeys, rvals,
                  gated ? (const DevState*)c.h->dstate : (const DevState*)nullptr);
}

#define FLIX_READ_INST(K)                                                                                       \
    template cudaError_t partition<K>(Ctx&, const K*, uint64_t, const K*, uint64_t, const uint32_t*, uint32_t*, \
                                      uint32_t*);                                                               \
    template cudaError_t read_point<K>(Ctx&, int, const K*, const uint32_t*, uint64_t, const uint32_t*,        \
                                       const uint8_t*, K*, K*, uint8_t*);                                      \
    template cudaError_t range_count<K>(Ctx&, const K*, const uint32_t*, uint64_t, const uint32_t*,           \
                                        const uint8_t*, const K*, uint32_t*, uint32_t*, uint32_t*, uint64_t*); \
    template cudaError_t range_fill<K>(Ctx&, const uint32_t*, uint64_t, const uint8_t*, const uint32_t*,       \
                                       const uint32_t*, const uint32_t*, const uint64_t*, K*, K*, bool);

FLIX_READ_INST(uint32_t)
FLIX_READ_INST(uint64_t)

}  // namespace flix
