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

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int PT_THREADS = 256;
constexpr int PT_ITEMS = 8;
constexpr int PT_TILE = PT_THREADS * PT_ITEMS;
constexpr int RP_THREADS = 256;

// Merge-path split points: ca[t] = A items among the first min(t * PT_TILE, nA + m) items of the
// merge of A = mkba and B = the sorted batch (B wins ties), for t = 0..ntiles.  One warp per split
// point: each round probes 32 points of the bracket at once (the test A[a] >= B[d - 1 - a] turns
// from false to true once along it), so about five dependent rounds replace a binary search's 25.
template <class K>
__global__ void __launch_bounds__(256) k_corank(const K* __restrict__ mkba, uint64_t nA, const K* __restrict__ skeys,
                                                uint64_t mmax, const uint32_t* __restrict__ m_dev,
                                                uint64_t* __restrict__ ca, uint32_t ntiles)
{
    grid_dep_enter();
    const uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = threadIdx.x & 31;
    if (t > ntiles) return;                     // whole warps leave together
    const uint64_t m = m_dev ? (uint64_t)*m_dev : mmax;
    const uint64_t L = nA + m;
    const uint64_t d = (uint64_t)t * PT_TILE < L ? (uint64_t)t * PT_TILE : L;
    uint64_t lo = d > m ? d - m : 0, hi = d < nA ? d : nA;   // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const uint64_t x = lo + ((hi - lo) * (lane + 1)) / 33;   // lo <= x < hi
        const uint32_t bal = __ballot_sync(FULL, mkba[x] >= skeys[d - 1 - x]);
        const uint32_t f = bal ? __ffs(bal) - 1 : 32;
        const uint64_t xf = __shfl_sync(FULL, x, f & 31);
        const uint64_t xp = __shfl_sync(FULL, x, (f + 31) & 31);
        if (f < 32) hi = xf;
        lo = f == 0 ? lo : xp + 1;
    }
    const uint64_t x = lo + lane;
    const uint32_t bal = __ballot_sync(FULL, x < hi && mkba[x] >= skeys[d - 1 - x]);
    if (lane == 0) ca[t] = bal ? lo + __ffs(bal) - 1 : hi;
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
// be null).  Inside the tile each thread merges PT_ITEMS consecutive merged items: it finds where
// its diagonal crosses the two sorted slices (a binary search in shared memory), then walks its
// items in order, a batch key taking the bucket after the mkba entries passed so far and an mkba
// entry the count of batch keys passed so far (ties: the batch key first).  Results are staged in
// shared memory and written out coalesced.
template <class K>
__global__ void __launch_bounds__(PT_THREADS) k_partition(const K* __restrict__ mkba, const K* __restrict__ skeys,
                                                          const uint64_t* __restrict__ ca, uint64_t nA, uint64_t mmax,
                                                          const uint32_t* __restrict__ m_dev,
                                                          uint32_t* __restrict__ off, uint32_t* __restrict__ bk)
{
    grid_dep_enter();
    __shared__ K sA[PT_TILE];
    __shared__ K sB[PT_TILE];
    __shared__ uint32_t sout[PT_TILE];   // bk of B item t at t; off of A item t at PT_TILE - 1 - t
    const uint64_t m = m_dev ? (uint64_t)*m_dev : mmax;
    const uint64_t L = nA + m;
    const uint64_t d0 = (uint64_t)blockIdx.x * PT_TILE;
    if (d0 >= L) return;
    const uint64_t d1 = d0 + PT_TILE < L ? d0 + PT_TILE : L;
    if (off && blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
    const uint64_t a0 = ca[blockIdx.x], a1 = ca[blockIdx.x + 1];
    const uint64_t b0 = d0 - a0, b1 = d1 - a1;
    const uint32_t la = (uint32_t)(a1 - a0), lb = (uint32_t)(b1 - b0);
    {
        // every load of the tile is issued before the first store to shared memory
        K ra[PT_ITEMS], rb[PT_ITEMS];
#pragma unroll
        for (int r = 0; r < PT_ITEMS; r++) {
            const uint32_t t = r * PT_THREADS + threadIdx.x;
            if (t < la) ra[r] = mkba[a0 + t];
            if (t < lb) rb[r] = skeys[b0 + t];
        }
#pragma unroll
        for (int r = 0; r < PT_ITEMS; r++) {
            const uint32_t t = r * PT_THREADS + threadIdx.x;
            if (t < la) sA[t] = ra[r];
            if (t < lb) sB[t] = rb[r];
        }
    }
    __syncthreads();
    const uint32_t n = la + lb;
    const uint32_t k0 = threadIdx.x * PT_ITEMS;
    if (k0 < n) {
        // split of diagonal k0: the smallest i with sA[i] >= sB[k0 - 1 - i] (A items among the first k0)
        uint32_t lo = k0 > lb ? k0 - lb : 0, hi = k0 < la ? k0 : la;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (sA[mid] >= sB[k0 - 1 - mid]) hi = mid; else lo = mid + 1;
        }
        uint32_t i = lo, j = k0 - lo;
        const uint32_t kend = k0 + PT_ITEMS < n ? k0 + PT_ITEMS : n;
        for (uint32_t k = k0; k < kend; k++) {
            if (j < lb && (i >= la || !(sA[i] < sB[j]))) {
                sout[j] = i;                      // batch key j: i mkba entries of the tile are below it
                j++;
            } else {
                sout[PT_TILE - 1 - i] = j;        // mkba entry i: j batch keys of the tile are <= it
                i++;
            }
        }
    }
    __syncthreads();
    if (bk)
        for (uint32_t t = threadIdx.x; t < lb; t += PT_THREADS) bk[b0 + t] = (uint32_t)(a0 + sout[t]);
    if (off)
        for (uint32_t t = threadIdx.x; t < la; t += PT_THREADS) off[a0 + t + 1] = (uint32_t)(b0 + sout[PT_TILE - 1 - t]);
}

// Windowed result delivery (see read_point), passed by value.  Window w holds input positions
// [w << shift, (w + 1) << shift); the reads of a batch deliver every input position exactly once, so
// window w's region of the tagged arrays is that same range, and a block reserves its place in it
// from the window's cursor.
constexpr uint32_t RP_MAX_WIN = 256;
template <class K>
struct ReadWin {
    int shift;
    uint32_t* cur;           // per window: results placed so far (zero before the read kernel)
    uint32_t* idx;           // input position of each windowed result
    K* rk;
    K* rv;
    uint8_t* rf;
};

// Point reads, one thread per sorted query (bucket bk from the partition).  Results go to the
// query's input position, or, with win, tagged with it into its window's region for k_win_scatter:
// a block counts its results per window in shared memory, then reserves one run per window with
// one atomic on the window's cursor.
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_read_point(DevIdx<K> ix, int mode, const K* __restrict__ skeys,
                                                           const uint32_t* __restrict__ sidx, uint64_t m,
                                                           const uint32_t* __restrict__ bk,
                                                           const uint8_t* __restrict__ ops, K* __restrict__ keys_out,
                                                           K* __restrict__ vals_out, uint8_t* __restrict__ found_out,
                                                           const ReadWin<K> win, uint32_t nwin)
{
    grid_dep_enter();
    __shared__ uint32_t s_wcnt[RP_MAX_WIN];
    __shared__ uint32_t s_wbase[RP_MAX_WIN];
    if (nwin) {
        for (uint32_t w = threadIdx.x; w < nwin; w += RP_THREADS) s_wcnt[w] = 0;
        __syncthreads();
    }
    const uint64_t j = (uint64_t)blockIdx.x * RP_THREADS + threadIdx.x;
    const bool active = j < m;              // every thread stays for the block's barriers
    const K KM = key_max<K>();
    uint32_t idx = 0;
    K rk = KM, rv = KM;
    uint8_t f = 0;
    if (active) {
        idx = sidx[j];
        const int op = mode ? mode : ops[idx];
        if (op == FLIX_OP_LOOKUP || op == FLIX_OP_SUCC || op == FLIX_OP_PRED) {
            const K q = skeys[j];
            const uint32_t b = bk[j];
            uint32_t node, sz, nx, prev;
            K bd;
            if (find_node(ix, b, q, node, sz, bd, nx, prev)) {   // else: chain error flagged, default results
                const K* nk = ix.keys + (uint64_t)node * ix.NS;
                uint32_t pos;
                K kpos = K(0);
                if (op == FLIX_OP_PRED) {
                    pos = node_upper_bound(nk, 0, sz, q);
                    if (pos > 0) kpos = __ldg(nk + pos - 1);
                } else {
                    pos = node_lower_bound(nk, sz, q);
                    if (pos < sz) kpos = __ldg(nk + pos);
                }
                point_result(ix, op, q, b, node, sz, nx, prev, pos, kpos, rk, rv, f);
            }
        }
    }
    if (!nwin) {
        if (active) {
            if (keys_out) keys_out[idx] = rk;
            if (vals_out) vals_out[idx] = rv;
            if (found_out) found_out[idx] = f;
        }
        return;
    }
    const uint32_t w = idx >> win.shift;
    const uint32_t r = active ? atomicAdd(&s_wcnt[w], 1u) : 0u;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < nwin; t += RP_THREADS) {
        const uint32_t c = s_wcnt[t];
        s_wbase[t] = c ? (t << win.shift) + atomicAdd(win.cur + t, c) : 0u;
    }
    __syncthreads();
    if (active) {
        const uint64_t at = (uint64_t)s_wbase[w] + r;
        win.idx[at] = idx;
        if (keys_out) win.rk[at] = rk;
        if (vals_out) win.rv[at] = rv;
        if (found_out) win.rf[at] = f;
    }
}

// Second half of the windowed delivery: results are read in window order, so the scattered
// writes of the blocks in flight fall in a few windows' worth of output and merge in L2.  (One
// result per thread: four per thread, loads first, measured slower.)
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_win_scatter(const uint32_t* __restrict__ widx, uint64_t m,
                                                            const K* __restrict__ rk, const K* __restrict__ rv,
                                                            const uint8_t* __restrict__ rf, K* __restrict__ keys_out,
                                                            K* __restrict__ vals_out, uint8_t* __restrict__ found_out)
{
    grid_dep_enter();
    const uint64_t p = (uint64_t)blockIdx.x * RP_THREADS + threadIdx.x;
    if (p >= m) return;
    const uint32_t i = widx[p];
    if (keys_out) keys_out[i] = rk[p];
    if (vals_out) vals_out[i] = rv[p];
    if (found_out) found_out[i] = rf[p];
}

// Range count: per range query, the start (bucket, node, position) and the number of stored keys
// in [lo, hi].  Nodes whose maxKey <= hi are counted from their size alone.  (One thread per query:
// a batch holds enough queries to keep every SM busy; the persistent queue kernel, with few queries
// per batch, counts each by a warp instead.)
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_range_count(DevIdx<K> ix, const K* __restrict__ skeys,
                                                            const uint32_t* __restrict__ sidx, uint64_t m,
                                                            const uint32_t* __restrict__ bk,
                                                            const uint8_t* __restrict__ ops, const K* __restrict__ hi_arr,
                                                            uint32_t* __restrict__ start_bucket,
                                                            uint32_t* __restrict__ start_node,
                                                            uint32_t* __restrict__ start_pos, uint64_t* __restrict__ cnt)
{
    grid_dep_enter();
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
    uint32_t prev;
    if (!find_node(ix, bb, lo, node, sz, bd, nx, prev)) {
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
            // entering the next bucket: node bb is usually its first node (see find_node), so its
            // metadata is read beside the head and kept when the head confirms it
            bool spec = false;
            uint32_t s_sz = 0, s_nx = NIL;
            K s_bd = K(0);
            while (node == NIL) {
                if (++bb >= ix.nb) break;
                node = ix.head[bb];
                s_sz = ix.size[bb];
                s_bd = ix.bound[bb];
                s_nx = ix.next[bb];
                spec = true;
            }
            if (node == NIL) break;
            if (spec && node == bb) {
                sz = s_sz;
                bd = s_bd;
                nx = s_nx;
            } else {
                sz = ix.size[node];
                bd = ix.bound[node];
                nx = ix.next[node];
            }
            pos = 0;
        }
    }
    cnt[idx] = c;
}

// Range fill: one warp per sorted query (range_fill_warp).
template <class K>
__global__ void __launch_bounds__(RP_THREADS) k_range_fill(DevIdx<K> ix, const uint32_t* __restrict__ sidx,
                                                           uint64_t m, const uint8_t* __restrict__ ops,
                                                           const uint32_t* __restrict__ start_bucket,
                                                           const uint32_t* __restrict__ start_node,
                                                           const uint32_t* __restrict__ start_pos,
                                                           const uint64_t* __restrict__ roff, K* __restrict__ rkeys,
                                                           K* __restrict__ rvals, const DevState* __restrict__ ds)
{
    grid_dep_enter();
    if (ds && !ds->admitted) return;
    const uint64_t j = ((uint64_t)blockIdx.x * RP_THREADS + threadIdx.x) >> 5;
    if (j >= m) return;
    const uint32_t idx = sidx[j];
    if (ops && ops[idx] != FLIX_OP_RANGE) return;
    uint64_t o = roff[idx];
    uint64_t c = roff[idx + 1] - o;
    if (c == 0) return;
    range_fill_warp(ix, (uint64_t)start_bucket[j], start_node[j], start_pos[j], o, c, rkeys, rvals);
}

}  // namespace

// Forces the module loader to load every kernel of this file now (see preload_kernels).
void preload_read_kernels()
{
    cudaFuncAttributes a;
#define FLIX_TOUCH(...) cudaFuncGetAttributes(&a, __VA_ARGS__)
#define FLIX_TOUCH_K(K)                      \
    FLIX_TOUCH(k_corank<K>);                 \
    FLIX_TOUCH(k_partition<K>);              \
    FLIX_TOUCH(k_read_point<K>);             \
    FLIX_TOUCH(k_win_scatter<K>);            \
    FLIX_TOUCH(k_range_count<K>);            \
    FLIX_TOUCH(k_range_fill<K>)
    FLIX_TOUCH_K(uint32_t);
    FLIX_TOUCH_K(uint64_t);
#undef FLIX_TOUCH_K
#undef FLIX_TOUCH
}

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
    cudaError_t e = launch(c, K_PARTITION, dim3(div_up(((uint64_t)grid + 1) * 32, 256)), dim3(256), 0, k_corank<K>,
                           mkba, nb, skeys, m, m_dev, ca, grid);
    if (e) return e;
    return launch(c, K_PARTITION, dim3(grid), dim3(PT_THREADS), 0, k_partition<K>, mkba, skeys, (const uint64_t*)ca,
                  nb, m, m_dev, off, bk);
}

// Results scattered to random input positions cost a read-modify-write of a DRAM sector each once
// they no longer fit in L2.  Above RP_WIN_BYTES of results, homogeneous reads deliver them in two
// steps instead: the read kernel writes each result, tagged with its input position, into the
// region of its window of input positions (about RP_WIN_TARGET bytes of output per window), and
// k_win_scatter reads the regions in order and writes the results to their positions.
constexpr uint64_t RP_WIN_BYTES = 96ull << 20;
constexpr uint64_t RP_WIN_TARGET = 4ull << 20;

template <class K>
size_t read_point_scratch_bytes(uint64_t m)
{
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    return al(m * sizeof(K)) * 2 + al(m) + al(m * 4) + al(RP_MAX_WIN * 4) + 1024;
}

template <class K>
cudaError_t read_point(Ctx& c, int mode, const K* skeys, const uint32_t* sidx, uint64_t m, const uint32_t* bk,
                       const uint8_t* ops, K* keys_out, K* vals_out, uint8_t* found_out)
{
    if (m == 0) return cudaSuccess;
    const uint32_t nblk = div_up(m, RP_THREADS);
    const uint64_t per = (keys_out ? sizeof(K) : 0) + (vals_out ? sizeof(K) : 0) + (found_out ? 1 : 0);
    if (!ops && m * per > RP_WIN_BYTES && m < (1ull << 32)) {
        // window size: a power of two near RP_WIN_TARGET bytes of output, at most RP_MAX_WIN windows
        int shift = 0;
        while (shift < 31 && ((2ull << shift) * per <= RP_WIN_TARGET || ((m - 1) >> shift) + 1 > RP_MAX_WIN)) shift++;
        const uint32_t nwin = (uint32_t)(((m - 1) >> shift) + 1);
        Arena& A = c.h->arena;
        const size_t mark = A.used;
        ReadWin<K> hw;
        hw.shift = shift;
        hw.cur = A.take<uint32_t>(nwin);
        hw.idx = A.take<uint32_t>(m);
        hw.rk = keys_out ? A.take<K>(m) : nullptr;
        hw.rv = vals_out ? A.take<K>(m) : nullptr;
        hw.rf = found_out ? A.take<uint8_t>(m) : nullptr;
        if (hw.cur && hw.idx && (!keys_out || hw.rk) && (!vals_out || hw.rv) && (!found_out || hw.rf)) {
            cudaError_t e = fill_bytes(c, hw.cur, 0, (size_t)nwin * 4);
            if (!e)
                e = launch(c, K_READ_POINT, dim3(nblk), dim3(RP_THREADS), 0, k_read_point<K>, dev_view<K>(c.h), mode,
                           skeys, sidx, m, bk, ops, keys_out, vals_out, found_out, hw, nwin);
            if (!e)
                e = launch(c, K_UNSORT, dim3(nblk), dim3(RP_THREADS), 0, k_win_scatter<K>, (const uint32_t*)hw.idx, m,
                           (const K*)hw.rk, (const K*)hw.rv, (const uint8_t*)hw.rf, keys_out, vals_out, found_out);
            return e;
        }
        A.used = mark;   // no room for the windowed results: scatter directly
    }
    return launch(c, K_READ_POINT, dim3(nblk), dim3(RP_THREADS), 0, k_read_point<K>, dev_view<K>(c.h), mode, skeys,
                  sidx, m, bk, ops, keys_out, vals_out, found_out, ReadWin<K>{}, 0u);
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
    template size_t read_point_scratch_bytes<K>(uint64_t);                                                     \
    template cudaError_t range_count<K>(Ctx&, const K*, const uint32_t*, uint64_t, const uint32_t*,           \
                                        const uint8_t*, const K*, uint32_t*, uint32_t*, uint32_t*, uint64_t*); \
    template cudaError_t range_fill<K>(Ctx&, const uint32_t*, uint64_t, const uint8_t*, const uint32_t*,       \
                                       const uint32_t*, const uint32_t*, const uint64_t*, K*, K*, bool);

FLIX_READ_INST(uint32_t)
FLIX_READ_INST(uint64_t)

}  // namespace flix
