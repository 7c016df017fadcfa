// Internal definitions shared by the FliX CUDA sources (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <initializer_list>
#include <string>
#include <utility>
#include <vector>

#include "flix.h"

namespace flix {

constexpr uint32_t NIL = 0xFFFFFFFFu;

// Net effect of one key's update run within a batch (composition of its inserts and deletes in
// submission order): insert-if-absent, delete, or delete-then-insert ("upsert": present afterwards
// with the new value whatever the prior state).
enum Eff : uint32_t { EFF_NONE = 0, EFF_INS = 1, EFF_DEL = 2, EFF_UPS = 3 };

// Device error word bits (checked at the next synchronising call).
enum : uint32_t { ERR_CHAIN = 1u, ERR_BADKEY = 2u, ERR_RANGE = 4u, ERR_STEPS = 8u, ERR_SPIN = 16u, ERR_SORT = 32u, ERR_TIMEOUT = 64u };

template <class K>
__host__ __device__ constexpr K key_max() { return static_cast<K>(~K(0)); }

// Outside stream capture every kernel of the library is launched with programmatic stream
// serialization, so that it can be scheduled while the kernel before it on the stream is still
// finishing (the gap between two dependent kernels drops from about 4 us to about 1.4 us on this
// GPU).  Each kernel starts with this: it first waits until the kernel before it has completed and
// its writes are visible, and only then lets the next kernel launch.  So at most one kernel is
// resident and waiting behind the one that runs, every kernel it waits on has completed the wait
// itself, and no kernel sees a partial result of an earlier one.
__device__ __forceinline__ void grid_dep_enter()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Device view of the data layer (Sec. 3.2).  Node pool in structure-of-arrays form: node n's keys
// are keys[n*NS .. n*NS+size[n]) in ascending order, values alongside; bound[n] is its maxKey and
// next[n] its node-link.  mkba[b] is bucket b's maxBucket and head[b] its first node.
template <class K>
struct DevIdx {
    K* keys;
    K* vals;
    uint32_t* size;
    K* bound;
    uint32_t* next;
    K* mkba;
    uint32_t* head;
    uint32_t NS;
    uint32_t nb;
    uint32_t cap;   // node-pool capacity: no chain walk takes more steps
    uint32_t* err;
    uint32_t lane_path;   // nonzero: a light one-node bucket's updates are applied by one thread
};

enum KernelId {
    K_READBACK, K_SORT_HIST, K_SORT_UP, K_SORT_SCAN, K_SORT_DOWN, K_SORT_ONESWEEP, K_SORT_PLAN, K_SORT_IDLE, K_SORT_FINISH,
    K_SCAN_PART, K_SCAN_TOP, K_SCAN_APPLY,
    K_PARTITION, K_READ_POINT, K_UNSORT, K_RANGE_COUNT, K_RANGE_FILL,
    K_VALIDATE, K_FOLD_FLAGS, K_FOLD_INIT, K_FOLD_DEL, K_FOLD_INS, K_FOLD_EMIT, K_FOLD_WRITE,
    K_UPD_COUNT, K_ALLOC_COPY, K_UPD_APPLY, K_ADMIT,
    K_LIVE_COUNT, K_GATHER, K_CUT_KEYS, K_CUT_META, K_DEDUPE, K_STATS, K_FILL, K_SPLIT, K_MERGE, K_HEAVY,
    K_QUEUE, K_NUM
};

// Device allocations of a handle: the caller's allocator (flix_config) or cudaMalloc/cudaFree.
struct DevAlloc {
    void* (*alloc)(size_t, void*) = nullptr;
    void (*free)(void*, void*) = nullptr;
    void* ctx = nullptr;
};
cudaError_t dev_malloc(const DevAlloc& da, void** p, size_t bytes);
void dev_free(const DevAlloc& da, void* p);   // synchronises the device first

// Bump allocator over one device buffer, reset at the start of every call.
struct Arena {
    DevAlloc da;
    char* base = nullptr;
    size_t cap = 0;
    size_t used = 0;
    cudaError_t ensure(size_t bytes);
    void reset() { used = 0; }
    template <class T>
    T* take(size_t count)
    {
        size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
        if (used + bytes > cap) return nullptr;
        T* p = reinterpret_cast<T*>(base + used);
        used += bytes;
        return p;
    }
    void release();
};

struct ProfRec {
    int kid;
    double bytes;   // algorithmic bytes the launch moves, where the host knows them (else 0)
    cudaEvent_t a, b;
};

// Device-side plan of one batch sort (written by the plan kernel, read by the passes and the
// finish kernels): passes shift[0..npass) in LSD order; finish = 1 when groups of keys equal under
// pmask still need sorting; nbig and cursor count and hand out the long groups.
struct SortPlan {
    uint32_t npass;
    uint32_t finish;
    uint32_t shift[8];
    unsigned long long pmask;
    unsigned long long nbig;
    unsigned long long cursor;
};

// Device-resident allocator and admission state of a handle.  free_top is authoritative on the
// device so that update batches can be admitted without a host round trip: the admit kernel compares
// the batch's node demand with free_top, and the alloc, apply and commit kernels act only if it
// admitted the batch.
struct DevState {
    unsigned long long free_top;   // number of ids on the free stack
    unsigned long long admitted;   // 1 while an admitted batch is being applied
    unsigned long long from;       // first popped stack slot (= free_top - need)
    unsigned long long next_top;   // free_top after the batch (from + freed)
    unsigned long long need;       // nodes the batch allocates
    unsigned long long freed;      // nodes the batch frees
    unsigned long long applied;    // 1 if the last committed batch was admitted
};

// Status bits an asynchronous batch reports (flix_apply_async).
enum : uint64_t { ST_BADKEY = 1, ST_NODES = 2, ST_RANGE = 4 };

}  // namespace flix

struct flix_index {
    flix_config cfg;
    int kw;             // key width in bits (32 or 64)
    size_t ks;          // key size in bytes
    uint32_t NS;        // node capacity
    uint32_t p;         // keys per node after a build or restructure
    uint64_t cap = 0;   // node-pool capacity
    uint64_t nb = 0;    // buckets
    uint64_t free_top = 0;  // number of ids on the free stack (host mirror of the device state)
    int device = 0;
    int nsm = 148;      // SMs of the device
    flix::DevAlloc da;  // device allocator

    // node pool and buckets (device)
    void* keys = nullptr;
    void* vals = nullptr;
    uint32_t* size = nullptr;
    void* bound = nullptr;
    uint32_t* next = nullptr;
    uint32_t* tnode = nullptr;     // per-node scratch: merged size from the update count pass
    void* mkba = nullptr;
    uint32_t* head = nullptr;
    uint32_t* free_ids = nullptr;  // free stack: ids [0, free_top) are free nodes
    void* keys2 = nullptr;         // second key/value node arrays of the one-pass restructure
    void* vals2 = nullptr;
    uint64_t cap2 = 0;             // their capacity in nodes (0: not allocated)
    void* mkba2 = nullptr;         // second MKBA and bucket heads of the elastic split
    uint32_t* head2 = nullptr;
    uint64_t capb2 = 0;            // their capacity in buckets (0: not allocated)
    uint32_t* err = nullptr;       // device error word
    flix::DevState* dstate = nullptr;

    flix::Arena arena;
    uint64_t* hpin = nullptr;      // small mapped pinned host buffer for read-backs (64 words)
    uint64_t* hpin_dev = nullptr;  // its device address

    bool prof_on = false;
    std::vector<flix::ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    uint64_t launches = 0;
    std::string last_error;

    void* qstage = nullptr;        // pinned staging of a persistent queue's batch descriptors
    size_t qstage_bytes = 0;
    cudaEvent_t qstage_ev = nullptr;   // recorded after the staging copy was issued

    // a mixed batch's update preparation runs on side_st beside its reads (fork and join events)
    cudaStream_t side_st = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr;
};

namespace flix {

extern const char* kKernelNames[K_NUM];

// Per-call launch context.
struct Ctx {
    flix_index* h;
    cudaStream_t st;
};

cudaEvent_t prof_event(flix_index* h);

// Launch with profiling hooks; `bytes` = the launch's algorithmic bytes for the per-kernel roofline.
template <class Kern, class... Args>
cudaError_t launch_b(Ctx& c, int kid, double bytes, dim3 grid, dim3 block, size_t smem, Kern kern, Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    cudaEvent_t a = nullptr, b = nullptr;
    if (c.h->prof_on) {
        a = prof_event(c.h);
        b = prof_event(c.h);
        cudaEventRecord(a, c.st);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.st;
    // kernels captured into a graph keep full dependencies: a replay submits every node at once
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(c.st, &cap);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = cap == cudaStreamCaptureStatusNone ? 1 : 0;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (c.h->prof_on) {
        cudaEventRecord(b, c.st);
        c.h->prof.push_back(ProfRec{kid, bytes, a, b});
    }
    c.h->launches++;
    return e;
}

// A cooperative launch (every block resident at once, for kernels with a grid barrier); it waits
// for the previous launch on the stream to complete, like a launch without dependent-launch overlap.
template <class Kern, class... Args>
cudaError_t launch_coop(Ctx& c, int kid, double bytes, dim3 grid, dim3 block, size_t smem, Kern kern, Args... args)
{
    if (grid.x == 0 || grid.y == 0 || grid.z == 0) return cudaSuccess;
    cudaEvent_t a = nullptr, b = nullptr;
    if (c.h->prof_on) {
        a = prof_event(c.h);
        b = prof_event(c.h);
        cudaEventRecord(a, c.st);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, args...);
    if (c.h->prof_on) {
        cudaEventRecord(b, c.st);
        c.h->prof.push_back(ProfRec{kid, bytes, a, b});
    }
    c.h->launches++;
    return e;
}

template <class Kern, class... Args>
cudaError_t launch(Ctx& c, int kid, dim3 grid, dim3 block, size_t smem, Kern kern, Args... args)
{
    return launch_b(c, kid, 0.0, grid, block, smem, kern, args...);
}

inline uint32_t div_up(uint64_t a, uint64_t b) { return static_cast<uint32_t>((a + b - 1) / b); }

template <class K>
DevIdx<K> dev_view(flix_index* h)
{
    DevIdx<K> d;
    d.keys = static_cast<K*>(h->keys);
    d.vals = static_cast<K*>(h->vals);
    d.size = h->size;
    d.bound = static_cast<K*>(h->bound);
    d.next = h->next;
    d.mkba = static_cast<K*>(h->mkba);
    d.head = h->head;
    d.NS = h->NS;
    d.nb = static_cast<uint32_t>(h->nb);
    d.cap = static_cast<uint32_t>(h->cap);
    d.err = h->err;
    d.lane_path = h->cfg.bucket_threads != 32;
    return d;
}

// ---- node search helpers (device) ------------------------------------------------------------
//
// NC: node data is read through the non-coherent (read-only) cache; a kernel that itself changes
// nodes between its reads (the persistent queue kernel) passes false and reads coherently.

template <bool NC, class T>
__device__ __forceinline__ T ld_node(const T* p)
{
    if (NC) return __ldg(p);
    return *p;
}

// First position in nk[0..sz) whose key is >= q.
template <class K, bool NC = true>
__device__ __forceinline__ uint32_t node_lower_bound(const K* __restrict__ nk, uint32_t sz, K q)
{
    uint32_t base = 0, len = sz;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (ld_node<NC>(nk + base + half) < q) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// First position in nk[from..sz) whose key is > q.
template <class K, bool NC = true>
__device__ __forceinline__ uint32_t node_upper_bound(const K* __restrict__ nk, uint32_t from, uint32_t sz, K q)
{
    uint32_t base = from, len = sz - from;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (!(q < ld_node<NC>(nk + base + half))) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// From bucket b's first node, walk node-links to the first node whose maxKey >= q (Sec. 4.1);
// prev = the node walked past last (NIL when the walk ends at the first node).  Node b is bucket
// b's first node after every bulk load and restructure (until an elastic split renumbers the
// buckets or the node leaves its chain), so its metadata is read beside the bucket's head (b < nb
// <= cap) and kept when the head confirms it: one dependent load less on the usual walk.
template <class K, bool NC = true>
__device__ __forceinline__ bool find_node(const DevIdx<K>& ix, uint32_t b, K q, uint32_t& node, uint32_t& sz, K& bd,
                                          uint32_t& nx, uint32_t& prev)
{
    prev = NIL;
    node = ld_node<NC>(ix.head + b);
    sz = ld_node<NC>(ix.size + b);
    bd = ld_node<NC>(ix.bound + b);
    nx = ld_node<NC>(ix.next + b);
    if (node != b) {
        sz = ld_node<NC>(ix.size + node);
        bd = ld_node<NC>(ix.bound + node);
        nx = ld_node<NC>(ix.next + node);
    }
    uint32_t steps = 0;
    while (q > bd) {
        if (nx == NIL || ++steps > ix.cap) { atomicOr(ix.err, ERR_CHAIN); return false; }
        prev = node;
        node = nx;
        sz = ld_node<NC>(ix.size + node);
        bd = ld_node<NC>(ix.bound + node);
        nx = ld_node<NC>(ix.next + node);
    }
    return true;
}

// Result of one point read once its node is known (Sec. 4.1 walk done): pos is the first of the
// node's sz keys >= q (LOOKUP, SUCC) or > q (PRED), and kpos the key at pos (LOOKUP, SUCC, when
// pos < sz) or at pos - 1 (PRED, when pos > 0).  A successor past the node continues with the
// first key of the next non-empty node in chain order, into the following buckets (Sec. 6.5: the
// smallest key >= q); a predecessor before the node's first key takes the last key of the node
// walked past, else of the nearest earlier bucket whose chain holds a key.
template <class K, bool NC = true>
__device__ __forceinline__ void point_result(const DevIdx<K>& ix, int op, K q, uint32_t b, uint32_t node, uint32_t sz,
                                             uint32_t nx, uint32_t prev, uint32_t pos, K kpos, K& rk, K& rv,
                                             uint8_t& f)
{
    const uint32_t NS = ix.NS;
    if (op == FLIX_OP_PRED) {
        // chain nodes other than a bucket's only node are never empty
        uint32_t pn = NIL, pp = 0;
        if (pos > 0) {
            rk = kpos;
            rv = ix.vals[(uint64_t)node * NS + pos - 1];
            f = 1;
            return;
        }
        if (prev != NIL && ix.size[prev] > 0) {
            pn = prev;
            pp = ix.size[prev] - 1;
        } else {
            uint64_t guard = 0;
            const uint64_t lim = (uint64_t)ix.cap + ix.nb + 1;
            for (int64_t bb = (int64_t)b - 1; bb >= 0 && pn == NIL && guard < lim; bb--) {
                uint32_t x = ix.head[bb];
                uint32_t last = x;
                while (x != NIL && guard++ < lim) {
                    last = x;
                    x = ix.next[x];
                }
                const uint32_t ls = ix.size[last];
                if (ls > 0) {
                    pn = last;
                    pp = ls - 1;
                }
            }
        }
        if (pn != NIL) {
            rk = ix.keys[(uint64_t)pn * NS + pp];
            rv = ix.vals[(uint64_t)pn * NS + pp];
            f = 1;
        }
        return;
    }
    if (op == FLIX_OP_LOOKUP) {
        if (pos < sz && kpos == q) {
            rk = q;
            rv = ld_node<NC>(ix.vals + (uint64_t)node * NS + pos);
            f = 1;
        }
        return;
    }
    if (pos < sz) {
        rk = kpos;
        rv = ld_node<NC>(ix.vals + (uint64_t)node * NS + pos);
        f = 1;
        return;
    }
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

// Range count by one warp (all 32 lanes call it with the same arguments): the stored keys <= hi
// from slot pos of `node` in bucket bb onwards.  Like the fill, the warp takes the next nodes in
// chain order 32 at a time (lane 0 the current node, lane l > 0 the first node of bucket bb + l,
// a batch ending at the first node whose chain continues); a node whose maxKey is <= hi counts
// its size from its position; the first node whose maxKey is > hi counts its keys <= hi by a binary
// search and ends the count.
template <class K, bool NC = true>
__device__ __forceinline__ uint64_t range_count_warp(const DevIdx<K>& ix, uint64_t bb, uint32_t node, uint32_t pos, K hi)
{
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t NS = ix.NS;
    const uint32_t lane = threadIdx.x & 31;
    uint64_t c = 0;
    for (uint64_t guard = 0, lim = (uint64_t)ix.cap + ix.nb + 1; guard < lim; guard++) {
        uint32_t n_l = NIL, p_l = 0, sz_l = 0, nx_l = NIL;
        K bd_l = K(0);
        if (lane == 0) {
            n_l = node;
            p_l = pos;
        } else if (bb + lane < ix.nb) {
            n_l = ld_node<NC>(ix.head + bb + lane);
        }
        if (n_l != NIL) {
            sz_l = ld_node<NC>(ix.size + n_l);
            nx_l = ld_node<NC>(ix.next + n_l);
            bd_l = ld_node<NC>(ix.bound + n_l);
        }
        const uint32_t cont = __ballot_sync(FULL, n_l != NIL && nx_l != NIL);
        const uint32_t past = __ballot_sync(FULL, n_l != NIL && bd_l > hi);
        const uint32_t none = __ballot_sync(FULL, n_l == NIL);
        // the batch: lanes up to the first that continues its chain, ends the count or has no node
        const uint32_t stop = cont | past | none;
        const uint32_t last = stop ? __ffs(stop) - 1 : 31;
        uint32_t mine = 0;
        if (lane <= last && n_l != NIL && sz_l > p_l) {
            if (bd_l <= hi) mine = sz_l - p_l;
            else mine = node_upper_bound<K, NC>(ix.keys + (uint64_t)n_l * NS, p_l, sz_l, hi) - p_l;
        }
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) mine += __shfl_xor_sync(FULL, mine, d);
        c += mine;
        if ((past | none) & (0xFFFFFFFFu >> (31 - last))) break;   // a node past hi, or no node left
        // continue after the batch's last node: along its link, or at the next bucket's first node
        const uint32_t lnx = __shfl_sync(FULL, nx_l, last);
        if (lnx != NIL) {
            bb += last;
            node = lnx;
        } else {
            bb += last + 1;
            if (bb >= ix.nb) break;
            node = ld_node<NC>(ix.head + bb);
        }
        pos = 0;
    }
    return c;
}

// Range fill by one warp (all 32 lanes call it with the same arguments): c pairs starting at slot
// pos of `node` in bucket bb, written to rkeys/rvals[o..o+c) in key order.  The warp takes the
// next nodes in chain order 32 at a time: lane 0 the current node (from the current position), lane
// l > 0 the first node of bucket bb + l; their sizes and node-links load in parallel, and a batch
// ends at the first node whose chain continues (the walk goes on from its link).  A warp scan of
// the nodes' available counts gives each node's output offset, and the pairs are copied with one
// independent load per pair (each lane finds its pair's node by a shuffle search over the offsets).
template <class K, bool NC = true, uint32_t R = 1>
__device__ __forceinline__ void range_fill_warp(const DevIdx<K>& ix, uint64_t bb, uint32_t node, uint32_t pos,
                                                uint64_t o, uint64_t c, K* __restrict__ rkeys, K* __restrict__ rvals)
{
    constexpr uint32_t FULL = 0xFFFFFFFFu;
    const uint32_t NS = ix.NS;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t guard = 0, lim = (uint64_t)ix.cap + ix.nb + 1; guard < lim && c > 0; guard++) {
        // lane 0: the current node; lane l > 0: the first node of bucket bb + l
        uint32_t n_l = NIL, p_l = 0, sz_l = 0, nx_l = NIL;
        bool have = false;
        if (lane == 0) {
            n_l = node;
            p_l = pos;
        } else if (bb + lane < ix.nb) {
            // node b is usually bucket b's first node (see find_node): its metadata is read beside
            // the head and kept when the head confirms it
            const uint32_t b_l = (uint32_t)(bb + lane);
            n_l = ld_node<NC>(ix.head + b_l);
            sz_l = ld_node<NC>(ix.size + b_l);
            nx_l = ld_node<NC>(ix.next + b_l);
            have = n_l == b_l;
        }
        if (n_l != NIL && !have) {
            sz_l = ld_node<NC>(ix.size + n_l);
            nx_l = ld_node<NC>(ix.next + n_l);
        } else if (n_l == NIL) {
            sz_l = 0;
            nx_l = NIL;
        }
        // the batch ends at the first node whose chain continues
        const uint32_t cont = __ballot_sync(FULL, nx_l != NIL);
        const uint32_t last = cont ? __ffs(cont) - 1 : 31;
        const uint32_t avail = (lane <= last && sz_l > p_l) ? sz_l - p_l : 0u;
        uint32_t incl = avail;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, incl, d);
            if (lane >= (uint32_t)d) incl += y;
        }
        const uint32_t total = __shfl_sync(FULL, incl, 31);
        const uint32_t take = (uint64_t)total < c ? total : (uint32_t)c;
        // R pairs per lane in flight: every load of a round is issued before its stores (a warp on
        // its own, as in the persistent queue kernel, wants several; a full grid of warps, one)
        for (uint32_t t0 = 0; t0 < take; t0 += 32 * R) {
            K kr[R], vr[R];
#pragma unroll
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t t = t0 + r * 32 + lane;
                // the pair's node: the first lane whose inclusive count exceeds t
                uint32_t src = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1) {
                    const uint32_t probe = src + step - 1;
                    if (__shfl_sync(FULL, incl, probe) <= t) src += step;
                }
                const uint32_t base = __shfl_sync(FULL, incl - avail, src);
                const uint32_t sn = __shfl_sync(FULL, n_l, src);
                const uint32_t sp = __shfl_sync(FULL, p_l, src);
                if (t < take) {
                    const uint64_t slot = (uint64_t)sn * NS + sp + (t - base);
                    kr[r] = ix.keys[slot];
                    vr[r] = ix.vals[slot];
                }
            }
#pragma unroll
            for (uint32_t r = 0; r < R; r++) {
                const uint32_t t = t0 + r * 32 + lane;
                if (t < take) {
                    rkeys[o + t] = kr[r];
                    rvals[o + t] = vr[r];
                }
            }
        }
        o += take;
        c -= take;
        if (c == 0) break;
        // continue after the batch's last node: along its link, or at the next bucket's first node
        const uint32_t lnx = __shfl_sync(FULL, nx_l, last);
        if (lnx != NIL) {
            bb += last;
            node = lnx;
        } else {
            bb += last + 1;
            if (bb >= ix.nb) {
                if (lane == 0) atomicOr(ix.err, ERR_RANGE);
                return;
            }
            node = ix.head[bb];
        }
        pos = 0;
    }
}

// Read up to 8 device values (4 or 8 bytes each) into h->hpin[word0 + i] and synchronise the stream
// (flix_capi.cu); returns a FLIX_ status.
int readback_at(flix_index* h, cudaStream_t st, uint32_t word0,
                std::initializer_list<std::pair<const void*, size_t>> items);

// Every kernel of the library, loaded at handle creation (flix_capi.cu: preload_kernels).  Under
// lazy module loading a kernel is otherwise loaded at its first launch, and a first launch inside
// a CUDA graph replay was measured at ~0.7 s.
void preload_kernels();
void preload_sort_kernels();
void preload_read_kernels();
void preload_update_kernels();
void preload_build_kernels();
void preload_persist_kernels();

// The persistent queue of small mixed batches (flix_persist.cu).
template <class K>
int apply_queue(flix_index* h, const flix_batch* hb, uint32_t count, uint32_t wait_us, uint64_t* d_flags_or,
                cudaStream_t st);

// Device fills and small copies as kernels on the call's stream (flix_capi.cu): a cudaMemsetAsync
// or cudaMemcpyAsync may be carried out by a copy engine, where it would wait behind bulk transfers
// that other streams have queued.
cudaError_t fill_bytes(Ctx& c, void* dst, uint8_t value, size_t bytes);
cudaError_t copy_words(Ctx& c, void* dst, const void* src, uint32_t words);

// ---- sort and scan primitives (flix_sort.cu) -------------------------------------------------

// Scratch bytes sort_pairs needs for n items.
template <class K>
size_t sort_scratch_bytes(uint64_t n);

// Stable sort of the keys kin[0..n) with their positions: kout ascending, vout[i] = input position
// of kout[i] (equal keys keep input order).  vin must be nullptr (the payload is the position) and
// n < 2^32 - 1.  Scratch from the arena.
template <class K>
cudaError_t sort_pairs(Ctx& c, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, uint64_t n);

// Exclusive prefix sum out[0..n] of in[0..n) (out[n] = total).  Tin: uint32_t or uint64_t.
template <class Tin, class Tout>
cudaError_t scan_exclusive(Ctx& c, const Tin* in, Tout* out, uint64_t n);
template <class Tout>
size_t scan_scratch_bytes(uint64_t n);

// ---- read path (flix_read.cu) ----------------------------------------------------------------

// off[0..nb]: off[i] = number of sorted keys <= mkba[i-1] (off[0] = 0), by a merge-path co-rank
// of the sorted MKBA with the sorted batch.  m_dev (optional) holds the batch length on the device
// (then m is an upper bound).
// bk (optional): bk[j] = bucket of sorted key j.  off (optional) as above.
// Scratch bytes partition takes from the arena.
size_t partition_scratch_bytes(uint64_t nb, uint64_t m);

template <class K>
cudaError_t partition(Ctx& c, const K* mkba, uint64_t nb, const K* skeys, uint64_t m,
                      const uint32_t* m_dev, uint32_t* off, uint32_t* bk);

// Scratch bytes read_point may take from the arena (it scatters directly when they are missing).
template <class K>
size_t read_point_scratch_bytes(uint64_t m);

template <class K>
cudaError_t read_point(Ctx& c, int mode, const K* skeys, const uint32_t* sidx, uint64_t m,
                       const uint32_t* bk, const uint8_t* ops, K* keys_out, K* vals_out,
                       uint8_t* found_out);

// Range count: per range op its start (bucket, node, position) in sorted order and its pair
// count cnt[idx] in submission order (0 for non-range ops when ops != nullptr).
template <class K>
cudaError_t range_count(Ctx& c, const K* skeys, const uint32_t* sidx, uint64_t m, const uint32_t* bk,
                        const uint8_t* ops, const K* hi, uint32_t* start_bucket, uint32_t* start_node,
                        uint32_t* start_pos, uint64_t* cnt);

// gated: write only if the device admission state admitted the batch
template <class K>
cudaError_t range_fill(Ctx& c, const uint32_t* sidx, uint64_t m, const uint8_t* ops,
                       const uint32_t* start_bucket, const uint32_t* start_node, const uint32_t* start_pos,
                       const uint64_t* off, K* rkeys, K* rvals, bool gated);

// ---- update path (flix_update.cu) ------------------------------------------------------------

template <class K>
cudaError_t validate_inserts(Ctx& c, const uint8_t* ops, const K* keys, uint64_t n, uint32_t* flag);

// Reduce the sorted batch to one net update per key: ukey/uop/uval[0..U), U in *u_dev.
// hom_op: FLIX_OP_INSERT or FLIX_OP_DELETE for homogeneous batches, 0 for mixed (ops used).
template <class K>
cudaError_t fold_updates(Ctx& c, const K* skeys, const uint32_t* sidx, uint64_t m, const uint8_t* ops,
                         int hom_op, const K* aux, K* ukey, uint32_t* uop, K* uval, uint32_t* u_dev);

// Nodes that receive more than 2048 updates of a batch ("heavy"): listed by the count pass,
// skipped by update_apply's key placement, merged by update_heavy (a block per node).
struct HeavyList {
    void* list = nullptr;
    uint32_t* n = nullptr;   // device count
    uint32_t cap = 0;
    void* snap_k = nullptr;  // snapshots of the heavy nodes' keys and values (cap x NS each)
    void* snap_v = nullptr;
    uint32_t* nchunks = nullptr;     // device count of their chunks; nchunks[1], nchunks[2]: block
                                     // counters of the find and count kernels (zero between batches)
    uint32_t* chunk_add = nullptr;   // absent keys each chunk inserts
    uint32_t* chunk_pre = nullptr;   // their exclusive prefix
    uint32_t chunk_cap = 0;
    uint64_t batch = 0;              // updates of the batch (none is heavy unless > HEAVY_U)
};
template <class K>
cudaError_t update_count(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval, const uint32_t* uoff,
                         uint64_t* nf, uint8_t* allgone, const HeavyList& hl);

template <class K>
cudaError_t update_apply(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval,
                         const uint32_t* uoff, const uint64_t* nf_off, const uint8_t* allgone,
                         const uint32_t* alloc_ids);

size_t heavy_scratch_bytes(uint64_t n);
HeavyList heavy_list(Ctx& c, uint64_t n);   // from the arena, for a batch of n updates
template <class K>
cudaError_t update_heavy(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval, const uint64_t* nf_off,
                         const uint32_t* alloc_ids, const HeavyList& hl);

// Device admission of an update batch: node demand nf_total (need | freed << 32) against free_top,
// the reserved-key flag, and the range total against range_cap.  status (optional, 4 words):
// flags (ST_*), range total, need, free_top before the batch.
cudaError_t admit(Ctx& c, const uint64_t* nf_total, const uint32_t* badkey, const uint64_t* range_total,
                  uint64_t range_cap, uint64_t* status);
cudaError_t commit(Ctx& c);
cudaError_t set_free_top(Ctx& c, uint64_t value);

// Copy the admitted batch's popped node ids (at most cap_out) out of the free stack.
cudaError_t alloc_copy(Ctx& c, const uint32_t* free_ids, uint32_t* out, uint64_t cap_out);

// ---- build / restructure / export (flix_build.cu) --------------------------------------------

// Live pairs per bucket by walking each chain up to 64 nodes; *long_flag = 1 if a chain is longer
// (cnt is then incomplete and the node-order functions below must be used instead).
template <class K>
cudaError_t live_count(Ctx& c, uint64_t* cnt, uint32_t* long_flag);

// The nodes in use in chain order, found without walking chains: order[0..m) node ids sorted by
// maxKey (bound[] the sorted maxKeys), noff[0..m] the exclusive prefix of their sizes (noff[m] =
// live pairs).  Synchronises once (to read m).  Scratch from the arena.
template <class K>
struct NodeOrder {
    uint64_t m = 0;
    uint32_t* order = nullptr;
    uint64_t* noff = nullptr;
    K* bound = nullptr;
};
template <class K>
size_t node_order_scratch_bytes(uint64_t cap);
template <class K>
int node_order(Ctx& c, NodeOrder<K>& no);
// The live pairs in key order, by node (flat, or straight into the second node arrays).
template <class K>
cudaError_t gather_nodes(Ctx& c, const NodeOrder<K>& no, K* out_k, K* out_v);
template <class K>
cudaError_t gather_nodes_cut(Ctx& c, const NodeOrder<K>& no, uint64_t nb_new, K* k2, K* v2);
// Longest chain (in nodes), from the buckets of the nodes in chain order.
template <class K>
cudaError_t chain_max_by_nodes(Ctx& c, const NodeOrder<K>& no, uint64_t* out_max);

template <class K>
cudaError_t gather_live(Ctx& c, const uint64_t* goff, K* out_k, K* out_v);

// Cut n sorted distinct pairs into single-node buckets of p keys (Sec. 3.2); resets the free list.
template <class K>
cudaError_t cut_buckets(Ctx& c, const K* sk, const K* sv, uint64_t n, uint64_t nb_new);

// One-pass restructure: the live pairs (goff = global rank of every bucket's first pair) go to
// their canonical node and slot in the second arrays k2/v2; maxKey and maxBucket of every group
// but the last are set on the way.  Then cut_buckets(c, nullptr, nullptr, n, nb_new) writes the
// rest of the metadata once k2/v2 have become the pool's arrays.
template <class K>
cudaError_t gather_cut(Ctx& c, const uint64_t* goff, uint64_t n, uint64_t nb_new, K* k2, K* v2);

template <class K>
cudaError_t dedupe_sorted(Ctx& c, const K* skeys, const uint32_t* sidx, const K* vals, uint64_t n,
                          K* ok, K* ov, uint32_t* n_dev);

template <class K>
cudaError_t stats_kernel(Ctx& c, uint64_t* out3);

// Elastic bucket split (Sec. 3.4).  split_count: cnt[b] = the new buckets bucket b becomes (its
// chain length when that exceeds max_chain and the bucket is selected, else 1); buckets are
// selected by a non-empty update range uoff[b] < uoff[b+1], or all when uoff is null.
// split_write: with boff the exclusive scan of cnt, writes the new MKBA and bucket heads (a split
// chain's nodes become single-node buckets with their maxKey as maxBucket).
template <class K>
cudaError_t split_count(Ctx& c, uint32_t max_chain, const uint32_t* uoff, uint64_t* cnt);
template <class K>
cudaError_t split_write(Ctx& c, const uint64_t* cnt, const uint64_t* boff, K* mkba2, uint32_t* head2);
// Underfull-neighbour merge in the selected buckets (uoff as above); freed nodes go on the free
// stack; *freed (may be null) counts them.  gated: only if the batch just run was admitted.
template <class K>
cudaError_t merge_underfull(Ctx& c, const uint32_t* uoff, int gated, unsigned long long* freed);

}  // namespace flix
