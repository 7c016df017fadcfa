// Update path: validation, per-key net effect of the sorted update list, node-demand count, free
// list allocation and the in-place apply (insert with split, Sec. 4.3.2; delete with compaction
// and node reclamation, Sec. 4.4).
//
// A warp owns 32 consecutive buckets: its lanes load every bucket's sublist bounds and first node
// in parallel, then the warp works through the buckets that have updates, walking each chain
// (Sec. 4.1: an update goes to the first node with key <= maxKey).  For each node that receives updates the warp lifts the node's keys and values
// into shared memory (the paper lifts them into the tile's registers, Sec. 4.3.2), marks the
// deleted slots (Tab. 3's mask), and computes every surviving or inserted key's position in the
// merged run: a node key's position is its slot minus the deletions before it plus the inserted
// keys before it; an inserted key's position is the count of surviving node keys below it plus the
// inserted keys before it.  The merged run of t keys is laid out canonically: one node if
// t <= NS, else floor(t / (NS/2)) nodes of NS/2 keys with the remainder in the last; the node keeps
// the first piece, new nodes (popped from the free stack in bucket order) take the others, every
// piece but the last takes its largest key as maxKey and the last keeps the node's maxKey.  An
// emptied node leaves the chain and its id is pushed on the free stack, unless the bucket's whole
// chain emptied, in which case its first node stays as an empty node.
//
// A count pass computes each node's merged size and each bucket's node demand before anything is
// written, so that a batch the pool cannot hold is rejected with the structure unchanged.
#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int UP_THREADS = 128;
constexpr int UP_WARPS = UP_THREADS / 32;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <class K>
__global__ void k_validate(const uint8_t* __restrict__ ops, const K* __restrict__ keys, uint64_t n, uint32_t* flag)
{
    grid_dep_enter();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if ((ops == nullptr || ops[i] == FLIX_OP_INSERT) && keys[i] == key_max<K>()) atomicOr(flag, ERR_BADKEY);
}

// head[j] = 1 where a new key starts in the sorted batch
template <class K>
__global__ void k_fold_flags(const K* __restrict__ skeys, uint64_t m, uint32_t* __restrict__ head)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    head[j] = (j == 0 || skeys[j] != skeys[j - 1]) ? 1u : 0u;
}

__global__ void k_fold_init(uint64_t m, uint32_t* __restrict__ lastdel, uint32_t* __restrict__ firstins,
                            uint32_t* __restrict__ emit)
{
    grid_dep_enter();
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m) return;
    lastdel[r] = 0;
    firstins[r] = NIL;
    emit[r] = 0;
}

// run id of sorted position j = inclusive count of heads up to j, minus one
__device__ __forceinline__ uint32_t run_id(const uint32_t* __restrict__ head, const uint32_t* __restrict__ hex, uint64_t j)
{
    return hex[j] + head[j] - 1;
}

// last delete of each run (position + 1)
__global__ void k_fold_del(const uint32_t* __restrict__ sidx, uint64_t m, const uint8_t* __restrict__ ops,
                           const uint32_t* __restrict__ head, const uint32_t* __restrict__ hex,
                           uint32_t* __restrict__ lastdel)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (ops[sidx[j]] == FLIX_OP_DELETE) atomicMax(&lastdel[run_id(head, hex, j)], (uint32_t)(j + 1));
}

// first insert after the run's last delete
__global__ void k_fold_ins(const uint32_t* __restrict__ sidx, uint64_t m, const uint8_t* __restrict__ ops,
                           const uint32_t* __restrict__ head, const uint32_t* __restrict__ hex,
                           const uint32_t* __restrict__ lastdel, uint32_t* __restrict__ firstins)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m) return;
    if (ops[sidx[j]] != FLIX_OP_INSERT) return;
    const uint32_t r = run_id(head, hex, j);
    if ((uint32_t)(j + 1) > lastdel[r]) atomicMin(&firstins[r], (uint32_t)j);
}

// per run: net effect, emit flag and head position
__global__ void k_fold_emit(uint64_t m, const uint32_t* __restrict__ head, const uint32_t* __restrict__ hex,
                            const uint32_t* __restrict__ lastdel, const uint32_t* __restrict__ firstins,
                            uint32_t* __restrict__ emit, uint32_t* __restrict__ eff, uint32_t* __restrict__ hpos)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m || !head[j]) return;
    const uint32_t r = hex[j];
    const uint32_t ld = lastdel[r], fi = firstins[r];
    uint32_t e;
    if (ld == 0) e = fi == NIL ? EFF_NONE : EFF_INS;
    else e = fi == NIL ? EFF_DEL : EFF_UPS;
    emit[r] = e != EFF_NONE;
    eff[r] = e;
    hpos[r] = (uint32_t)j;
}

template <class K>
__global__ void k_fold_write_mixed(uint64_t m, const K* __restrict__ skeys, const uint32_t* __restrict__ sidx,
                                   const K* __restrict__ aux, const uint32_t* __restrict__ emit,
                                   const uint32_t* __restrict__ epos, const uint32_t* __restrict__ eff,
                                   const uint32_t* __restrict__ hpos, const uint32_t* __restrict__ firstins,
                                   K* __restrict__ ukey, uint32_t* __restrict__ uop, K* __restrict__ uval)
{
    grid_dep_enter();
    const uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= m || !emit[r]) return;
    const uint32_t p = epos[r];
    ukey[p] = skeys[hpos[r]];
    uop[p] = eff[r];
    const uint32_t fi = firstins[r];
    uval[p] = fi != NIL ? aux[sidx[fi]] : K(0);
}

// homogeneous batch: every head emits; a stable sort puts the first submitted op at the head
template <class K>
__global__ void k_fold_write_hom(uint64_t m, uint32_t eff, const K* __restrict__ skeys,
                                 const uint32_t* __restrict__ sidx, const K* __restrict__ aux,
                                 const uint32_t* __restrict__ head, const uint32_t* __restrict__ hex,
                                 K* __restrict__ ukey, uint32_t* __restrict__ uop, K* __restrict__ uval)
{
    grid_dep_enter();
    const uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m || !head[j]) return;
    const uint32_t p = hex[j];
    ukey[p] = skeys[j];
    uop[p] = eff;
    uval[p] = (eff == EFF_INS && aux) ? aux[sidx[j]] : K(0);
}

__device__ __forceinline__ uint32_t pieces_of(uint32_t t, uint32_t NS)
{
    if (t == 0) return 0;
    if (t <= NS) return 1;
    return t / (NS >> 1);
}

// position in nk[0..sz) (shared memory) of the first key >= q
template <class K>
__device__ __forceinline__ uint32_t smem_lower_bound(const K* nk, uint32_t sz, K q)
{
    uint32_t base = 0, len = sz;
    while (len > 0) {
        uint32_t half = len >> 1;
        if (nk[base + half] < q) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// End of the prefix of the sorted updates [j, ue) whose key <= bd (the updates routed to the
// current node): a 32-way search by the whole warp, 32 independent probes per round.
template <class K>
__device__ __forceinline__ uint32_t routed_end(const K* __restrict__ ukey, uint32_t j, uint32_t ue, K bd)
{
    const uint32_t lane = threadIdx.x & 31;
    uint32_t lo = j, hi = ue;   // keys below lo are <= bd, keys from hi on are > bd
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo) / 32;
        const uint32_t c = __popc(__ballot_sync(FULL, ukey[lo + (lane + 1) * step - 1] <= bd));
        // probes 0..c-1 hold keys <= bd, probe c (if any) a key > bd
        if (c < 32) hi = lo + (c + 1) * step - 1;
        lo += c * step;
    }
    const bool in = lo + lane < hi && ukey[lo + lane] <= bd;
    return lo + __popc(__ballot_sync(FULL, in));
}

template <class K>
__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// First-node state of the 32 consecutive buckets a warp owns (lane l: bucket b0 + l): the bucket's
// update sublist [us, ue) and its first node's id, size, maxKey and node-link, all loaded in
// parallel before the warp works through the buckets that have updates.
template <class K>
struct UGroup {
    uint32_t us, ue, node, sz, nx;
    K bd;
};

template <class K>
__device__ __forceinline__ uint32_t load_ugroup(const DevIdx<K>& ix, const uint32_t* __restrict__ uoff, uint64_t b0,
                                                uint32_t lane, UGroup<K>& g)
{
    const uint64_t b = b0 + lane;
    const bool valid = b < ix.nb;
    g.us = valid ? uoff[b] : 0u;
    g.ue = valid ? uoff[b + 1] : 0u;
    const bool touched = g.us < g.ue;
    g.node = NIL;
    g.sz = 0;
    g.nx = NIL;
    g.bd = K(0);
    if (touched) {
        // node b is usually bucket b's first node (see find_node): its metadata is read beside the
        // head and replaced when the head names another node
        g.node = ix.head[b];
        g.sz = ix.size[b];
        g.bd = ix.bound[b];
        g.nx = ix.next[b];
        if (g.node != (uint32_t)b) {
            g.sz = ix.size[g.node];
            g.bd = ix.bound[g.node];
            g.nx = ix.next[g.node];
        }
    }
    return __ballot_sync(FULL, touched);
}

constexpr int MAXQ = 4;   // node slots per lane when a node is held in registers (NS <= 128)

// Load the first sz keys (and values if vals != nullptr) of a node into per-lane registers.
template <class K>
__device__ __forceinline__ void lift_regs(const K* __restrict__ nk, const K* __restrict__ nv, uint32_t sz,
                                          uint32_t lane, K (&rk)[MAXQ], K (&rv)[MAXQ])
{
#pragma unroll
    for (int q = 0; q < MAXQ; q++) {
        const uint32_t s = lane + 32 * q;
        if (s < sz) {
            rk[q] = nk[s];
            if (nv) rv[q] = nv[s];
        }
    }
}

template <class K>
__device__ __forceinline__ void stage_regs(K* sk, K* sv, uint32_t sz, uint32_t lane, const K (&rk)[MAXQ],
                                           const K (&rv)[MAXQ])
{
#pragma unroll
    for (int q = 0; q < MAXQ; q++) {
        const uint32_t s = lane + 32 * q;
        if (s < sz) {
            sk[s] = rk[q];
            if (sv) sv[s] = rv[q];
        }
    }
}

// A bucket whose chain is one node and that receives at most FAST_U updates is handled by one
// lane (every lane of a warp on its own bucket at once) instead of by the whole warp: the count
// pass looks each update up in the node, and, when the merged run still fits the node, the apply
// pass merges in place (deletions compact forward, then insertions merge backward from the end).
// The result is the layout the warp path gives.
constexpr uint32_t FAST_U = 8;

// position in nk[0..sz) (global memory) of the first key >= q
template <class K>
__device__ __forceinline__ uint32_t gmem_lower_bound(const K* nk, uint32_t sz, K q)
{
    uint32_t base = 0, len = sz;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (nk[base + half] < q) { base += half + 1; len -= half + 1; }
        else len = half;
    }
    return base;
}

// merged size of a one-node bucket: sz + absent inserts/upserts - present deletes
template <class K>
__device__ __forceinline__ uint32_t lane_count(const K* nk, uint32_t sz, const K* __restrict__ ukey,
                                               const uint32_t* __restrict__ uop, uint32_t us, uint32_t ue)
{
    uint32_t t = sz;
    for (uint32_t u = us; u < ue; u++) {
        const K key = ukey[u];
        const uint32_t op = uop[u];
        const uint32_t pos = gmem_lower_bound(nk, sz, key);
        const bool present = pos < sz && nk[pos] == key;
        if (!present && (op == EFF_INS || op == EFF_UPS)) t++;
        if (present && op == EFF_DEL) t--;
    }
    return t;
}

// Moves node slots [lo, hi] to [lo + d, hi + d] (d > 0: from the top down) or to [lo - e, hi - e]
// (e > 0, from the bottom up), eight slots per round: a round's loads are all issued before its
// stores, and no store of a round touches a slot a later round reads.
constexpr int MOVE_BATCH = 8;

template <class K>
__device__ __forceinline__ void move_up(K* nk, K* nv, int64_t lo, int64_t hi, uint32_t d)
{
    for (int64_t top = hi; top >= lo; top -= MOVE_BATCH) {
        K tk[MOVE_BATCH], tv[MOVE_BATCH];
#pragma unroll
        for (int q = 0; q < MOVE_BATCH; q++)
            if (top - q >= lo) { tk[q] = nk[top - q]; tv[q] = nv[top - q]; }
#pragma unroll
        for (int q = 0; q < MOVE_BATCH; q++)
            if (top - q >= lo) { nk[top - q + d] = tk[q]; nv[top - q + d] = tv[q]; }
    }
}

template <class K>
__device__ __forceinline__ void move_down(K* nk, K* nv, uint32_t lo, uint32_t hi_excl, uint32_t e)
{
    for (uint32_t bot = lo; bot < hi_excl; bot += MOVE_BATCH) {
        K tk[MOVE_BATCH], tv[MOVE_BATCH];
#pragma unroll
        for (int q = 0; q < MOVE_BATCH; q++)
            if (bot + q < hi_excl) { tk[q] = nk[bot + q]; tv[q] = nv[bot + q]; }
#pragma unroll
        for (int q = 0; q < MOVE_BATCH; q++)
            if (bot + q < hi_excl) { nk[bot + q - e] = tk[q]; nv[bot + q - e] = tv[q]; }
    }
}

// In-place merge of a one-node bucket's updates into its node; t = merged size (<= NS).
template <class K>
__device__ __forceinline__ void lane_apply(K* nk, K* nv, uint32_t sz, uint32_t t, const K* __restrict__ ukey,
                                           const uint32_t* __restrict__ uop, const K* __restrict__ uval, uint32_t us,
                                           uint32_t ue)
{
    // Deletions of present keys close their slots (the run between two deletions moves down by the
    // deletions so far); upserts of present keys take the new value in place.
    uint32_t rc = 0, ndel = 0;   // slots below rc are final
    for (uint32_t u = us; u < ue; u++) {
        const uint32_t op = uop[u];
        if (op == EFF_INS) continue;
        const K key = ukey[u];
        const uint32_t pos = rc + gmem_lower_bound(nk + rc, sz - rc, key);
        if (pos >= sz || nk[pos] != key) continue;
        if (op == EFF_UPS) {
            nv[pos] = uval[u];
            continue;
        }
        if (ndel) move_down(nk, nv, rc, pos, ndel);
        rc = pos + 1;
        ndel++;
    }
    if (ndel) move_down(nk, nv, rc, sz, ndel);
    const uint32_t sz1 = sz - ndel;
    // Insertions (and upserts) of absent keys, from the largest: the node keys above one move up by
    // the insertions still to place, which leaves its slot free; w - (r + 1) insertions remain.
    int64_t r = (int64_t)sz1 - 1;
    int64_t w = t;
    for (int64_t u = (int64_t)ue - 1; u >= (int64_t)us && w > r + 1; u--) {
        const uint32_t op = uop[u];
        if (op == EFF_DEL) continue;
        const K uk = ukey[u];
        // number of kept keys <= uk
        uint32_t base = 0, len = (uint32_t)(r + 1);
        while (len > 0) {
            const uint32_t half = len >> 1;
            if (!(uk < nk[base + half])) { base += half + 1; len -= half + 1; }
            else len = half;
        }
        if (base > 0 && nk[base - 1] == uk) continue;   // present: no insertion
        const uint32_t d = (uint32_t)(w - 1 - r);
        if ((int64_t)base <= r) move_up(nk, nv, base, r, d);
        w -= r + 1 - base;
        nk[w - 1] = uk;
        nv[w - 1] = uval[u];
        w--;
        r = (int64_t)base - 1;
    }
}

// A node that receives more than HEAVY_U updates (a whole batch landing in one bucket, as sorted
// or clustered keys do) is merged by a block of its own (k_update_heavy) rather than by the warp
// that owns its bucket; the warp still writes the node's chain metadata.
constexpr uint32_t HEAVY_U = 2048;
constexpr int HV_THREADS = 256;
constexpr int HV_ITEMS = 8;
constexpr int HV_CHUNK = HV_THREADS * HV_ITEMS;

struct HeavyNode {
    uint32_t node, j, k, t, sz;
    uint32_t need_before;   // nodes the bucket's earlier chain nodes allocate in this batch
    uint64_t b;             // its bucket
    uint32_t chunk0;        // its first chunk of HV_CHUNK updates in the chunk arrays
    uint32_t add, del;      // absent keys it inserts, present keys it deletes
    uint32_t delm[4];       // node slots the batch deletes (NS <= 128)
};
constexpr uint32_t HEAVY_FLAG = 0x80000000u;   // tnode[node] = slot | HEAVY_FLAG between find and count
constexpr int FIND_GROUPS = 8;                 // groups of 32 buckets per warp of k_heavy_find

// Heavy nodes are handled in chunks of HV_CHUNK updates, spread over all blocks:
//   k_heavy_find   lists the nodes with more than HEAVY_U updates (only buckets with that many
//                  updates are walked) and snapshots each one's keys and values; its last block
//                  to finish numbers the chunks (first chunk of each node);
//   k_heavy_count  per chunk: present keys it deletes (marked) or upserts (snapshot value replaced)
//                  and absent keys it inserts (counted per chunk and per node); its last block
//                  takes the prefix of the chunk counts, so each chunk knows the inserts before it;
//   k_update_count takes a heavy node's merged size from these counts;
//   k_update_heavy per chunk: places its inserted keys and the node keys in its key range.
// Every kernel reads the snapshot, because placing writes into the node itself.

template <class K>
__global__ void __launch_bounds__(UP_THREADS, 10) k_update_count(DevIdx<K> ix, const K* __restrict__ ukey,
                                                             const uint32_t* __restrict__ uop,
                                                             const uint32_t* __restrict__ uoff,
                                                             uint32_t* __restrict__ tnode, uint64_t* __restrict__ nf,
                                                             uint8_t* __restrict__ allgone,
                                                             HeavyNode* __restrict__ heavy, uint32_t* __restrict__ heavy_n,
                                                             uint32_t heavy_cap)
{
    grid_dep_enter();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t NS = ix.NS;
    K* sk = reinterpret_cast<K*>(smem_raw) + (size_t)w * NS;
    const uint64_t b0 = ((uint64_t)blockIdx.x * UP_WARPS + w) * 32;
    if (b0 >= ix.nb) return;
    UGroup<K> g;
    uint32_t mask = load_ugroup(ix, uoff, b0, lane, g);
    if (b0 + lane < ix.nb && !((mask >> lane) & 1u)) {
        nf[b0 + lane] = 0;
        allgone[b0 + lane] = 0;
    }
    const bool fast = ((mask >> lane) & 1u) && ix.lane_path && g.nx == NIL && g.ue - g.us <= FAST_U;
    if (fast) {
        const uint32_t t = lane_count<K>(ix.keys + (uint64_t)g.node * NS, g.sz, ukey, uop, g.us, g.ue);
        tnode[g.node] = t;
        const uint32_t q = pieces_of(t, NS);
        nf[b0 + lane] = q > 1 ? q - 1 : 0;   // an emptied only node stays: nothing freed
        allgone[b0 + lane] = t == 0;
    }
    mask &= ~__ballot_sync(FULL, fast);
    while (mask) {
        const uint32_t i = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t ue = __shfl_sync(FULL, g.ue, i);
        uint32_t j = __shfl_sync(FULL, g.us, i);
        uint32_t node = __shfl_sync(FULL, g.node, i);
        uint32_t sz = __shfl_sync(FULL, g.sz, i);
        uint32_t nx = __shfl_sync(FULL, g.nx, i);
        K bd = __shfl_sync(FULL, g.bd, i);
        uint64_t need = 0, dropped = 0;
        bool all_dropped = true;
        uint32_t steps = 0;
        for (;;) {
            K rk[MAXQ], rv[MAXQ];
            lift_regs<K>(ix.keys + (uint64_t)node * NS, nullptr, sz, lane, rk, rv);   // overlaps routed_end
            const uint32_t k = routed_end(ukey, j, ue, bd);
            if (k == j) {
                all_dropped = false;
            } else if (k - j > HEAVY_U) {
                // listed by k_heavy_find and counted by k_heavy_count
                const uint32_t slot = tnode[node];
                uint32_t t = 0;
                if (slot & HEAVY_FLAG) {
                    HeavyNode& hn = heavy[slot & ~HEAVY_FLAG];
                    t = sz + hn.add - hn.del;
                    __syncwarp();
                    if (lane == 0) {
                        tnode[node] = t;
                        hn.t = t;
                        hn.need_before = (uint32_t)need;
                    }
                } else if (lane == 0) {
                    atomicOr(ix.err, ERR_STEPS);   // the list overflowed
                }
                const uint32_t q = pieces_of(t, NS);
                if (q > 1) need += q - 1;
                if (t == 0) dropped++;
                else all_dropped = false;
                j = k;
                __syncwarp();
            } else {
                stage_regs<K>(sk, nullptr, sz, lane, rk, rv);
                __syncwarp();
                uint32_t add = 0, del = 0;
                // four rounds of 32 updates per step: their loads are independent
                for (uint32_t c0 = j; c0 < k; c0 += 128) {
                    K key[4];
                    uint32_t op[4];
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        const uint32_t u = c0 + r * 32 + lane;
                        op[r] = u < k ? uop[u] : EFF_NONE;
                        key[r] = u < k ? ukey[u] : K(0);
                    }
#pragma unroll
                    for (int r = 0; r < 4; r++) {
                        if (op[r] == EFF_NONE) continue;
                        const uint32_t pos = smem_lower_bound(sk, sz, key[r]);
                        const bool present = pos < sz && sk[pos] == key[r];
                        if (!present && (op[r] == EFF_INS || op[r] == EFF_UPS)) add++;
                        if (present && op[r] == EFF_DEL) del++;
                    }
                }
                add = warp_sum<K>(add);
                del = warp_sum<K>(del);
                const uint32_t t = sz + add - del;
                if (lane == 0) tnode[node] = t;
                const uint32_t q = pieces_of(t, NS);
                if (q > 1) need += q - 1;
                if (t == 0) dropped++;
                else all_dropped = false;
                j = k;
                __syncwarp();
            }
            if (j >= ue) break;
            node = nx;
            if (node == NIL || ++steps > ix.cap) {
                if (lane == 0) atomicOr(ix.err, ERR_CHAIN);
                return;
            }
            sz = ix.size[node];
            bd = ix.bound[node];
            nx = ix.next[node];
        }
        uint64_t freed = dropped;
        uint8_t ag = 0;
        if (all_dropped && nx == NIL) {   // every node of the chain empties: the first one stays
            freed = dropped - 1;
            ag = 1;
        }
        if (lane == 0) {
            nf[b0 + i] = need | (freed << 32);
            allgone[b0 + i] = ag;
        }
    }
}

template <class K>
__global__ void __launch_bounds__(UP_THREADS) k_update_apply(DevIdx<K> ix, const K* __restrict__ ukey,
                                                             const uint32_t* __restrict__ uop, const K* __restrict__ uval,
                                                             const uint32_t* __restrict__ uoff,
                                                             const uint32_t* __restrict__ tnode,
                                                             const uint64_t* __restrict__ nf_off,
                                                             const uint8_t* __restrict__ allgone,
                                                             const uint32_t* __restrict__ alloc_ids,
                                                             uint32_t* __restrict__ free_ids,
                                                             const DevState* __restrict__ ds)
{
    grid_dep_enter();
    if (!ds->admitted) return;
    const uint64_t push_base = ds->from;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t NS = ix.NS, S2 = NS >> 1;
    // per-warp shared layout: keys[NS], vals[NS], addcnt[NS + 1], delmask[NS/32 + 1]
    const size_t per_warp = (size_t)NS * 2 * sizeof(K) + (size_t)(NS + 1) * 4 + (NS / 32 + 1) * 4;
    unsigned char* base = smem_raw + (size_t)w * ((per_warp + 15) & ~size_t(15));
    K* sk = reinterpret_cast<K*>(base);
    K* sv = sk + NS;
    uint32_t* addcnt = reinterpret_cast<uint32_t*>(sv + NS);
    uint32_t* delmask = addcnt + NS + 1;
    const uint64_t b0 = ((uint64_t)blockIdx.x * UP_WARPS + w) * 32;
    if (b0 >= ix.nb) return;
    UGroup<K> g;
    uint32_t mask = load_ugroup(ix, uoff, b0, lane, g);
    // per-bucket allocation cursors and the first node's merged size, also in parallel
    uint64_t nfo_l = 0;
    uint32_t t0_l = 0, ag_l = 0;
    if ((mask >> lane) & 1u) {
        nfo_l = nf_off[b0 + lane];
        ag_l = allgone[b0 + lane];
        t0_l = tnode[g.node];
    }
    const bool fast = ((mask >> lane) & 1u) && ix.lane_path && g.nx == NIL && g.ue - g.us <= FAST_U && t0_l <= NS;
    if (fast) {
        lane_apply<K>(ix.keys + (uint64_t)g.node * NS, ix.vals + (uint64_t)g.node * NS, g.sz, t0_l, ukey, uop, uval,
                      g.us, g.ue);
        ix.size[g.node] = t0_l;
    }
    mask &= ~__ballot_sync(FULL, fast);
    const uint32_t lt = lanemask_lt();
    while (mask) {
        const uint32_t i = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint64_t b = b0 + i;
        const uint32_t ue = __shfl_sync(FULL, g.ue, i);
        uint32_t j = __shfl_sync(FULL, g.us, i);
        uint32_t node = __shfl_sync(FULL, g.node, i);
        uint32_t sz = __shfl_sync(FULL, g.sz, i);
        uint32_t nx = __shfl_sync(FULL, g.nx, i);
        K bd = __shfl_sync(FULL, g.bd, i);
        uint32_t t = __shfl_sync(FULL, t0_l, i);
        const uint64_t nfo = __shfl_sync(FULL, nfo_l, i);
        const bool ag = __shfl_sync(FULL, ag_l, i) != 0;
        const uint64_t need_base = nfo & 0xFFFFFFFFull;
        const uint64_t free_base = nfo >> 32;
        uint32_t prev_tail = NIL;
        uint64_t acur = 0, fcur = 0;
        bool first = true, last_dropped = false;
        uint32_t steps = 0;
        for (;;) {
            K rk[MAXQ], rv[MAXQ];
            lift_regs<K>(ix.keys + (uint64_t)node * NS, ix.vals + (uint64_t)node * NS, sz, lane, rk, rv);
            const uint32_t k = routed_end(ukey, j, ue, bd);
            if (k == j) {
                prev_tail = node;
                last_dropped = false;
            } else {
                const uint32_t q = pieces_of(t, NS);
                if (k - j > HEAVY_U) {
                    // a heavy node: its keys are placed by k_update_heavy, its chain metadata here
                } else {
                stage_regs<K>(sk, sv, sz, lane, rk, rv);
                for (uint32_t s = lane; s <= NS; s += 32) addcnt[s] = 0;
                if (lane <= NS / 32) delmask[lane] = 0;
                __syncwarp();
                // output slot of merged position p: piece r (the node for r = 0, new nodes after)
                auto place = [&](uint32_t p, K key, K val) {
                    uint32_t r = 0;
                    if (q > 1) { r = p / S2; if (r > q - 1) r = q - 1; }
                    const uint32_t slot = p - r * S2;
                    const uint32_t dn = r == 0 ? node : alloc_ids[need_base + acur + r - 1];
                    ix.keys[(uint64_t)dn * NS + slot] = key;
                    ix.vals[(uint64_t)dn * NS + slot] = val;
                    if (q > 1 && r < q - 1 && slot == S2 - 1) ix.bound[dn] = key;
                };
                // pass 1: deletions mark their slot (Tab. 3's mask); upserts of present keys replace values
                for (uint32_t c0 = j; c0 < k; c0 += 32) {
                    const uint32_t u = c0 + lane;
                    if (u < k) {
                        const K key = ukey[u];
                        const uint32_t op = uop[u];
                        const uint32_t pos = smem_lower_bound(sk, sz, key);
                        if (pos < sz && sk[pos] == key) {
                            if (op == EFF_DEL) atomicOr(&delmask[pos >> 5], 1u << (pos & 31));
                            else if (op == EFF_UPS) sv[pos] = uval[u];
                        }
                    }
                }
                __syncwarp();
                // pass 2: inserted keys take their merged position
                uint32_t added_before = 0;
                for (uint32_t c0 = j; c0 < k; c0 += 32) {
                    const uint32_t u = c0 + lane;
                    bool add = false;
                    K key = K(0);
                    uint32_t pos = 0;
                    if (u < k) {
                        key = ukey[u];
                        const uint32_t op = uop[u];
                        pos = smem_lower_bound(sk, sz, key);
                        const bool present = pos < sz && sk[pos] == key;
                        add = !present && (op == EFF_INS || op == EFF_UPS);
                    }
                    const uint32_t am = __ballot_sync(FULL, add);
                    if (add) {
                        uint32_t dels_below = 0;
                        for (uint32_t wd = 0; wd < (pos >> 5); wd++) dels_below += __popc(delmask[wd]);
                        if (pos & 31) dels_below += __popc(delmask[pos >> 5] & ((1u << (pos & 31)) - 1));
                        const uint32_t p = pos - dels_below + added_before + __popc(am & lt);
                        place(p, key, uval[u]);
                        atomicAdd(&addcnt[pos], 1u);
                    }
                    added_before += __popc(am);
                }
                __syncwarp();
                // pass 3: surviving node keys shift by (inserted before) - (deleted before)
                uint32_t carry = 0;
                for (uint32_t c0 = 0; c0 < sz; c0 += 32) {
                    const uint32_t s = c0 + lane;
                    uint32_t a = s < sz ? addcnt[s] : 0;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        uint32_t y = __shfl_up_sync(FULL, a, o);
                        if (lane >= o) a += y;
                    }
                    if (s < sz && !((delmask[s >> 5] >> (s & 31)) & 1u)) {
                        uint32_t dels_below = 0;
                        for (uint32_t wd = 0; wd < (s >> 5); wd++) dels_below += __popc(delmask[wd]);
                        if (s & 31) dels_below += __popc(delmask[s >> 5] & ((1u << (s & 31)) - 1));
                        place(s - dels_below + carry + a, sk[s], sv[s]);
                    }
                    carry += __shfl_sync(FULL, a, 31);
                }
                }
                // chain metadata
                if (t == 0) {
                    if (ag && first) {
                        // the whole chain empties: its first node stays as the bucket's only node
                        if (lane == 0) ix.size[node] = 0;
                        prev_tail = node;
                        last_dropped = false;
                    } else {
                        if (lane == 0) {
                            if (prev_tail == NIL) ix.head[b] = nx; else ix.next[prev_tail] = nx;
                            free_ids[push_base + free_base + fcur] = node;
                        }
                        fcur++;
                        last_dropped = (nx == NIL);
                    }
                } else {
                    for (uint32_t r = lane; r < q; r += 32) {
                        const uint32_t dn = r == 0 ? node : alloc_ids[need_base + acur + r - 1];
                        const uint32_t dnext = r + 1 < q ? alloc_ids[need_base + acur + r] : nx;
                        ix.size[dn] = r + 1 < q ? S2 : t - (q - 1) * S2;
                        ix.next[dn] = dnext;
                        if (r + 1 == q) ix.bound[dn] = bd;
                    }
                    if (lane == 0) {
                        if (prev_tail == NIL) ix.head[b] = node; else ix.next[prev_tail] = node;
                    }
                    prev_tail = q > 1 ? alloc_ids[need_base + acur + q - 2] : node;
                    acur += q - 1;
                    last_dropped = false;
                }
                j = k;
                __syncwarp();
            }
            first = false;
            if (j >= ue) break;
            node = nx;
            if (node == NIL || ++steps > ix.cap) {
                if (lane == 0) atomicOr(ix.err, ERR_CHAIN);
                return;
            }
            sz = ix.size[node];
            bd = ix.bound[node];
            nx = ix.next[node];
            t = tnode[node];
        }
        if (last_dropped && lane == 0 && prev_tail != NIL) ix.bound[prev_tail] = ix.mkba[b];
    }
}

// Chunks of the heavy nodes: chunk g belongs to the node h with chunk0[h] <= g < chunk0[h + 1].
__device__ __forceinline__ uint32_t heavy_of_chunk(const HeavyNode* __restrict__ heavy, uint32_t nh, uint32_t g)
{
    uint32_t lo = 0, len = nh;
    while (len > 0) {            // last h with chunk0[h] <= g
        const uint32_t half = len >> 1;
        if (heavy[lo + half].chunk0 <= g) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo - 1;
}

// Numbers the heavy nodes' chunks (one block of any multiple of 32 threads up to 256): chunk0 of
// each node, the total in *nchunks.  The records come from other blocks: read past L1.
__device__ void heavy_chunks(HeavyNode* __restrict__ heavy, const uint32_t* __restrict__ heavy_n, uint32_t heavy_cap,
                             uint32_t* __restrict__ nchunks, uint32_t chunk_cap, uint32_t* __restrict__ err)
{
    __shared__ uint32_t sw[8];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t nh = min(__ldcg(heavy_n), heavy_cap);
    uint32_t carry = 0;
    for (uint32_t h0 = 0; h0 < nh; h0 += blockDim.x) {
        const uint32_t h = h0 + threadIdx.x;
        const uint32_t c = h < nh ? (__ldcg(&heavy[h].k) - __ldcg(&heavy[h].j) + HV_CHUNK - 1) / HV_CHUNK : 0;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) sw[w] = x;
        __syncthreads();
        uint32_t wbase = 0, total = 0;
        for (uint32_t q = 0; q < nw; q++) {
            if (q < w) wbase += sw[q];
            total += sw[q];
        }
        if (h < nh) heavy[h].chunk0 = carry + wbase + x - c;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry > chunk_cap) {
            atomicOr(err, ERR_STEPS);
            carry = chunk_cap;
        }
        nchunks[0] = carry;
    }
}

// Lists the heavy nodes: a warp walks the chains of its buckets that hold more than HEAVY_U
// updates (the same walk as the count pass: routed_end per node), records each node with more than
// HEAVY_U of them, marks it in tnode and snapshots its keys and values.  Other warps only read
// their buckets' update ranges.
template <class K>
__global__ void __launch_bounds__(UP_THREADS) k_heavy_find(DevIdx<K> ix, const K* __restrict__ ukey,
                                                           const uint32_t* __restrict__ uoff,
                                                           uint32_t* __restrict__ tnode, HeavyNode* __restrict__ heavy,
                                                           uint32_t* __restrict__ heavy_n, uint32_t heavy_cap,
                                                           K* __restrict__ snap_k, K* __restrict__ snap_v,
                                                           uint32_t* __restrict__ nchunks, uint32_t chunk_cap)
{
    grid_dep_enter();
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t NS = ix.NS;
    bool failed = false;
    // a warp takes FIND_GROUPS groups of 32 buckets, their update ranges loaded at once
    const uint64_t g0 = ((uint64_t)blockIdx.x * UP_WARPS + w) * FIND_GROUPS;
    uint32_t usv[FIND_GROUPS], uev[FIND_GROUPS];
#pragma unroll
    for (int q = 0; q < FIND_GROUPS; q++) {
        const uint64_t bl = (g0 + q) * 32 + lane;
        usv[q] = bl < ix.nb ? uoff[bl] : 0u;
        uev[q] = bl < ix.nb ? uoff[bl + 1] : 0u;
    }
#pragma unroll 1
    for (int q = 0; q < FIND_GROUPS && !failed; q++) {
    const uint64_t b0 = (g0 + q) * 32;
    const uint32_t us = usv[q], ue0 = uev[q];
    uint32_t mask = __ballot_sync(FULL, ue0 - us > HEAVY_U);
    while (mask && !failed) {
        const uint32_t i = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t ue = __shfl_sync(FULL, ue0, i);
        uint32_t j = __shfl_sync(FULL, us, i);
        uint32_t node = ix.head[b0 + i];
        uint32_t sz = ix.size[node], nx = ix.next[node];
        K bd = ix.bound[node];
        uint32_t steps = 0;
        for (;;) {
            const uint32_t k = routed_end(ukey, j, ue, bd);
            if (k - j > HEAVY_U) {
                uint32_t slot = 0;
                if (lane == 0) slot = atomicAdd(heavy_n, 1u);
                slot = __shfl_sync(FULL, slot, 0);
                if (slot < heavy_cap) {
                    if (lane == 0) {
                        HeavyNode hn;
                        hn.node = node; hn.j = j; hn.k = k; hn.t = 0; hn.sz = sz; hn.need_before = 0;
                        hn.b = b0 + i; hn.chunk0 = 0; hn.add = 0; hn.del = 0;
                        hn.delm[0] = hn.delm[1] = hn.delm[2] = hn.delm[3] = 0;
                        heavy[slot] = hn;
                        tnode[node] = slot | HEAVY_FLAG;
                    }
                    for (uint32_t s2 = lane; s2 < sz; s2 += 32) {
                        snap_k[(uint64_t)slot * NS + s2] = ix.keys[(uint64_t)node * NS + s2];
                        snap_v[(uint64_t)slot * NS + s2] = ix.vals[(uint64_t)node * NS + s2];
                    }
                } else if (lane == 0) {
                    atomicOr(ix.err, ERR_STEPS);
                }
            }
            j = k;
            if (j >= ue) break;
            node = nx;
            if (node == NIL || ++steps > ix.cap) {
                if (lane == 0) atomicOr(ix.err, ERR_CHAIN);
                failed = true;
                break;
            }
            sz = ix.size[node];
            bd = ix.bound[node];
            nx = ix.next[node];
        }
    }
    }
    // the last block to finish numbers the chunks
    __shared__ uint32_t s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&nchunks[1], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        heavy_chunks(heavy, heavy_n, heavy_cap, nchunks, chunk_cap, ix.err);
        if (threadIdx.x == 0) nchunks[1] = 0;
    }
}

// Exclusive prefix of the chunk counts over all chunks (one block of HV_THREADS threads); a chunk's
// inserts before it in its node are chunk_pre[g] - chunk_pre[chunk0].  The counts come from other
// blocks: read past L1.
__device__ void heavy_scan(const uint32_t* __restrict__ chunk_add, uint32_t ng, uint32_t* __restrict__ chunk_pre)
{
    __shared__ uint32_t sw[HV_THREADS / 32];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t carry = 0;
    for (uint32_t g0 = 0; g0 < ng; g0 += HV_THREADS) {
        const uint32_t g = g0 + threadIdx.x;
        const uint32_t c = g < ng ? __ldcg(chunk_add + g) : 0;
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) sw[w] = x;
        __syncthreads();
        uint32_t wbase = 0, total = 0;
        for (int q = 0; q < HV_THREADS / 32; q++) {
            if (q < (int)w) wbase += sw[q];
            total += sw[q];
        }
        if (g < ng) chunk_pre[g] = carry + wbase + x - c;
        carry += total;
        __syncthreads();
    }
}

// Per chunk of a heavy node: present keys it deletes are marked, present keys it upserts take
// their new value in the snapshot, absent keys it inserts are counted (chunk_add[g] and the node's
// add; deletions in the node's del).
template <class K>
__global__ void __launch_bounds__(HV_THREADS) k_heavy_count(uint32_t NS, const K* __restrict__ ukey,
                                                           const uint32_t* __restrict__ uop, const K* __restrict__ uval,
                                                           HeavyNode* __restrict__ heavy,
                                                           const uint32_t* __restrict__ heavy_n, uint32_t heavy_cap,
                                                           const K* __restrict__ snap_k, K* __restrict__ snap_v,
                                                           uint32_t* __restrict__ nchunks,
                                                           uint32_t* __restrict__ chunk_add,
                                                           uint32_t* __restrict__ chunk_pre)
{
    grid_dep_enter();
    __shared__ K nk[128];
    __shared__ uint32_t sa[HV_THREADS / 32], sd[HV_THREADS / 32];
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nh = min(*heavy_n, heavy_cap), ng = *nchunks;
    for (uint32_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const uint32_t h = heavy_of_chunk(heavy, nh, g);
        const uint32_t sz = heavy[h].sz;
        const uint32_t c0 = heavy[h].j + (g - heavy[h].chunk0) * HV_CHUNK;
        const uint32_t cn = min((uint32_t)HV_CHUNK, heavy[h].k - c0);
        for (uint32_t s2 = threadIdx.x; s2 < sz; s2 += HV_THREADS) nk[s2] = snap_k[(uint64_t)h * NS + s2];
        __syncthreads();
        uint32_t add = 0, del = 0;
#pragma unroll
        for (int r = 0; r < HV_ITEMS; r++) {
            const uint32_t i = r * HV_THREADS + threadIdx.x;
            if (i < cn) {
                const K key = ukey[c0 + i];
                const uint32_t op = uop[c0 + i];
                const uint32_t pos = smem_lower_bound(nk, sz, key);
                const bool present = pos < sz && nk[pos] == key;
                if (present && op == EFF_DEL) {
                    atomicOr(&heavy[h].delm[pos >> 5], 1u << (pos & 31));
                    del++;
                }
                if (present && op == EFF_UPS) snap_v[(uint64_t)h * NS + pos] = uval[c0 + i];
                add += !present && (op == EFF_INS || op == EFF_UPS);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            add += __shfl_xor_sync(FULL, add, o);
            del += __shfl_xor_sync(FULL, del, o);
        }
        if (lane == 0) { sa[w] = add; sd[w] = del; }
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t ta = 0, td = 0;
            for (int q = 0; q < HV_THREADS / 32; q++) { ta += sa[q]; td += sd[q]; }
            chunk_add[g] = ta;
            if (ta) atomicAdd(&heavy[h].add, ta);
            if (td) atomicAdd(&heavy[h].del, td);
        }
        __syncthreads();   // nk, sa and sd are rewritten for the next chunk
    }
    // the last block to finish takes the prefix of the chunk counts
    __shared__ uint32_t s_last;
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&nchunks[2], 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last) {
        __threadfence();
        heavy_scan(chunk_add, ng, chunk_pre);
        if (threadIdx.x == 0) nchunks[2] = 0;
    }
}

// Places a heavy node's pairs, one chunk of its updates per block step.  The snapshot of the node
// (with upserted values) and its deletion marks are staged in shared memory.  An inserted key goes
// to (surviving node keys below it) + (inserted keys before it: the chunk's carry from the scan
// plus a block scan inside the chunk); a surviving node key goes to (surviving node keys below it)
// + (inserted keys below it), placed by the chunk whose key range holds it (the first chunk also
// takes the keys below every update, the last the keys above).  Same positions and pieces as the
// warp path; piece metadata comes from k_update_apply.
template <class K>
__global__ void __launch_bounds__(HV_THREADS) k_update_heavy(DevIdx<K> ix, const K* __restrict__ ukey,
                                                             const uint32_t* __restrict__ uop,
                                                             const K* __restrict__ uval,
                                                             const uint32_t* __restrict__ alloc_ids,
                                                             const uint64_t* __restrict__ nf_off,
                                                             const HeavyNode* __restrict__ heavy,
                                                             const uint32_t* __restrict__ heavy_n, uint32_t heavy_cap,
                                                             const K* __restrict__ snap_k, const K* __restrict__ snap_v,
                                                             const uint32_t* __restrict__ nchunks,
                                                             const uint32_t* __restrict__ chunk_pre,
                                                             const DevState* __restrict__ ds)
{
    grid_dep_enter();
    if (!ds->admitted) return;
    __shared__ K nk[128], nv[128];
    __shared__ uint32_t delm[4];
    __shared__ K ck[HV_CHUNK];
    __shared__ uint32_t cex[HV_CHUNK + 1];
    __shared__ uint32_t sw[HV_THREADS / 32];
    const uint32_t NS = ix.NS, S2 = NS >> 1;
    const uint32_t lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t nh = min(*heavy_n, heavy_cap), ng = *nchunks;
    for (uint32_t g = blockIdx.x; g < ng; g += gridDim.x) {
        const uint32_t h = heavy_of_chunk(heavy, nh, g);
        const HeavyNode hn = heavy[h];
        const uint32_t sz = hn.sz;
        const uint32_t hq = pieces_of(hn.t, NS);
        const uint64_t abase = (nf_off[hn.b] & 0xFFFFFFFFull) + hn.need_before;   // alloc_ids of its pieces 1..
        const uint32_t c = g - hn.chunk0;
        const uint32_t c0 = hn.j + c * HV_CHUNK;
        const uint32_t cn = min((uint32_t)HV_CHUNK, hn.k - c0);
        const bool last = c0 + cn == hn.k;
        const uint32_t carry = chunk_pre[g] - chunk_pre[hn.chunk0];
        for (uint32_t s2 = threadIdx.x; s2 < sz; s2 += HV_THREADS) {
            nk[s2] = snap_k[(uint64_t)h * NS + s2];
            nv[s2] = snap_v[(uint64_t)h * NS + s2];
        }
        if (threadIdx.x < 4) delm[threadIdx.x] = hn.delm[threadIdx.x];
        __syncthreads();
        auto place = [&](uint32_t p, K key, K val) {
            uint32_t r = 0;
            if (hq > 1) { r = p / S2; if (r > hq - 1) r = hq - 1; }
            const uint32_t slot = p - r * S2;
            const uint32_t dn = r == 0 ? hn.node : alloc_ids[abase + r - 1];
            ix.keys[(uint64_t)dn * NS + slot] = key;
            ix.vals[(uint64_t)dn * NS + slot] = val;
            if (hq > 1 && r < hq - 1 && slot == S2 - 1) ix.bound[dn] = key;
        };
        auto dels_below = [&](uint32_t pos) {
            uint32_t d = 0;
            for (uint32_t wd = 0; wd < (pos >> 5); wd++) d += __popc(delm[wd]);
            if (pos & 31) d += __popc(delm[pos >> 5] & ((1u << (pos & 31)) - 1));
            return d;
        };
        // items i = threadIdx.x * HV_ITEMS + r: consecutive per thread, for the scan
        uint32_t pos[HV_ITEMS];
        bool add[HV_ITEMS];
        uint32_t cnt = 0;
#pragma unroll
        for (int r = 0; r < HV_ITEMS; r++) {
            const uint32_t i = threadIdx.x * HV_ITEMS + r;
            add[r] = false;
            pos[r] = 0;
            if (i < cn) {
                const K key = ukey[c0 + i];
                const uint32_t op = uop[c0 + i];
                const uint32_t lo = smem_lower_bound(nk, sz, key);
                pos[r] = lo;
                const bool present = lo < sz && nk[lo] == key;
                add[r] = !present && (op == EFF_INS || op == EFF_UPS);
                ck[i] = key;
                cnt += add[r];
            }
        }
        uint32_t x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        if (lane == 31) sw[w] = x;
        __syncthreads();
        uint32_t wbase = 0, total = 0;
        for (int q2 = 0; q2 < HV_THREADS / 32; q2++) {
            if (q2 < (int)w) wbase += sw[q2];
            total += sw[q2];
        }
        uint32_t ex = wbase + x - cnt;
#pragma unroll
        for (int r = 0; r < HV_ITEMS; r++) {
            const uint32_t i = threadIdx.x * HV_ITEMS + r;
            if (i < cn) cex[i] = ex;
            ex += add[r];
        }
        if (threadIdx.x == 0) cex[cn] = total;
        __syncthreads();   // ck and cex complete
#pragma unroll
        for (int r = 0; r < HV_ITEMS; r++) {
            const uint32_t i = threadIdx.x * HV_ITEMS + r;
            if (add[r]) place(pos[r] - dels_below(pos[r]) + carry + cex[i], ck[i], uval[c0 + i]);
        }
        // the node keys in this chunk's key range: (key before the chunk, last key of the chunk]
        const K lo_key = c > 0 ? ukey[c0 - 1] : K(0);
        const K hi_key = ck[cn - 1];
        for (uint32_t s2 = threadIdx.x; s2 < sz; s2 += HV_THREADS) {
            const K key = nk[s2];
            if (c > 0 && !(lo_key < key)) continue;
            if (!last && hi_key < key) continue;
            if ((delm[s2 >> 5] >> (s2 & 31)) & 1u) continue;
            const uint32_t lo = smem_lower_bound(ck, cn, key);
            place(s2 - dels_below(s2) + carry + cex[lo], key, nv[s2]);
        }
        __syncthreads();   // shared state is rewritten for the next chunk
    }
}

__global__ void k_alloc_copy(const uint32_t* __restrict__ free_ids, const DevState* __restrict__ ds,
                             uint32_t* __restrict__ out, uint64_t cap_out)
{
    grid_dep_enter();
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (!ds->admitted || i >= ds->need || i >= cap_out) return;
    out[i] = free_ids[ds->from + i];
}

__global__ void k_admit(DevState* __restrict__ ds, const uint64_t* __restrict__ nf_total,
                        const uint32_t* __restrict__ badkey, const uint64_t* __restrict__ range_total,
                        uint64_t range_cap, uint64_t* __restrict__ status)
{
    grid_dep_enter();
    const uint64_t v = *nf_total;
    const uint64_t need = v & 0xFFFFFFFFull, freed = v >> 32;
    const uint64_t top = ds->free_top;
    const uint64_t rt = range_total ? *range_total : 0;
    uint64_t flags = 0;
    if (*badkey & ERR_BADKEY) flags |= ST_BADKEY;
    if (need > top) flags |= ST_NODES;
    if (rt > range_cap) flags |= ST_RANGE;
    const bool ok = flags == 0;
    ds->admitted = ok;
    ds->need = need;
    ds->freed = freed;
    ds->from = ok ? top - need : top;
    ds->next_top = ok ? top - need + freed : top;
    if (status) {
        status[0] = flags;
        status[1] = rt;
        status[2] = need;
        status[3] = top;
    }
}

__global__ void k_commit(DevState* __restrict__ ds)
{
    grid_dep_enter();
    if (ds->admitted) ds->free_top = ds->next_top;
    ds->applied = ds->admitted;
    ds->admitted = 0;
}

__global__ void k_set_free_top(DevState* __restrict__ ds, uint64_t value)
{
    grid_dep_enter();
    ds->free_top = value;
    ds->admitted = 0;
}

template <class K>
size_t count_smem(uint32_t NS) { return (size_t)UP_WARPS * NS * sizeof(K); }

template <class K>
size_t apply_smem(uint32_t NS)
{
    const size_t per_warp = (size_t)NS * 2 * sizeof(K) + (size_t)(NS + 1) * 4 + (NS / 32 + 1) * 4;
    return (size_t)UP_WARPS * ((per_warp + 15) & ~size_t(15));
}

}  // namespace

// Forces the module loader to load every kernel of this file now (see preload_kernels).
void preload_update_kernels()
{
    cudaFuncAttributes a;
#define FLIX_TOUCH(...) cudaFuncGetAttributes(&a, __VA_ARGS__)
    FLIX_TOUCH(k_fold_init);
    FLIX_TOUCH(k_fold_del);
    FLIX_TOUCH(k_fold_ins);
    FLIX_TOUCH(k_fold_emit);
    FLIX_TOUCH(k_alloc_copy);
    FLIX_TOUCH(k_admit);
    FLIX_TOUCH(k_commit);
    FLIX_TOUCH(k_set_free_top);
#define FLIX_TOUCH_K(K)                      \
    FLIX_TOUCH(k_validate<K>);               \
    FLIX_TOUCH(k_fold_flags<K>);             \
    FLIX_TOUCH(k_fold_write_mixed<K>);       \
    FLIX_TOUCH(k_fold_write_hom<K>);         \
    FLIX_TOUCH(k_update_count<K>);           \
    FLIX_TOUCH(k_update_apply<K>);           \
    FLIX_TOUCH(k_update_heavy<K>);           \
    FLIX_TOUCH(k_heavy_find<K>);             \
    FLIX_TOUCH(k_heavy_count<K>)
    FLIX_TOUCH_K(uint32_t);
    FLIX_TOUCH_K(uint64_t);
#undef FLIX_TOUCH_K
#undef FLIX_TOUCH
}

template <class K>
cudaError_t validate_inserts(Ctx& c, const uint8_t* ops, const K* keys, uint64_t n, uint32_t* flag)
{
    return launch(c, K_VALIDATE, dim3(div_up(n, 256)), dim3(256), 0, k_validate<K>, ops, keys, n, flag);
}

template <class K>
cudaError_t fold_updates(Ctx& c, const K* skeys, const uint32_t* sidx, uint64_t m, const uint8_t* ops, int hom_op,
                         const K* aux, K* ukey, uint32_t* uop, K* uval, uint32_t* u_dev)
{
    Arena& A = c.h->arena;
    uint32_t* head = A.take<uint32_t>(m + 1);
    uint32_t* hex = A.take<uint32_t>(m + 1);
    if (!head || !hex) return cudaErrorMemoryAllocation;
    const uint32_t g = div_up(m ? m : 1, 256);
    cudaError_t e;
    if (m == 0) return fill_bytes(c, u_dev, 0, 4);
    if ((e = launch(c, K_FOLD_FLAGS, dim3(g), dim3(256), 0, k_fold_flags<K>, skeys, m, head))) return e;
    if ((e = scan_exclusive<uint32_t, uint32_t>(c, head, hex, m))) return e;
    if (hom_op) {
        // U = number of distinct keys = hex[m]
        if ((e = copy_words(c, u_dev, hex + m, 1))) return e;
        const uint32_t eff = hom_op == FLIX_OP_INSERT ? EFF_INS : EFF_DEL;
        return launch(c, K_FOLD_WRITE, dim3(g), dim3(256), 0, k_fold_write_hom<K>, m, eff, skeys, sidx, aux,
                      (const uint32_t*)head, (const uint32_t*)hex, ukey, uop, uval);
    }
    uint32_t* lastdel = A.take<uint32_t>(m);
    uint32_t* firstins = A.take<uint32_t>(m);
    uint32_t* emit = A.take<uint32_t>(m + 1);
    uint32_t* eff = A.take<uint32_t>(m);
    uint32_t* hpos = A.take<uint32_t>(m);
    uint32_t* epos = A.take<uint32_t>(m + 1);
    if (!lastdel || !firstins || !emit || !eff || !hpos || !epos) return cudaErrorMemoryAllocation;
    if ((e = launch(c, K_FOLD_INIT, dim3(g), dim3(256), 0, k_fold_init, m, lastdel, firstins, emit))) return e;
    if ((e = launch(c, K_FOLD_DEL, dim3(g), dim3(256), 0, k_fold_del, sidx, m, ops, (const uint32_t*)head,
                    (const uint32_t*)hex, lastdel)))
        return e;
    if ((e = launch(c, K_FOLD_INS, dim3(g), dim3(256), 0, k_fold_ins, sidx, m, ops, (const uint32_t*)head,
                    (const uint32_t*)hex, (const uint32_t*)lastdel, firstins)))
        return e;
    if ((e = launch(c, K_FOLD_EMIT, dim3(g), dim3(256), 0, k_fold_emit, m, (const uint32_t*)head,
                    (const uint32_t*)hex, (const uint32_t*)lastdel, (const uint32_t*)firstins, emit, eff, hpos)))
        return e;
    if ((e = scan_exclusive<uint32_t, uint32_t>(c, emit, epos, m))) return e;
    if ((e = copy_words(c, u_dev, epos + m, 1))) return e;
    return launch(c, K_FOLD_WRITE, dim3(g), dim3(256), 0, k_fold_write_mixed<K>, m, skeys, sidx, aux,
                  (const uint32_t*)emit, (const uint32_t*)epos, (const uint32_t*)eff, (const uint32_t*)hpos,
                  (const uint32_t*)firstins, ukey, uop, uval);
}

template <class K>
cudaError_t update_count(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval, const uint32_t* uoff,
                         uint64_t* nf, uint8_t* allgone, const HeavyList& hl)
{
    const uint32_t grid = div_up(div_up(c.h->nb, 32), UP_WARPS);
    cudaError_t e = fill_bytes(c, hl.n, 0, 16);   // heavy count, chunk count, block counters
    if (e) return e;
    K* snap_k = static_cast<K*>(hl.snap_k);
    K* snap_v = static_cast<K*>(hl.snap_v);
    HeavyNode* heavy = static_cast<HeavyNode*>(hl.list);
    if (hl.batch > HEAVY_U) {   // no node can take more than HEAVY_U updates of a smaller batch
        const uint32_t fgrid = div_up(div_up(c.h->nb, 32), (uint64_t)UP_WARPS * FIND_GROUPS);
        if ((e = launch(c, K_HEAVY, dim3(fgrid), dim3(UP_THREADS), 0, k_heavy_find<K>, dev_view<K>(c.h), ukey, uoff,
                        c.h->tnode, heavy, hl.n, hl.cap, snap_k, snap_v, hl.nchunks, hl.chunk_cap)))
            return e;
        if ((e = launch(c, K_HEAVY, dim3(4 * c.h->nsm), dim3(HV_THREADS), 0, k_heavy_count<K>, c.h->NS, ukey, uop,
                        uval, heavy, (const uint32_t*)hl.n, hl.cap, (const K*)snap_k, snap_v, hl.nchunks, hl.chunk_add,
                        hl.chunk_pre)))
            return e;
    }
    return launch(c, K_UPD_COUNT, dim3(grid), dim3(UP_THREADS), count_smem<K>(c.h->NS), k_update_count<K>,
                  dev_view<K>(c.h), ukey, uop, uoff, c.h->tnode, nf, allgone, static_cast<HeavyNode*>(hl.list),
                  hl.n, hl.cap);
}

uint32_t heavy_cap_of(uint64_t n) { return (uint32_t)(n / HEAVY_U + 2); }   // disjoint runs of > HEAVY_U updates
// a run of u updates has ceil(u / HV_CHUNK) chunks
uint32_t chunk_cap_of(uint64_t n) { return (uint32_t)(n / HV_CHUNK + heavy_cap_of(n) + 1); }

HeavyList heavy_list(Ctx& c, uint64_t n)
{
    HeavyList hl;
    hl.cap = heavy_cap_of(n);
    hl.chunk_cap = chunk_cap_of(n);
    hl.batch = n;
    hl.list = c.h->arena.take<HeavyNode>(hl.cap);
    hl.n = c.h->arena.take<uint32_t>(4);
    hl.nchunks = hl.n ? hl.n + 1 : nullptr;
    const size_t snap = (size_t)hl.cap * c.h->NS * c.h->ks;
    hl.snap_k = c.h->arena.take<unsigned char>(snap);
    hl.snap_v = c.h->arena.take<unsigned char>(snap);
    hl.chunk_add = c.h->arena.take<uint32_t>(hl.chunk_cap);
    hl.chunk_pre = c.h->arena.take<uint32_t>(hl.chunk_cap);
    if (!hl.snap_k || !hl.snap_v || !hl.nchunks || !hl.chunk_add || !hl.chunk_pre) hl.list = nullptr;
    return hl;
}

// (with the largest node, 128 slots of 8 bytes)
size_t heavy_scratch_bytes(uint64_t n)
{
    const size_t al256 = 256;
    auto a = [&](size_t b) { return (b + al256 - 1) / al256 * al256; };
    return a((size_t)heavy_cap_of(n) * sizeof(HeavyNode)) + a(4) + 2 * a((size_t)heavy_cap_of(n) * 128 * 8) + a(4) +
           2 * a((size_t)chunk_cap_of(n) * 4) + 256;
}

template <class K>
cudaError_t update_apply(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval, const uint32_t* uoff,
                         const uint64_t* nf_off, const uint8_t* allgone, const uint32_t* alloc_ids)
{
    const uint32_t grid = div_up(div_up(c.h->nb, 32), UP_WARPS);
    return launch(c, K_UPD_APPLY, dim3(grid), dim3(UP_THREADS), apply_smem<K>(c.h->NS), k_update_apply<K>,
                  dev_view<K>(c.h), ukey, uop, uval, uoff, (const uint32_t*)c.h->tnode, nf_off, allgone, alloc_ids,
                  c.h->free_ids, (const DevState*)c.h->dstate);
}

template <class K>
cudaError_t update_heavy(Ctx& c, const K* ukey, const uint32_t* uop, const K* uval, const uint64_t* nf_off,
                         const uint32_t* alloc_ids, const HeavyList& hl)
{
    if (hl.batch <= HEAVY_U) return cudaSuccess;
    return launch(c, K_HEAVY, dim3(4 * c.h->nsm), dim3(HV_THREADS), 0, k_update_heavy<K>, dev_view<K>(c.h), ukey, uop,
                  uval, alloc_ids, nf_off, (const HeavyNode*)hl.list, (const uint32_t*)hl.n, hl.cap,
                  (const K*)hl.snap_k, (const K*)hl.snap_v, (const uint32_t*)hl.nchunks,
                  (const uint32_t*)hl.chunk_pre, (const DevState*)c.h->dstate);
}

cudaError_t alloc_copy(Ctx& c, const uint32_t* free_ids, uint32_t* out, uint64_t cap_out)
{
    return launch(c, K_ALLOC_COPY, dim3(div_up(cap_out, 256)), dim3(256), 0, k_alloc_copy, free_ids,
                  (const DevState*)c.h->dstate, out, cap_out);
}

cudaError_t admit(Ctx& c, const uint64_t* nf_total, const uint32_t* badkey, const uint64_t* range_total,
                  uint64_t range_cap, uint64_t* status)
{
    return launch(c, K_ADMIT, dim3(1), dim3(1), 0, k_admit, c.h->dstate, nf_total, badkey, range_total, range_cap,
                  status);
}

cudaError_t commit(Ctx& c) { return launch(c, K_ADMIT, dim3(1), dim3(1), 0, k_commit, c.h->dstate); }

cudaError_t set_free_top(Ctx& c, uint64_t value)
{
    c.h->free_top = value;
    return launch(c, K_ADMIT, dim3(1), dim3(1), 0, k_set_free_top, c.h->dstate, value);
}

#define FLIX_UPD_INST(K)                                                                                        \
    template cudaError_t validate_inserts<K>(Ctx&, const uint8_t*, const K*, uint64_t, uint32_t*);             \
    template cudaError_t fold_updates<K>(Ctx&, const K*, const uint32_t*, uint64_t, const uint8_t*, int,       \
                                         const K*, K*, uint32_t*, K*, uint32_t*);                              \
    template cudaError_t update_count<K>(Ctx&, const K*, const uint32_t*, const K*, const uint32_t*, uint64_t*,  \
                                         uint8_t*, const HeavyList&);                                          \
    template cudaError_t update_apply<K>(Ctx&, const K*, const uint32_t*, const K*, const uint32_t*,           \
                                         const uint64_t*, const uint8_t*, const uint32_t*);                    \
    template cudaError_t update_heavy<K>(Ctx&, const K*, const uint32_t*, const K*, const uint64_t*,           \
                                         const uint32_t*, const HeavyList&);

FLIX_UPD_INST(uint32_t)
FLIX_UPD_INST(uint64_t)

}  // namespace flix
