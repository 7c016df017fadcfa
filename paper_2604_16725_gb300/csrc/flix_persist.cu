// The batched form's persistent kernel: a queue of small mixed batches run in order by one
// cooperative launch (no launch per batch).  A grid of one wave of blocks takes the batches one
// after another; each batch goes through the method's steps as phases separated by grid barriers:
//
//   A  (block 0)   wait for the batch's ready word; sort the batch's inserts and deletes by (key,
//                  position) in shared memory (Sec. 3.3: updates are sorted before buckets pull
//                  them); fold each key's inserts and deletes into one net update (submission order)
//   B  (all)       snapshot reads (lookup, successor, predecessor, range count): bucket = number of
//                  maxBucket values below the key (Sec. 3.3), walk to the node (Sec. 4.1), search it;
//                  the bucket of every net update
//   C  (all)       one thread per touched bucket: merged size of every node of its chain and the
//                  nodes the bucket needs and frees; (block 0) the range offsets
//   D  (block 0)   admission: free nodes, range capacity, reserved key; the popped node ids
//   E1 (all)       range pairs, still on the pre-batch state
//   E2 (all)       one thread per touched bucket: merge, canonical split and compaction of every node
//                  (Sec. 4.3.2, Sec. 4.4), relink, reclaim; then (block 0) the commit
//
// The layout each batch leaves is the one the per-kernel path leaves (canonical pieces; emptied
// nodes leave the chain unless the whole chain empties; the last node's maxKey stays maxBucket).
// Every wait is bounded by a time limit: a wait that gives up stops the queue, marks the batches not
// run, and sets a timeout bit in the handle's error word.
#include <algorithm>

#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int PQ_THREADS = 256;
constexpr uint32_t PQ_MAX = FLIX_QUEUE_BATCH_MAX;
constexpr uint64_t PQ_NOT_RUN = 8;      // status[0] flag of a batch the queue did not reach
constexpr int PQ_CHUNK = 8;             // node pairs a merging thread has in flight

// Device copy of one flix_batch.
struct PQBatch {
    const uint8_t* ops;
    const void* keys;
    const void* aux;
    uint64_t n;
    void* keys_out;
    void* vals_out;
    uint8_t* found;
    uint64_t* range_off;
    void* range_keys;
    void* range_vals;
    uint64_t range_cap;
    uint64_t* status;
    const uint32_t* ready;
};

// Scratch of the queue (one batch at a time), from the handle's arena.
template <class K>
struct PQScratch {
    uint64_t* cnt;      // range pair count per input position
    uint32_t* rb;       // range start per input position: bucket, node, slot
    uint32_t* rn;
    uint32_t* rp;
    K* ukey;            // net updates in key order
    uint32_t* uop;
    K* uval;
    uint32_t* ub;       // their buckets
    uint32_t* need;     // per bucket run head: nodes needed, nodes freed, and their prefixes
    uint32_t* freed;
    uint32_t* aoff;
    uint32_t* foff;
    uint32_t* pop;      // the node ids popped for the batch
    K* mk;              // merged runs: (NS + 1) slots per net update
    K* mv;
    uint32_t* word;     // 0 U, 1 admitted, 2 need, 3 freed, 4 stop, 5 badkey, 8..9 grid barrier
    unsigned long long* wide;   // 0 free nodes before the batch, 1 range pair total
};

__device__ __forceinline__ uint32_t ld_vol(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }
__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Grid barrier of a cooperative launch (every block resident): arrival count and generation in
// word[8..9].  A wait longer than limit_ns sets the stop word and returns false; every block leaves
// the queue after a barrier at which the stop word is set.
__device__ bool grid_barrier(uint32_t* word, uint64_t limit_ns)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        uint32_t* cnt = word + 8;
        uint32_t* gen = word + 9;
        const uint32_t g = ld_vol(gen);
        __threadfence();
        if (atomicAdd(cnt, 1u) == gridDim.x - 1) {
            *reinterpret_cast<volatile uint32_t*>(cnt) = 0;
            __threadfence();
            atomicAdd(gen, 1u);
        } else {
            const uint64_t t0 = global_ns();
            while (ld_vol(gen) == g) {
                if (global_ns() - t0 > limit_ns) {
                    atomicOr(word + 4, 1u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok && ld_vol(word + 4) == 0;
    }
    __syncthreads();
    return s_ok;
}

// Exclusive scan of one value per thread over the block (PQ_THREADS), total in *tot.
template <class T>
__device__ __forceinline__ T block_scan(T v, T* sw, T& tot)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    constexpr int NW = PQ_THREADS / 32;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < NW ? sw[lane] : T(0);
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            const T y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NW) sw[lane] = t;
    }
    __syncthreads();
    const T base = w ? sw[w - 1] : T(0);
    tot = sw[NW - 1];
    __syncthreads();
    return base + x - v;
}

// Bucket of key q: the number of maxBucket values below it.
template <class K>
__device__ __forceinline__ uint32_t bucket_of(const DevIdx<K>& ix, K q)
{
    uint32_t lo = 0, len = ix.nb;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (ix.mkba[lo + half] < q) { lo += half + 1; len -= half + 1; }
        else len = half;
    }
    return lo;
}

// Pieces of a merged run of t keys (t <= NS: one node; else floor(t / (NS/2)), the last holding the
// remainder) and the size of piece r.
__device__ __forceinline__ uint32_t n_pieces(uint32_t t, uint32_t NS) { return t == 0 ? 0 : (t <= NS ? 1 : t / (NS / 2)); }
__device__ __forceinline__ uint32_t piece_size(uint32_t t, uint32_t NS, uint32_t q, uint32_t r)
{
    return q == 1 ? t : (r + 1 < q ? NS / 2 : t - (q - 1) * (NS / 2));
}

// Merged size of node x under the net updates [j, k) routed to it.
template <class K>
__device__ uint32_t merged_size(const DevIdx<K>& ix, uint32_t x, const K* ukey, const uint32_t* uop, uint32_t j,
                                uint32_t k)
{
    const K* nk = ix.keys + (uint64_t)x * ix.NS;
    const uint32_t sz = ix.size[x];
    uint32_t t = sz;
    for (uint32_t u = j; u < k; u++) {
        const uint32_t p = node_lower_bound<K, false>(nk, sz, ukey[u]);
        const bool present = p < sz && nk[p] == ukey[u];
        if (present && uop[u] == EFF_DEL) t--;
        if (!present && (uop[u] == EFF_INS || uop[u] == EFF_UPS)) t++;
    }
    return t;
}

template <class K>
__global__ void __launch_bounds__(PQ_THREADS) k_queue(DevIdx<K> ix, const PQBatch* __restrict__ q, uint32_t count,
                                                      PQScratch<K> S, DevState* __restrict__ ds, uint32_t* free_ids,
                                                      uint64_t limit_ns, unsigned long long* flags_or)
{
    grid_dep_enter();
    __shared__ K s_k[PQ_MAX];
    __shared__ uint32_t s_p[PQ_MAX];
    __shared__ uint32_t s_sw[PQ_THREADS / 32];
    __shared__ unsigned long long s_sw64[PQ_THREADS / 32];
    __shared__ int s_flag;
    const K KM = key_max<K>();
    const uint32_t NS = ix.NS;
    const uint32_t gtid = blockIdx.x * PQ_THREADS + threadIdx.x, gstride = gridDim.x * PQ_THREADS;
    uint32_t bi = 0;
    for (; bi < count; bi++) {
        const PQBatch B = q[bi];
        const uint32_t n = (uint32_t)B.n;
        const K* keys = static_cast<const K*>(B.keys);
        const K* aux = static_cast<const K*>(B.aux);
        // ---- A: wait, sort, fold (block 0) ----------------------------------------------------
        if (blockIdx.x == 0) {
            if (threadIdx.x == 0) {
                int ok = 1;
                if (B.ready) {
                    const uint64_t t0 = global_ns();
                    while (ld_vol(B.ready) == 0) {
                        if (global_ns() - t0 > limit_ns) {
                            atomicOr(S.word + 4, 1u);
                            ok = 0;
                            break;
                        }
                        __nanosleep(64);
                    }
                }
                __threadfence();
                s_flag = ok;
                S.word[5] = 0;
            }
            __syncthreads();
            if (s_flag) {
                // only the inserts and deletes are sorted: reads look their keys up one by one
                constexpr uint32_t PER = PQ_MAX / PQ_THREADS;
                uint32_t mine = 0, bad = 0;
#pragma unroll
                for (uint32_t r = 0; r < PER; r++) {
                    const uint32_t i = threadIdx.x * PER + r;
                    if (i < n) {
                        const uint8_t op = B.ops[i];
                        mine += op == FLIX_OP_INSERT || op == FLIX_OP_DELETE;
                        bad |= op == FLIX_OP_INSERT && keys[i] == KM;
                    }
                }
                uint32_t m;
                uint32_t o = block_scan<uint32_t>(mine, s_sw, m);
#pragma unroll
                for (uint32_t r = 0; r < PER; r++) {
                    const uint32_t i = threadIdx.x * PER + r;
                    if (i < n && (B.ops[i] == FLIX_OP_INSERT || B.ops[i] == FLIX_OP_DELETE)) {
                        s_k[o] = keys[i];
                        s_p[o] = i;
                        o++;
                    }
                }
                uint32_t P2 = 2;
                while (P2 < m) P2 <<= 1;
                for (uint32_t i = m + threadIdx.x; i < P2; i += PQ_THREADS) {
                    s_k[i] = KM;
                    s_p[i] = 0xFFFFFFFFu;
                }
                if (__syncthreads_or(bad) && threadIdx.x == 0) S.word[5] = 1;
                for (uint32_t k = 2; k <= P2; k <<= 1) {
                    for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                        for (uint32_t t = threadIdx.x; t < P2 / 2; t += PQ_THREADS) {
                            const uint32_t a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                            const uint32_t b = a + j;
                            const bool up = (a & k) == 0;
                            const K ka = s_k[a], kb = s_k[b];
                            const uint32_t pa = s_p[a], pb = s_p[b];
                            const bool b_less = kb < ka || (kb == ka && pb < pa);
                            const bool a_less = ka < kb || (ka == kb && pa < pb);
                            if (up ? b_less : a_less) {
                                s_k[a] = kb; s_k[b] = ka;
                                s_p[a] = pb; s_p[b] = pa;
                            }
                        }
                        __syncthreads();
                    }
                }
                // net update of each key's run (submission order: positions ascend in a run)
                uint32_t has[PER];
                K nkv[PER];
                uint32_t nop[PER];
                mine = 0;
#pragma unroll
                for (uint32_t r = 0; r < PER; r++) {
                    const uint32_t i = threadIdx.x * PER + r;
                    has[r] = 0;
                    if (i >= m || (i > 0 && s_k[i - 1] == s_k[i])) continue;
                    bool present = false, deleted = false;
                    K v = K(0);
                    for (uint32_t e = i; e < m && s_k[e] == s_k[i]; e++) {
                        if (B.ops[s_p[e]] == FLIX_OP_INSERT) {
                            if (!present) { present = true; v = aux[s_p[e]]; }
                        } else {
                            present = false;
                            deleted = true;
                        }
                    }
                    has[r] = 1;
                    nop[r] = !present ? EFF_DEL : (deleted ? EFF_UPS : EFF_INS);
                    nkv[r] = v;
                    mine++;
                }
                uint32_t tot;
                o = block_scan<uint32_t>(mine, s_sw, tot);
#pragma unroll
                for (uint32_t r = 0; r < PER; r++) {
                    if (!has[r]) continue;
                    const uint32_t i = threadIdx.x * PER + r;
                    S.ukey[o] = s_k[i];
                    S.uop[o] = nop[r];
                    S.uval[o] = nkv[r];
                    o++;
                }
                if (threadIdx.x == 0) S.word[0] = tot;
            }
        }
        if (!grid_barrier(S.word, limit_ns)) break;
        const uint32_t U = S.word[0];
        // ---- B: snapshot reads, buckets of the net updates -------------------------------------
        for (uint32_t pos = gtid; pos < n; pos += gstride) {
            const uint8_t op = B.ops[pos];
            const K key = keys[pos];
            K rk = KM, rv = KM;
            uint8_t f = 0;
            if (op == FLIX_OP_LOOKUP || op == FLIX_OP_SUCC || op == FLIX_OP_PRED) {
                const uint32_t b = bucket_of(ix, key);
                uint32_t node, sz, nx, prev;
                K bd;
                if (find_node<K, false>(ix, b, key, node, sz, bd, nx, prev)) {
                    const K* nk = ix.keys + (uint64_t)node * NS;
                    uint32_t p;
                    K kp = K(0);
                    if (op == FLIX_OP_PRED) {
                        p = node_upper_bound<K, false>(nk, 0, sz, key);
                        if (p > 0) kp = nk[p - 1];
                    } else {
                        p = node_lower_bound<K, false>(nk, sz, key);
                        if (p < sz) kp = nk[p];
                    }
                    point_result<K, false>(ix, op, key, b, node, sz, nx, prev, p, kp, rk, rv, f);
                }
            }
            if (op != FLIX_OP_RANGE) S.cnt[pos] = 0;       // a range op's count comes from its warp below
            if (B.keys_out) static_cast<K*>(B.keys_out)[pos] = rk;
            if (B.vals_out) static_cast<K*>(B.vals_out)[pos] = rv;
            if (B.found) B.found[pos] = f;
        }
        // range counts, one warp per range op (the pairs follow on the snapshot in phase E1)
        for (uint32_t pos = gtid >> 5; pos < n; pos += gstride >> 5) {
            if (B.ops[pos] != FLIX_OP_RANGE) continue;          // warp-uniform
            const K lo = keys[pos], hi = aux[pos];
            const uint32_t bb = bucket_of(ix, lo);
            uint32_t node, sz, nx, prev;
            K bd;
            uint64_t c = 0;
            uint32_t rn = NIL, rp = 0;
            if (lo <= hi && find_node<K, false>(ix, bb, lo, node, sz, bd, nx, prev)) {
                rn = node;
                rp = node_lower_bound<K, false>(ix.keys + (uint64_t)node * NS, sz, lo);
                c = range_count_warp<K, false>(ix, bb, node, rp, hi);
            }
            if ((threadIdx.x & 31) == 0) {
                S.rb[pos] = bb;
                S.rn[pos] = rn;
                S.rp[pos] = rp;
                S.cnt[pos] = c;
            }
        }
        for (uint32_t u = gtid; u < U; u += gstride) S.ub[u] = bucket_of(ix, S.ukey[u]);
        if (!grid_barrier(S.word, limit_ns)) break;
        // ---- C: node demand per touched bucket; range offsets -----------------------------------
        for (uint32_t u = gtid; u < U; u += gstride) {
            S.need[u] = 0;
            S.freed[u] = 0;
            const uint32_t b = S.ub[u];
            if (u > 0 && S.ub[u - 1] == b) continue;       // not the first net update of its bucket
            uint32_t e = u;
            while (e < U && S.ub[e] == b) e++;
            uint32_t need = 0, emptied = 0, nodes = 0, j = u;
            uint32_t steps = 0;
            for (uint32_t x = ix.head[b]; x != NIL; x = ix.next[x]) {
                if (++steps > ix.cap) { atomicOr(ix.err, ERR_CHAIN); break; }
                nodes++;
                uint32_t k = j;
                while (k < e && S.ukey[k] <= ix.bound[x]) k++;
                if (k == j) continue;
                const uint32_t t = merged_size(ix, x, S.ukey, S.uop, j, k);
                if (t == 0) emptied++;
                else need += n_pieces(t, NS) - 1;
                j = k;
            }
            S.need[u] = need;
            S.freed[u] = emptied - (emptied == nodes && nodes > 0 ? 1u : 0u);
        }
        if (blockIdx.x == 0) {
            constexpr uint32_t PER = PQ_MAX / PQ_THREADS;
            unsigned long long mine = 0;
#pragma unroll
            for (uint32_t r = 0; r < PER; r++) {
                const uint32_t i = threadIdx.x * PER + r;
                if (i < n) mine += S.cnt[i];
            }
            unsigned long long tot;
            unsigned long long o = block_scan<unsigned long long>(mine, s_sw64, tot);
#pragma unroll
            for (uint32_t r = 0; r < PER; r++) {
                const uint32_t i = threadIdx.x * PER + r;
                if (i < n) {
                    if (B.range_off) B.range_off[i] = o;
                    o += S.cnt[i];
                }
            }
            if (threadIdx.x == 0) {
                if (B.range_off) B.range_off[n] = tot;
                S.wide[1] = tot;
            }
        }
        if (!grid_barrier(S.word, limit_ns)) break;
        // ---- D: admission (block 0) --------------------------------------------------------------
        if (blockIdx.x == 0) {
            constexpr uint32_t PER = PQ_MAX / PQ_THREADS;
            uint32_t mn = 0, mf = 0;
#pragma unroll
            for (uint32_t r = 0; r < PER; r++) {
                const uint32_t u = threadIdx.x * PER + r;
                if (u < U) { mn += S.need[u]; mf += S.freed[u]; }
            }
            uint32_t tn, tf;
            uint32_t on = block_scan<uint32_t>(mn, s_sw, tn);
            uint32_t of = block_scan<uint32_t>(mf, s_sw, tf);
#pragma unroll
            for (uint32_t r = 0; r < PER; r++) {
                const uint32_t u = threadIdx.x * PER + r;
                if (u < U) {
                    S.aoff[u] = on;
                    S.foff[u] = of;
                    on += S.need[u];
                    of += S.freed[u];
                }
            }
            const unsigned long long top = ds->free_top;
            uint64_t flags = 0;
            if (S.word[5]) flags |= ST_BADKEY;
            if (tn > top) flags |= ST_NODES;
            if (S.wide[1] > B.range_cap) flags |= ST_RANGE;
            const bool ok = flags == 0;
            for (uint32_t i = threadIdx.x; ok && i < tn; i += PQ_THREADS) S.pop[i] = free_ids[top - tn + i];
            if (threadIdx.x == 0) {
                S.word[1] = ok;
                S.word[2] = tn;
                S.word[3] = tf;
                S.wide[0] = top;
                if (flags_or && flags) atomicOr(flags_or, (unsigned long long)flags);
                if (B.status) {
                    B.status[0] = flags;
                    B.status[1] = S.wide[1];
                    B.status[2] = tn;
                    B.status[3] = top;
                }
            }
        }
        if (!grid_barrier(S.word, limit_ns)) break;
        const bool admitted = S.word[1] != 0;
        // ---- E1: range pairs on the pre-batch state, one warp per range op --------------------
        if (admitted) {
            const uint32_t gw = gtid >> 5, nwarps = gstride >> 5;
            for (uint32_t pos = gw; pos < n; pos += nwarps) {
                if (B.ops[pos] != FLIX_OP_RANGE) continue;      // warp-uniform: pos is the warp's
                const uint64_t c = S.cnt[pos];
                if (c == 0) continue;
                range_fill_warp<K, false, 4>(ix, (uint64_t)S.rb[pos], S.rn[pos], S.rp[pos], B.range_off[pos], c,
                                          static_cast<K*>(B.range_keys), static_cast<K*>(B.range_vals));
            }
        }
        if (!grid_barrier(S.word, limit_ns)) break;
        // ---- E2: per touched bucket: merge, split, compact, relink, reclaim ----------------------
        if (admitted) {
            const uint64_t fbase = S.wide[0] - S.word[2];      // first slot of the popped ids
            for (uint32_t u = gtid; u < U; u += gstride) {
                const uint32_t b = S.ub[u];
                if (u > 0 && S.ub[u - 1] == b) continue;
                uint32_t e = u;
                while (e < U && S.ub[e] == b) e++;
                K* mk = S.mk + (uint64_t)u * (NS + 1);
                K* mv = S.mv + (uint64_t)u * (NS + 1);
                uint32_t na = S.aoff[u], nf = S.foff[u];
                uint32_t tail = NIL, held = NIL, j = u;
                bool last_dropped = false;
                const uint32_t head0 = ix.head[b];
                uint32_t steps = 0;
                for (uint32_t x = head0; x != NIL;) {
                    if (++steps > ix.cap) { atomicOr(ix.err, ERR_CHAIN); break; }
                    const uint32_t nx = ix.next[x];
                    const K obound = ix.bound[x];
                    uint32_t k = j;
                    while (k < e && S.ukey[k] <= obound) k++;
                    uint32_t last = x;      // the last node this node became
                    if (k > j) {
                        // merge the node's pairs with its net updates into mk/mv
                        const K* nk = ix.keys + (uint64_t)x * NS;
                        const K* nv = ix.vals + (uint64_t)x * NS;
                        const uint32_t sz = ix.size[x];
                        uint32_t a = 0, c = j, t = 0;
                        // the node's pairs come in chunks of PQ_CHUNK, every load of a chunk issued
                        // before the merge uses it (the merge's stores could alias the loads, so
                        // one pair at a time would wait for each load)
                        K kb[PQ_CHUNK], vb[PQ_CHUNK];
                        uint32_t a0 = 0;
                        bool have = false;
                        while (a < sz || c < k) {
                            if (a < sz && (!have || a - a0 >= (uint32_t)PQ_CHUNK)) {
                                a0 = a;
                                have = true;
#pragma unroll
                                for (int i = 0; i < PQ_CHUNK; i++)
                                    if (a0 + i < sz) { kb[i] = nk[a0 + i]; vb[i] = nv[a0 + i]; }
                            }
                            const K ka = a < sz ? kb[a - a0] : K(0);
                            if (c >= k || (a < sz && ka < S.ukey[c])) {
                                mk[t] = ka; mv[t] = vb[a - a0]; t++; a++;
                            } else if (a < sz && ka == S.ukey[c]) {
                                if (S.uop[c] == EFF_UPS) { mk[t] = ka; mv[t] = S.uval[c]; t++; }
                                else if (S.uop[c] == EFF_INS) { mk[t] = ka; mv[t] = vb[a - a0]; t++; }
                                a++; c++;
                            } else {
                                if (S.uop[c] != EFF_DEL) { mk[t] = S.ukey[c]; mv[t] = S.uval[c]; t++; }
                                c++;
                            }
                        }
                        j = k;
                        if (t == 0) {
                            // emptied: leaves the chain; the chain's first node is held back in
                            // case the whole chain empties
                            if (x == head0 && tail == NIL) held = x;
                            else free_ids[fbase + nf++] = x;
                            last_dropped = nx == NIL;
                            x = nx;
                            continue;
                        }
                        const uint32_t qn = n_pieces(t, NS);
                        uint32_t node = x, o = 0;
                        for (uint32_t r = 0; r < qn; r++) {
                            if (r > 0) {
                                const uint32_t nn = S.pop[na++];
                                ix.next[node] = nn;
                                node = nn;
                            }
                            const uint32_t ps = piece_size(t, NS, qn, r);
                            // the merged run goes out in chunks: its loads first, then its stores
                            for (uint32_t s0 = 0; s0 < ps; s0 += PQ_CHUNK) {
                                K ck[PQ_CHUNK], cv[PQ_CHUNK];
#pragma unroll
                                for (int i = 0; i < PQ_CHUNK; i++)
                                    if (s0 + i < ps) { ck[i] = mk[o + s0 + i]; cv[i] = mv[o + s0 + i]; }
#pragma unroll
                                for (int i = 0; i < PQ_CHUNK; i++)
                                    if (s0 + i < ps) {
                                        ix.keys[(uint64_t)node * NS + s0 + i] = ck[i];
                                        ix.vals[(uint64_t)node * NS + s0 + i] = cv[i];
                                    }
                            }
                            o += ps;
                            ix.size[node] = ps;
                            ix.bound[node] = r + 1 < qn ? mk[o - 1] : obound;
                        }
                        ix.next[node] = nx;
                        last = node;
                    }
                    // x (or its pieces x..last) stays: link it behind the kept chain
                    if (tail == NIL) {
                        ix.head[b] = x;
                        if (held != NIL) {
                            free_ids[fbase + nf++] = held;
                            held = NIL;
                        }
                    } else {
                        ix.next[tail] = x;
                    }
                    tail = last;
                    last_dropped = false;
                    x = nx;
                }
                if (tail == NIL) {
                    // the whole chain emptied: its first node stays as the bucket's only, empty node
                    ix.size[held] = 0;
                    ix.bound[held] = ix.mkba[b];
                    ix.next[held] = NIL;
                    ix.head[b] = held;
                } else {
                    ix.next[tail] = NIL;
                    if (last_dropped) ix.bound[tail] = ix.mkba[b];   // maxBucket passes to the new last node
                }
            }
        }
        if (!grid_barrier(S.word, limit_ns)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            if (admitted) ds->free_top = S.wide[0] - S.word[2] + S.word[3];
            ds->applied = admitted;
            ds->admitted = 0;
        }
    }
    // batches the queue did not run (a wait gave up)
    if (bi < count && blockIdx.x == 0 && threadIdx.x == 0) {
        atomicOr(ix.err, ERR_TIMEOUT);
        for (uint32_t r = bi; r < count; r++)
            if (q[r].status) q[r].status[0] = PQ_NOT_RUN;
        if (flags_or) atomicOr(flags_or, (unsigned long long)PQ_NOT_RUN);
    }
}

}  // namespace

void preload_persist_kernels()
{
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_queue<uint32_t>);
    cudaFuncGetAttributes(&a, k_queue<uint64_t>);
}

template <class K>
int apply_queue(flix_index* h, const flix_batch* hb, uint32_t count, uint32_t wait_us, uint64_t* d_flags_or,
                cudaStream_t st)
{
    if (count == 0) return FLIX_OK;
    if (h->cfg.merge_underfull || h->cfg.split_chains_over) return FLIX_ENOTIMPL;
    for (uint32_t i = 0; i < count; i++)
        if (hb[i].n > PQ_MAX || (hb[i].n && (!hb[i].ops || !hb[i].keys || !hb[i].aux))) return FLIX_EINVAL;
    const uint32_t NS = h->NS;
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t ks = sizeof(K);
    const size_t need = al(count * sizeof(PQBatch)) + al(PQ_MAX * ks) * 3 + al(PQ_MAX * 4) * 11 + al(PQ_MAX * 8) +
                        al((2 * PQ_MAX + 16) * 4) + al(((size_t)PQ_MAX * (NS + 1) + NS) * ks) * 2 + al(64 * 4) +
                        al(4 * 8) + (1 << 12);
    cudaError_t e = h->arena.ensure(need);
    if (e) { h->last_error = cudaGetErrorString(e); return FLIX_ECUDA; }
    h->arena.reset();
    Arena& A = h->arena;
    PQBatch* dq = A.take<PQBatch>(count);
    PQScratch<K> S;
    S.cnt = A.take<uint64_t>(PQ_MAX);
    S.rb = A.take<uint32_t>(PQ_MAX);
    S.rn = A.take<uint32_t>(PQ_MAX);
    S.rp = A.take<uint32_t>(PQ_MAX);
    S.ukey = A.take<K>(PQ_MAX);
    S.uop = A.take<uint32_t>(PQ_MAX);
    S.uval = A.take<K>(PQ_MAX);
    S.ub = A.take<uint32_t>(PQ_MAX);
    S.need = A.take<uint32_t>(PQ_MAX);
    S.freed = A.take<uint32_t>(PQ_MAX);
    S.aoff = A.take<uint32_t>(PQ_MAX);
    S.foff = A.take<uint32_t>(PQ_MAX);
    S.pop = A.take<uint32_t>(2 * PQ_MAX + 16);
    S.mk = A.take<K>((size_t)PQ_MAX * (NS + 1) + NS);
    S.mv = A.take<K>((size_t)PQ_MAX * (NS + 1) + NS);
    S.word = A.take<uint32_t>(64);
    S.wide = A.take<unsigned long long>(4);
    if (!dq || !S.wide) return FLIX_ENOMEM;
    // descriptors: through the handle's pinned staging buffer (the previous copy out of it is done)
    const size_t qbytes = count * sizeof(PQBatch);
    if (h->qstage_bytes < qbytes) {
        if (h->qstage) {
            cudaEventSynchronize(h->qstage_ev);
            cudaFreeHost(h->qstage);
            h->qstage = nullptr;
        }
        if ((e = cudaHostAlloc(&h->qstage, qbytes, cudaHostAllocDefault))) {
            h->qstage_bytes = 0;
            h->last_error = cudaGetErrorString(e);
            return FLIX_ECUDA;
        }
        h->qstage_bytes = qbytes;
    } else {
        cudaEventSynchronize(h->qstage_ev);
    }
    PQBatch* hq = static_cast<PQBatch*>(h->qstage);
    for (uint32_t i = 0; i < count; i++) {
        PQBatch b;
        b.ops = hb[i].ops;
        b.keys = hb[i].keys;
        b.aux = hb[i].aux;
        b.n = hb[i].n;
        b.keys_out = hb[i].keys_out;
        b.vals_out = hb[i].vals_out;
        b.found = hb[i].found;
        b.range_off = hb[i].range_off;
        b.range_keys = hb[i].range_keys;
        b.range_vals = hb[i].range_vals;
        b.range_cap = hb[i].range_cap;
        b.status = hb[i].status;
        b.ready = hb[i].ready;
        hq[i] = b;
    }
    if ((e = cudaMemcpyAsync(dq, hq, qbytes, cudaMemcpyHostToDevice, st)) || (e = cudaEventRecord(h->qstage_ev, st))) {
        h->last_error = cudaGetErrorString(e);
        return FLIX_ECUDA;
    }
    Ctx c{h, st};
    if ((e = fill_bytes(c, S.word, 0, 64 * 4))) { h->last_error = cudaGetErrorString(e); return FLIX_ECUDA; }
    int per_sm = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_queue<K>, PQ_THREADS, 0)) || per_sm < 1) {
        h->last_error = e ? cudaGetErrorString(e) : "queue kernel does not fit an SM";
        return FLIX_ECUDA;
    }
    // one block per SM: a batch of at most PQ_MAX ops has far fewer threads of work than that
    const uint32_t grid = (uint32_t)h->nsm;
    DevIdx<K> ix = dev_view<K>(h);
    const PQBatch* dqc = dq;
    uint64_t limit_ns = (uint64_t)wait_us * 1000ull;
    DevState* ds = h->dstate;
    uint32_t* fid = h->free_ids;
    unsigned long long* fo = reinterpret_cast<unsigned long long*>(d_flags_or);
    void* args[] = {&ix, &dqc, &count, &S, &ds, &fid, &limit_ns, &fo};
    cudaEvent_t pa = nullptr, pb = nullptr;
    if (h->prof_on) {
        pa = prof_event(h);
        pb = prof_event(h);
        cudaEventRecord(pa, st);
    }
    e = cudaLaunchCooperativeKernel((const void*)k_queue<K>, dim3(grid), dim3(PQ_THREADS), args, 0, st);
    if (h->prof_on) {
        cudaEventRecord(pb, st);
        h->prof.push_back(ProfRec{K_QUEUE, 0.0, pa, pb});
    }
    h->launches++;
    if (e) { h->last_error = cudaGetErrorString(e); return FLIX_ECUDA; }
    return FLIX_OK;
}

template int apply_queue<uint32_t>(flix_index*, const flix_batch*, uint32_t, uint32_t, uint64_t*, cudaStream_t);
template int apply_queue<uint64_t>(flix_index*, const flix_batch*, uint32_t, uint32_t, uint64_t*, cudaStream_t);

}  // namespace flix
