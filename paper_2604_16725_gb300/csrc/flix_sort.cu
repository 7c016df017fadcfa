// Batch sort (Sec. 3.3: each batch is sorted by key before buckets pull their operations; Tab. 1
// times it) and prefix-sum primitives.
//
// The sort is a stable least-significant-digit radix sort of (key, position) pairs with 8-bit
// digits.  One read of the keys builds the digit histograms of every digit position, and a plan
// kernel picks the passes from them on the device: digits that are the same in every key are
// skipped, and when the highest few varying digits already split the batch into groups of at most
// one item on average, only those are sorted and a finish kernel sorts each group of equal prefix
// in place (for 2^24 uniform 64-bit keys: 3 passes instead of 8).  Each pass is one scatter kernel
// over 4096-item tiles (512 threads x 8 items, two blocks per SM): a tile ranks its items in
// shared memory (peers of a digit from 8 warp ballots, one per digit bit; stable: warp-striped
// items ranked in warp, item, lane order), learns where each digit's run of this tile starts in
// the output, and writes the locally sorted tile so that each digit's run is a contiguous store.
// The start of each (digit, tile) run comes either from
//   - one-sweep (after the single-pass "Onesweep" radix sort of Adinets and Merrill, 2022): every
//     tile publishes its per-digit counts and looks back through the published states of earlier
//     tiles (an aggregate, or an inclusive prefix that ends the walk), reading 8 earlier tiles per
//     round trip; tiles take their index from an atomic counter in start order, so each tile
//     waited on has already started, and every wait is bounded (a wait that runs out sets an
//     error bit); or
//   - reduce-then-scan: an upsweep kernel counts each tile's digits, a scan kernel turns the counts
//     into run starts, and the scatter reads them.
// Both give the same (stable) order; the one-sweep variant saves one read of the keys per pass.
#include <algorithm>

#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int NWARPS = 8;   // warps of the 256-thread helper kernels
constexpr int RADIX = 256;

constexpr int OS_THREADS = 512;
constexpr int OS_ITEMS = 8;
constexpr int OS_TILE = OS_THREADS * OS_ITEMS;
constexpr int OS_WARPS = OS_THREADS / 32;
constexpr int UP_THREADS_S = 256;
constexpr int UP_ITEMS = OS_TILE / UP_THREADS_S;
constexpr uint32_t ST_AGG = 1u << 30;
constexpr uint32_t ST_INC = 2u << 30;
constexpr uint32_t ST_COUNT = (1u << 30) - 1;
constexpr uint32_t LOOKBACK_SPIN_LIMIT = 1u << 22;
constexpr int LOOKBACK_WINDOW = 8;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Exclusive scan of one value per thread over a block of NW warps; `total` gets the block sum.
// sw must hold NW entries; the function ends with a barrier so sw can be reused.
template <class T, int NW = NWARPS>
__device__ __forceinline__ T block_excl_scan(T v, T* sw, T& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (w == 0) {
        T t = lane < NW ? sw[lane] : T(0);
#pragma unroll
        for (int o = 1; o < NW; o <<= 1) {
            T y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NW) sw[lane] = t;
    }
    __syncthreads();
    T wbase = w ? sw[w - 1] : T(0);
    total = sw[NW - 1];
    __syncthreads();
    return wbase + x - v;
}

template <class K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) { return static_cast<uint32_t>(k >> shift) & 255u; }

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }
__device__ __forceinline__ void st_volatile(uint32_t* p, uint32_t v) { *reinterpret_cast<volatile uint32_t*>(p) = v; }

// Stable rank of each lane's item among the warp's lanes with the same digit: the peer mask is
// built from NB ballots, one per digit bit (NB = 9 when the digit value RADIX marks a lane
// without an item).
template <int NB>
__device__ __forceinline__ uint32_t digit_peers(uint32_t d)
{
    uint32_t peers = FULL;
#pragma unroll
    for (int b = 0; b < NB; b++) {
        const uint32_t bit = (d >> b) & 1u;
        const uint32_t m = __ballot_sync(FULL, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

// Ranks the warp's OS_ITEMS x 32 items (item i of lane l is the warp's (i * 32 + l)-th) by digit:
// rank[i] = items of the same digit earlier in the warp; wh[d] ends as the warp's count of digit d.
// FULLT: every item is valid (no bounds test, 8 ballots).
template <class K, bool FULLT>
__device__ __forceinline__ void rank_warp(const K (&key)[OS_ITEMS], uint32_t (&rank)[OS_ITEMS], uint16_t* wh,
                                          uint64_t wbase, uint64_t n, int shift)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < OS_ITEMS; i++) {
        const uint32_t d = (FULLT || wbase + (uint64_t)i * 32 + lane < n) ? digit_of(key[i], shift) : RADIX;
        const uint32_t peers = digit_peers<FULLT ? 8 : 9>(d);
        const uint32_t leader = __ffs(peers) - 1;
        const bool lead = lane == leader && (FULLT || d < RADIX);
        uint32_t prior = 0;
        if (lead) prior = wh[d];
        prior = __shfl_sync(FULL, prior, leader);
        rank[i] = prior + __popc(peers & lt);
        if (lead) wh[d] = static_cast<uint16_t>(prior + __popc(peers));
        __syncwarp();
    }
}

// Where pass `pass` of a plan with np passes reads and writes: passes alternate between the output
// pair and the scratch pair so that the last one writes the output; the first reads the input with
// payload = position.
template <class K>
struct PassBufs {
    const K* kin;
    const uint32_t* vin;
    K* kout;
    uint32_t* vout;
};
template <class K>
__device__ __forceinline__ PassBufs<K> pass_bufs(int pass, uint32_t np, const K* kin, K* kout, uint32_t* vout, K* tk,
                                                 uint32_t* tv)
{
    const bool to_out = ((np - 1 - (uint32_t)pass) & 1u) == 0;
    PassBufs<K> b;
    b.kout = to_out ? kout : tk;
    b.vout = to_out ? vout : tv;
    b.kin = pass == 0 ? kin : (to_out ? tk : kout);
    b.vin = pass == 0 ? nullptr : (to_out ? tv : vout);
    return b;
}

// Reduce-then-scan: per-tile digit counts of one pass, counts[d * T + tile].
template <class K>
__global__ void __launch_bounds__(UP_THREADS_S) k_upsweep(const K* kin, K* kout, uint32_t* vout, K* tk, uint32_t* tv,
                                                          uint64_t n, int pass, const SortPlan* __restrict__ plan,
                                                          uint32_t* __restrict__ counts, uint32_t T)
{
    grid_dep_enter();
    const uint32_t np = plan->npass;
    if ((uint32_t)pass >= np) return;
    const int shift = plan->shift[pass];
    const K* keys = pass_bufs<K>(pass, np, kin, kout, vout, tk, tv).kin;
    __shared__ uint32_t sh[RADIX];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * OS_TILE;
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll 4
    for (int i = 0; i < UP_ITEMS; i++) {
        const uint64_t pos = base + (uint64_t)i * UP_THREADS_S + threadIdx.x;
        const uint32_t d = pos < n ? digit_of(keys[pos], shift) : RADIX;
        const uint32_t peers = digit_peers<9>(d);
        if (d < RADIX && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * T + blockIdx.x] = sh[threadIdx.x];
}

// Reduce-then-scan: offsets[d * T + t] = bases[d] + (items of digit d in tiles < t).
__global__ void __launch_bounds__(256) k_scan_digits(const uint32_t* __restrict__ counts, uint32_t T, int pass,
                                                    const SortPlan* __restrict__ plan,
                                                    const uint32_t* __restrict__ bases, uint32_t* __restrict__ offsets)
{
    grid_dep_enter();
    if ((uint32_t)pass >= plan->npass) return;
    __shared__ uint32_t sw[NWARPS];
    const uint32_t d = blockIdx.x;
    uint32_t carry = bases[(plan->shift[pass] >> 3) * RADIX + d];
    for (uint32_t t0 = 0; t0 < T; t0 += 256) {
        const uint32_t t = t0 + threadIdx.x;
        const uint32_t c = t < T ? counts[(uint64_t)d * T + t] : 0u;
        uint32_t tot;
        const uint32_t ex = block_excl_scan<uint32_t>(c, sw, tot);
        if (t < T) offsets[(uint64_t)d * T + t] = carry + ex;
        carry += tot;
    }
}

// One digit pass of the plan (np passes in all).  LOOKBACK selects one-sweep (status, tile_ctr) or
// reduce-then-scan (offsets).  PERSIST (one-sweep only): the grid is one wave of blocks that take
// tiles from the counter until none is left.
template <class K, bool LOOKBACK, bool PERSIST>
__device__ __forceinline__ void sweep_pass(const K* kin, K* kout, uint32_t* vout, K* tk, uint32_t* tv, uint64_t n,
                                           int pass, uint32_t np, const SortPlan* __restrict__ plan,
                                           const uint32_t* __restrict__ bases, const uint32_t* __restrict__ offsets,
                                           uint32_t T, uint32_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
                                           uint32_t* __restrict__ err)
{
    const int shift = plan->shift[pass];
    const PassBufs<K> io = pass_bufs<K>(pass, np, kin, kout, vout, tk, tv);
    bases += (shift >> 3) * RADIX;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + OS_TILE);
    uint16_t* whist = reinterpret_cast<uint16_t*>(sv + OS_TILE);                // [OS_WARPS][RADIX]
    uint32_t* goff = reinterpret_cast<uint32_t*>(whist + OS_WARPS * RADIX);     // [RADIX]
    uint32_t* sw = goff + RADIX;                                                // [OS_WARPS]
    uint32_t* s_tile = sw + OS_WARPS;

    for (;;) {
        if (LOOKBACK && threadIdx.x == 0) *s_tile = atomicAdd(tile_ctr, 1u);
        for (int i = threadIdx.x; i < OS_WARPS * RADIX / 2; i += OS_THREADS) reinterpret_cast<uint32_t*>(whist)[i] = 0;
        __syncthreads();
        const uint32_t tile = LOOKBACK ? *s_tile : blockIdx.x;
        if (PERSIST && tile >= T) break;
        const uint64_t base = (uint64_t)tile * OS_TILE;
        const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const bool full_tile = base + OS_TILE <= n;

        K key[OS_ITEMS];
        uint32_t val[OS_ITEMS];
        uint32_t rank[OS_ITEMS];
        const uint64_t wbase = base + (uint64_t)warp * 32 * OS_ITEMS;
#pragma unroll
        for (int i = 0; i < OS_ITEMS; i++) {
            const uint64_t pos = wbase + (uint64_t)i * 32 + lane;
            const bool ok = full_tile || pos < n;
            // the tail kernel reads what other blocks wrote in its previous pass: past L1
            key[i] = ok ? (PERSIST ? __ldcg(io.kin + pos) : io.kin[pos]) : K(0);
            val[i] = ok ? (io.vin ? (PERSIST ? __ldcg(io.vin + pos) : io.vin[pos]) : static_cast<uint32_t>(pos)) : 0u;
        }
        if (full_tile) rank_warp<K, true>(key, rank, whist + warp * RADIX, wbase, n, shift);
        else rank_warp<K, false>(key, rank, whist + warp * RADIX, wbase, n, shift);
        __syncthreads();
        uint32_t cnt = 0;
        if (threadIdx.x < RADIX) {
            const uint32_t d = threadIdx.x;
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < OS_WARPS; w++) {
                const uint32_t c = whist[w * RADIX + d];
                whist[w * RADIX + d] = (uint16_t)run;
                run += c;
            }
            cnt = run;
            // publish this tile's count early so that later tiles can pass over it
            if (LOOKBACK) st_volatile(status + (uint64_t)tile * RADIX + d, (tile == 0 ? ST_INC : ST_AGG) | cnt);
        }
        uint32_t tot;
        const uint32_t start = block_excl_scan<uint32_t, OS_WARPS>(cnt, sw, tot);
        if (threadIdx.x < RADIX) {
            const uint32_t d = threadIdx.x;
            // per (warp, digit): tile-local start of the warp's run of digit d
#pragma unroll
            for (int w = 0; w < OS_WARPS; w++) whist[w * RADIX + d] = (uint16_t)(whist[w * RADIX + d] + start);
            uint32_t gstart;
            if (LOOKBACK) {
                uint32_t excl = 0;
                int64_t t = (int64_t)tile - 1;
                uint32_t spins = 0;
                while (t >= 0) {
                    uint32_t v[LOOKBACK_WINDOW];
#pragma unroll
                    for (int q = 0; q < LOOKBACK_WINDOW; q++)
                        v[q] = (t - q >= 0) ? ld_volatile(status + (uint64_t)(t - q) * RADIX + d) : ST_INC;
                    bool done = false;
                    int q = 0;
                    for (; q < LOOKBACK_WINDOW; q++) {
                        if ((v[q] & ~ST_COUNT) == 0) break;   // not published yet: resume there
                        excl += v[q] & ST_COUNT;
                        if (v[q] & ST_INC) { done = true; break; }
                    }
                    if (done) break;
                    t -= q;
                    if (q < LOOKBACK_WINDOW && ++spins > LOOKBACK_SPIN_LIMIT) {
                        atomicOr(err, ERR_SPIN);
                        break;
                    }
                }
                if (tile != 0) st_volatile(status + (uint64_t)tile * RADIX + d, ST_INC | (excl + cnt));
                gstart = bases[d] + excl;
            } else {
                gstart = offsets[(uint64_t)d * T + tile];
            }
            // output position of tile-local sorted slot j of digit d is goff[d] + j (mod 2^32)
            goff[d] = gstart - start;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < OS_ITEMS; i++) {
            const uint64_t pos = wbase + (uint64_t)i * 32 + lane;
            if (full_tile || pos < n) {
                const uint32_t d = digit_of(key[i], shift);
                const uint32_t r = whist[warp * RADIX + d] + rank[i];
                sk[r] = key[i];
                sv[r] = val[i];
            }
        }
        __syncthreads();
        const uint32_t tile_n = (uint32_t)((n - base) < (uint64_t)OS_TILE ? (n - base) : OS_TILE);
        for (uint32_t j = threadIdx.x; j < tile_n; j += OS_THREADS) {
            const K k = sk[j];
            const uint32_t o = goff[digit_of(k, shift)] + j;
            io.kout[o] = k;
            io.vout[o] = sv[j];
        }
        if (!PERSIST) break;
        __syncthreads();   // the tile's shared memory is reused by the next one
    }
}

// One digit pass as its own launch; a pass beyond the plan's count returns at once.
template <class K, bool LOOKBACK>
__global__ void __launch_bounds__(OS_THREADS, 2) k_sweep(const K* kin, K* kout, uint32_t* vout, K* tk, uint32_t* tv,
                                                         uint64_t n, int pass, const SortPlan* __restrict__ plan,
                                                         const uint32_t* __restrict__ bases,
                                                         const uint32_t* __restrict__ offsets, uint32_t T,
                                                         uint32_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
                                                         uint32_t* __restrict__ err)
{
    grid_dep_enter();
    const uint32_t np = plan->npass;
    if ((uint32_t)pass >= np) return;
    sweep_pass<K, LOOKBACK, false>(kin, kout, vout, tk, tv, n, pass, np, plan, bases, offsets, T, status, tile_ctr,
                                   err);
}

// Every pass from p0 on that the plan takes, in one cooperative launch of one wave of blocks: each
// pass takes tiles from its own counter, and a grid barrier separates the passes.  The plan takes
// these passes only for dense or skewed keys, so the usual launch reads the pass count and returns;
// as separate launches each of them would cost a launch of its own.  The barrier counts arrivals
// in bar[0] (zero at the sort's start: barrier j waits for j * gridDim.x arrivals); a wait past
// about a second sets ERR_SPIN and the block returns, and blocks that see the bit stop waiting.
template <class K>
__global__ void __launch_bounds__(OS_THREADS, 2) k_sweep_tail(const K* kin, K* kout, uint32_t* vout, K* tk,
                                                              uint32_t* tv, uint64_t n, int p0,
                                                              const SortPlan* __restrict__ plan,
                                                              const uint32_t* __restrict__ bases, uint32_t T,
                                                              uint32_t* __restrict__ status,
                                                              uint32_t* __restrict__ tile_ctr, uint32_t* bar,
                                                              uint32_t* __restrict__ err)
{
    grid_dep_enter();
    const uint32_t np = plan->npass;
    __shared__ int s_stop;
    for (int p = p0; (uint32_t)p < np && p < (int)sizeof(K); p++) {
        sweep_pass<K, true, true>(kin, kout, vout, tk, tv, n, p, np, plan, bases, nullptr, T,
                                  status + (size_t)p * T * RADIX, tile_ctr + p, err);
        if ((uint32_t)p + 1 >= np) break;
        // grid barrier: every tile of pass p is written before any block reads for pass p + 1
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            const uint32_t target = (uint32_t)(p - p0 + 1) * gridDim.x;
            atomicAdd(bar, 1u);
            int stop = 0;
            uint64_t t0;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
            while (ld_volatile(bar) < target) {
                if (ld_volatile(err) & ERR_SPIN) { stop = 1; break; }
                uint64_t t1;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
                if (t1 - t0 > 1000000000ull) {
                    atomicOr(err, ERR_SPIN);
                    stop = 1;
                    break;
                }
                __nanosleep(100);
            }
            __threadfence();
            s_stop = stop;
        }
        __syncthreads();
        if (s_stop) return;
    }
}

template <class K>
size_t sweep_smem()
{
    return (size_t)OS_TILE * (sizeof(K) + 4) + (size_t)OS_WARPS * RADIX * 2 + (RADIX + OS_WARPS + 4) * 4;
}

// ---- pass plan -----------------------------------------------------------------------------------
//
// A digit whose histogram has one bin holding every item is the same in every key and orders
// nothing.  Of the others, the plan sorts by all of them (LSD order), unless a prefix of the
// highest h of them already splits the batch into groups of n / 2^(8h) <= 1 item on average;
// then it sorts by that prefix only and leaves the groups of equal prefix to the finish kernels
// (one pass costs more than finishing the groups a digit fewer leaves: at 2^24 uniform keys, 3
// passes and a finish that moves the 63% of items sharing their prefix beat 4 passes and a finish
// that moves 0.4%).  A digit whose fullest bin holds more than 4x its uniform share (n/64 + 256 items) is
// heavy; when every prefix digit is heavy, groups may be long (heavy keys) and the plan sorts by
// every digit.  A skew confined to some prefix digits (a dense key range) keeps the prefix plan,
// because the largest group is bounded by the lightest prefix digit's fullest bin.  In place, hist
// rows become the digit bases (items with a smaller digit) of every digit position.
template <class K>
__global__ void __launch_bounds__(RADIX) k_sort_plan(uint32_t* __restrict__ hist, uint64_t n, uint32_t h,
                                                      SortPlan* __restrict__ plan)
{
    grid_dep_enter();
    constexpr int P = sizeof(K);
    __shared__ uint32_t s_const[P], s_max[P];
    __shared__ float s_p2[P];
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    static_assert(P <= RADIX / 32, "one warp per digit position");
    // one warp per digit position: lane l holds bins 8l..8l+7
    if (warp < (uint32_t)P) {
        uint32_t* hp = hist + (size_t)warp * RADIX + lane * 8;
        uint32_t c[8], m = 0, run = 0;
        float q = 0.0f;
        bool one = false;
#pragma unroll
        for (int t = 0; t < 8; t++) {
            c[t] = hp[t];
            one |= (uint64_t)c[t] == n;
            m = max(m, c[t]);
            q += (float)c[t] * (float)c[t];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            m = max(m, __shfl_xor_sync(FULL, m, o));
            q += __shfl_xor_sync(FULL, q, o);
        }
        const bool all_one_bin = __any_sync(FULL, one);
        // exclusive scan of the 256 bins: within the lane, then over the lanes
#pragma unroll
        for (int t = 0; t < 8; t++) { const uint32_t x = c[t]; c[t] = run; run += x; }
        uint32_t x = run;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(FULL, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        const uint32_t before = x - run;
#pragma unroll
        for (int t = 0; t < 8; t++) hp[t] = before + c[t];
        if (lane == 0) {
            s_max[warp] = m;
            s_const[warp] = all_one_bin;
            s_p2[warp] = q / ((float)n * (float)n);   // chance that two items share this digit
        }
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    int nc[P];
    int m = 0;
    for (int p = P - 1; p >= 0; p--)
        if (!s_const[p]) nc[m++] = p;   // non-constant digits, most significant first
    SortPlan pl;
    pl.finish = 0;
    pl.pmask = ~0ull;
    pl.nbig = 0;
    pl.cursor = 0;
    for (int q = 0; q < 8; q++) pl.shift[q] = 0;
    if (m == 0) {          // every key equal: one stable pass copies the batch to the output
        pl.npass = 1;
    } else {
        int use = m;
        // prefix digits: at least h, and enough that the other items expected in a random item's
        // group, n times the chance that two items share every prefix digit (digits taken as
        // independent), stay at most 2 (uniform keys at h give about 1); dense or skewed keys
        // need more digits than uniform ones
        int hh = 0;
        float e = (float)n;
        while (hh < m) {
            e *= s_p2[nc[hh]];
            hh++;
            if (hh >= (int)h && e <= 2.0f) break;
        }
        if (hh < m) {
            // a group of g keys with one prefix puts g keys into one bin of every prefix digit, so
            // the largest group is at most the smallest largest-bin over the prefix digits: one
            // prefix digit without a heavy bin bounds every group the finish meets
            bool heavy = true;
            for (int q = 0; q < hh; q++) heavy &= (uint64_t)s_max[nc[q]] > n / 64 + 256;
            if (!heavy) {
                use = hh;
                pl.finish = 1;
                pl.pmask = ~0ull << (8 * nc[use - 1]);
            }
        }
        pl.npass = (uint32_t)use;
        for (int q = 0; q < use; q++) pl.shift[q] = 8 * nc[use - 1 - q];
    }
    *plan = pl;
}

// Digit histograms of every pass from one read of the keys.
template <class K>
__global__ void __launch_bounds__(256) k_hist_all(const K* __restrict__ keys, uint64_t n, uint32_t* __restrict__ hist)
{
    grid_dep_enter();
    constexpr int P = sizeof(K);
    __shared__ uint32_t sh[P * RADIX];
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // four keys in flight per thread: their loads are issued before any of the counts
    for (; i + 3 * stride < n; i += 4 * stride) {
        K k[4];
#pragma unroll
        for (int u = 0; u < 4; u++) k[u] = keys[i + u * stride];
#pragma unroll
        for (int u = 0; u < 4; u++)
#pragma unroll
            for (int p = 0; p < P; p++) atomicAdd(&sh[p * RADIX + digit_of(k[u], 8 * p)], 1u);
    }
    for (; i < n; i += stride) {
        const K k = keys[i];
#pragma unroll
        for (int p = 0; p < P; p++) atomicAdd(&sh[p * RADIX + digit_of(k, 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// ---- finishing the groups of equal prefix ----------------------------------------------------------
//
// After the prefix passes the batch is ordered by prefix, and inside a group of equal prefix by
// position (the passes are stable).  The payload is the item's position in the input, so the
// order the sort must produce is (key, payload) ascending, a strict total order; each group is
// sorted by it in place.  Groups of up to SMALL_SEG items are sorted in shared memory, each item
// moving to its rank in its group; longer ones are listed and sorted by a block each (bitonic in shared memory up to OS_TILE items,
// beyond that a chunked stable radix sort of the digits under the prefix, through the scratch pair).

constexpr int SMALL_SEG = 16;

template <class K>
__device__ __forceinline__ bool kv_less(K ka, uint32_t va, K kb, uint32_t vb)
{
    return ka < kb || (ka == kb && va < vb);
}

constexpr int FIN_THREADS = 256;
constexpr int FIN_ITEMS = 8;
constexpr int FIN_TILE = FIN_THREADS * FIN_ITEMS;

// One tile of FIN_TILE positions per block.  The tile's keys and payloads, the key before it and
// HALO positions after it are staged in shared memory (coalesced loads, all issued before the first
// store).  Each warp then marks, with one ballot per 32 positions, the positions that start a group
// of equal prefix (a head: the prefix differs from the position before), so that every position
// finds the bounds of its group from the head bits around it (a group of at most SMALL_SEG items
// spans at most two 32-bit words).  An item of a group of 2..SMALL_SEG items whose head lies in
// this tile takes its rank by (key, payload) among the group's items and stores itself at the
// group's head + rank when that differs from where it is.  A group's head lists the group when it
// is longer than SMALL_SEG.  Singletons and groups already in order store nothing.  A group belongs
// to the tile that holds its head, also where it runs into the next tile (into the halo), so two
// blocks never store the same position; and since sorting permutes a group only, every position
// keeps its prefix and the group bounds another block reads stay the same.
template <class K>
__global__ void __launch_bounds__(FIN_THREADS, 6) k_sort_finish(K* __restrict__ keys, uint32_t* __restrict__ vals,
                                                             uint64_t n, SortPlan* __restrict__ plan,
                                                             uint64_t* __restrict__ list, uint64_t list_cap,
                                                             uint32_t* __restrict__ err)
{
    grid_dep_enter();
    if (!plan->finish) return;
    constexpr int HALO = SMALL_SEG + 1;
    constexpr uint32_t SPAN = FIN_TILE + HALO;
    constexpr uint32_t NWORD = (SPAN + 31) / 32;
    __shared__ K tk[1 + SPAN];            // tk[1 + j] = key at base + j; tk[0] = key at base - 1
    __shared__ uint32_t tv[SPAN];
    __shared__ uint32_t headw[NWORD + 1]; // bit j % 32 of word j / 32: position j starts a group
    const uint64_t pm = plan->pmask;
    const uint64_t base = (uint64_t)blockIdx.x * FIN_TILE;
    const uint32_t lim = n - base < (uint64_t)SPAN ? (uint32_t)(n - base) : SPAN;
    const uint32_t lane = threadIdx.x & 31;
    {
        K rk[FIN_ITEMS + 1];
        uint32_t rv[FIN_ITEMS + 1];
#pragma unroll
        for (int r = 0; r <= FIN_ITEMS; r++) {
            const uint32_t j = r * FIN_THREADS + threadIdx.x;   // r == FIN_ITEMS: the halo
            if (j < lim && (r < FIN_ITEMS || threadIdx.x < (uint32_t)HALO)) {
                rk[r] = keys[base + j];
                rv[r] = vals[base + j];
            }
        }
#pragma unroll
        for (int r = 0; r <= FIN_ITEMS; r++) {
            const uint32_t j = r * FIN_THREADS + threadIdx.x;
            if (j < lim && (r < FIN_ITEMS || threadIdx.x < (uint32_t)HALO)) {
                tk[1 + j] = rk[r];
                tv[j] = rv[r];
            }
        }
    }
    if (threadIdx.x == 0) {
        tk[0] = base > 0 ? keys[base - 1] : K(0);
        headw[NWORD] = 0xFFFFFFFFu;
    }
    __syncthreads();
    // head bits: positions at or past lim count as heads (they end every group)
#pragma unroll
    for (int r = 0; r <= FIN_ITEMS; r++) {
        const uint32_t j = r * FIN_THREADS + threadIdx.x;
        if (r == FIN_ITEMS && threadIdx.x >= 32) break;          // warp 0 takes the halo word(s)
        bool head = true;
        if (j < lim) head = (j == 0 && base == 0) || (static_cast<uint64_t>(tk[1 + j] ^ tk[j]) & pm) != 0;
        const uint32_t bits = __ballot_sync(FULL, head);
        if (lane == 0 && j / 32 < NWORD) headw[j / 32] = bits;
    }
    __syncthreads();
    const uint32_t tile_end = lim < (uint32_t)FIN_TILE ? lim : (uint32_t)FIN_TILE;
#pragma unroll
    for (int r = 0; r <= FIN_ITEMS; r++) {
        const uint32_t j = r * FIN_THREADS + threadIdx.x;
        if (j >= lim || (r == FIN_ITEMS && threadIdx.x >= (uint32_t)HALO)) continue;
        const uint32_t w = j >> 5, b = j & 31;
        // group start: the last head at or before j (within SMALL_SEG positions, else the group is
        // long or begins in the tile before)
        const uint32_t upto = headw[w] & (0xFFFFFFFFu >> (31 - b));
        int64_t h;
        if (upto) h = (int64_t)(w * 32 + 31 - __clz(upto));
        else if (w > 0 && headw[w - 1]) h = (int64_t)((w - 1) * 32 + 31 - __clz(headw[w - 1]));
        else continue;                                          // no head within 32 positions
        if (j - (uint32_t)h >= (uint32_t)SMALL_SEG) continue;    // deep inside a long group
        if ((uint32_t)h >= tile_end) continue;                  // owned by the next tile
        // group end: the first head after j (headw[NWORD] is all heads); none in the next word
        // either means a group longer than 32
        const uint32_t after = headw[w] & (0xFFFFFFFEu << b);
        const uint32_t nxt = headw[w + 1];
        const uint32_t e = after ? w * 32 + __ffs(after) - 1 : (nxt ? (w + 1) * 32 + __ffs(nxt) - 1 : (w + 2) * 32);
        const uint32_t L = e - (uint32_t)h;
        if (L == 1) continue;
        if (L > (uint32_t)SMALL_SEG) {
            if (j == (uint32_t)h) {
                const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long*>(&plan->nbig), 1ull);
                if (slot < list_cap) list[slot] = base + j;
                else atomicOr(err, ERR_SORT);
            }
            continue;
        }
        const K kj = tk[1 + j];
        const uint32_t vj = tv[j];
        uint32_t rank = 0;
        for (uint32_t i = (uint32_t)h; i < e; i++) rank += kv_less(tk[1 + i], tv[i], kj, vj);
        const uint32_t to = (uint32_t)h + rank;
        if (to != j) {
            keys[base + to] = kj;
            vals[base + to] = vj;
        }
    }
}

// One block per listed group, taken from a shared cursor.
template <class K>
__global__ void __launch_bounds__(OS_THREADS, 1) k_sort_finish_big(K* __restrict__ keys, uint32_t* __restrict__ vals,
                                                                   K* __restrict__ tk, uint32_t* __restrict__ tv,
                                                                   uint64_t n, SortPlan* __restrict__ plan,
                                                                   const uint64_t* __restrict__ list, uint64_t list_cap)
{
    grid_dep_enter();
    if (!plan->finish) return;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + OS_TILE);
    uint16_t* whist = reinterpret_cast<uint16_t*>(sv + OS_TILE);                // [OS_WARPS][RADIX]
    uint32_t* s_cnt = reinterpret_cast<uint32_t*>(whist + OS_WARPS * RADIX);    // [RADIX]
    __shared__ unsigned long long s_item, s_end;
    __shared__ uint32_t s_off[RADIX], s_base[RADIX], s_skip;
    const uint64_t pm = plan->pmask;
    const int lo_shift = plan->shift[0];
    const uint64_t nbig = min((uint64_t)plan->nbig, list_cap);
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = atomicAdd(reinterpret_cast<unsigned long long*>(&plan->cursor), 1ull);
            s_end = n;
        }
        __syncthreads();
        const uint64_t item = s_item;
        if (item >= nbig) break;
        const uint64_t start = list[item];
        const K k0 = keys[start];
        // the group ends at the first position whose prefix differs
        for (uint64_t b = start + SMALL_SEG; b < n; b += OS_THREADS) {
            const uint64_t j = b + threadIdx.x;
            const bool stop = j < n && (static_cast<uint64_t>(keys[j] ^ k0) & pm) != 0;
            if (stop) atomicMin(&s_end, (unsigned long long)j);
            if (__syncthreads_or(stop)) break;
        }
        const uint64_t L = s_end - start;
        // a group already in (key, payload) order stays as it is: a key repeated across the batch,
        // mostly (the passes are stable, so its copies are in position order)
        bool descent = false;
        for (uint64_t j = start + 1 + threadIdx.x; j < start + L; j += OS_THREADS)
            descent |= kv_less(keys[j], vals[j], keys[j - 1], vals[j - 1]);
        if (!__syncthreads_or(descent)) continue;
        if (L <= (uint64_t)OS_TILE) {
            uint32_t P2 = 2;
            while (P2 < L) P2 <<= 1;
            for (uint32_t j = threadIdx.x; j < P2; j += OS_THREADS) {
                const bool ok = j < L;
                sk[j] = ok ? keys[start + j] : ~K(0);
                sv[j] = ok ? vals[start + j] : 0xFFFFFFFFu;   // positions are below 2^32 - 1: padding sorts last
            }
            __syncthreads();
            for (uint32_t k = 2; k <= P2; k <<= 1) {
                for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                    for (uint32_t t = threadIdx.x; t < P2 / 2; t += OS_THREADS) {
                        const uint32_t a = ((t & ~(j - 1)) << 1) | (t & (j - 1));
                        const uint32_t b = a + j;
                        const bool up = (a & k) == 0;
                        const K ka = sk[a], kb = sk[b];
                        const uint32_t va = sv[a], vb = sv[b];
                        if (up ? kv_less(kb, vb, ka, va) : kv_less(ka, va, kb, vb)) {
                            sk[a] = kb; sk[b] = ka;
                            sv[a] = vb; sv[b] = va;
                        }
                    }
                    __syncthreads();
                }
            }
            for (uint32_t j = threadIdx.x; j < L; j += OS_THREADS) {
                keys[start + j] = sk[j];
                vals[start + j] = sv[j];
            }
            __syncthreads();
            continue;
        }
        // Long group: stable LSD over the digits under the prefix, chunk by chunk (chunks in order,
        // items of a chunk ranked as in a sweep tile), between the group's range of the output
        // pair and the same range of the scratch pair.
        K* srck = keys + start;
        uint32_t* srcv = vals + start;
        K* dstk = tk + start;
        uint32_t* dstv = tv + start;
        for (int shift = 0; shift < lo_shift; shift += 8) {
            for (int d = threadIdx.x; d < RADIX; d += OS_THREADS) s_cnt[d] = 0;
            __syncthreads();
            for (uint64_t j = threadIdx.x; j < L; j += OS_THREADS) atomicAdd(&s_cnt[digit_of(srck[j], shift)], 1u);
            __syncthreads();
            if (threadIdx.x == 0) {
                uint32_t run = 0, skip = 0;
                for (int d = 0; d < RADIX; d++) {
                    s_off[d] = run;
                    skip |= (uint64_t)s_cnt[d] == L;
                    run += s_cnt[d];
                }
                s_skip = skip;
            }
            __syncthreads();
            if (s_skip) continue;    // one digit value in the whole group: the pass moves nothing
            for (uint64_t c0 = 0; c0 < L; c0 += OS_TILE) {
                for (int i = threadIdx.x; i < OS_WARPS * RADIX / 2; i += OS_THREADS)
                    reinterpret_cast<uint32_t*>(whist)[i] = 0;
                __syncthreads();
                K key[OS_ITEMS];
                uint32_t val[OS_ITEMS];
                uint32_t rank[OS_ITEMS];
                const uint64_t wb = c0 + (uint64_t)warp * 32 * OS_ITEMS;
#pragma unroll
                for (int i = 0; i < OS_ITEMS; i++) {
                    const uint64_t pos = wb + (uint64_t)i * 32 + lane;
                    key[i] = pos < L ? srck[pos] : K(0);
                    val[i] = pos < L ? srcv[pos] : 0u;
                }
                rank_warp<K, false>(key, rank, whist + warp * RADIX, wb, L, shift);
                __syncthreads();
                if (threadIdx.x < RADIX) {
                    const uint32_t d = threadIdx.x;
                    uint32_t run = 0;
                    for (int w = 0; w < OS_WARPS; w++) {
                        const uint32_t c = whist[w * RADIX + d];
                        whist[w * RADIX + d] = (uint16_t)run;
                        run += c;
                    }
                    s_base[d] = s_off[d];
                    s_off[d] += run;
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < OS_ITEMS; i++) {
                    const uint64_t pos = wb + (uint64_t)i * 32 + lane;
                    if (pos < L) {
                        const uint32_t d = digit_of(key[i], shift);
                        const uint64_t o = (uint64_t)s_base[d] + whist[warp * RADIX + d] + rank[i];
                        dstk[o] = key[i];
                        dstv[o] = val[i];
                    }
                }
                __syncthreads();
            }
            K* t0 = srck; srck = dstk; dstk = t0;
            uint32_t* t1 = srcv; srcv = dstv; dstv = t1;
        }
        if (srck != keys + start) {
            for (uint64_t j = threadIdx.x; j < L; j += OS_THREADS) {
                keys[start + j] = srck[j];
                vals[start + j] = srcv[j];
            }
        }
        __syncthreads();
    }
}

// ---- exclusive scan ----------------------------------------------------------------------------

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_part(const Tin* __restrict__ in, uint64_t n, Tout* __restrict__ part)
{
    grid_dep_enter();
    __shared__ Tout sw[NWARPS];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE;
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        uint64_t pos = base + (uint64_t)i * SCAN_THREADS + threadIdx.x;
        if (pos < n) s += static_cast<Tout>(in[pos]);
    }
    Tout tot;
    block_excl_scan<Tout>(s, sw, tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

template <class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_top(Tout* __restrict__ part, uint32_t ntiles, Tout* __restrict__ total_out)
{
    grid_dep_enter();
    __shared__ Tout sw[NWARPS];
    Tout carry = 0;
    for (uint32_t t0 = 0; t0 < ntiles; t0 += SCAN_THREADS) {
        uint32_t t = t0 + threadIdx.x;
        Tout v = t < ntiles ? part[t] : Tout(0);
        Tout tot;
        Tout ex = block_excl_scan<Tout>(v, sw, tot);
        if (t < ntiles) part[t] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total_out = carry;
}

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_apply(const Tin* __restrict__ in, uint64_t n,
                                                            const Tout* __restrict__ part, Tout* __restrict__ out)
{
    grid_dep_enter();
    __shared__ Tout sw[NWARPS];
    const uint64_t base = (uint64_t)blockIdx.x * SCAN_TILE + (uint64_t)threadIdx.x * SCAN_ITEMS;
    Tout v[SCAN_ITEMS];
    Tout s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        uint64_t pos = base + i;
        v[i] = pos < n ? static_cast<Tout>(in[pos]) : Tout(0);
        s += v[i];
    }
    Tout tot;
    Tout ex = block_excl_scan<Tout>(s, sw, tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        uint64_t pos = base + i;
        if (pos < n) out[pos] = ex;
        ex += v[i];
    }
}

}  // namespace

// Forces the module loader to load every kernel of this file now (see preload_kernels).
void preload_sort_kernels()
{
    cudaFuncAttributes a;
#define FLIX_TOUCH(...) cudaFuncGetAttributes(&a, __VA_ARGS__)
    FLIX_TOUCH(k_scan_digits);
    FLIX_TOUCH(k_scan_part<uint32_t, uint32_t>);
    FLIX_TOUCH(k_scan_part<uint32_t, uint64_t>);
    FLIX_TOUCH(k_scan_part<uint64_t, uint64_t>);
    FLIX_TOUCH(k_scan_part<uint8_t, uint32_t>);
    FLIX_TOUCH(k_scan_top<uint32_t>);
    FLIX_TOUCH(k_scan_top<uint64_t>);
    FLIX_TOUCH(k_scan_apply<uint32_t, uint32_t>);
    FLIX_TOUCH(k_scan_apply<uint32_t, uint64_t>);
    FLIX_TOUCH(k_scan_apply<uint64_t, uint64_t>);
    FLIX_TOUCH(k_scan_apply<uint8_t, uint32_t>);
#define FLIX_TOUCH_K(K)                      \
    FLIX_TOUCH(k_hist_all<K>);               \
    FLIX_TOUCH(k_sort_plan<K>);              \
    FLIX_TOUCH(k_upsweep<K>);                \
    FLIX_TOUCH(k_sweep<K, true>);            \
    FLIX_TOUCH(k_sweep_tail<K>);             \
    FLIX_TOUCH(k_sweep<K, false>);           \
    FLIX_TOUCH(k_sort_finish<K>);            \
    FLIX_TOUCH(k_sort_finish_big<K>)
    FLIX_TOUCH_K(uint32_t);
    FLIX_TOUCH_K(uint64_t);
#undef FLIX_TOUCH_K
#undef FLIX_TOUCH
}

template <class Tout>
size_t scan_scratch_bytes(uint64_t n)
{
    return ((size_t)div_up(n ? n : 1, SCAN_TILE) * sizeof(Tout) + 511) & ~size_t(255);
}

template <class Tin, class Tout>
cudaError_t scan_exclusive(Ctx& c, const Tin* in, Tout* out, uint64_t n)
{
    if (n == 0) return fill_bytes(c, out, 0, sizeof(Tout));
    const uint32_t ntiles = div_up(n, SCAN_TILE);
    Tout* part = c.h->arena.take<Tout>(ntiles);
    if (!part) return cudaErrorMemoryAllocation;
    cudaError_t e = launch(c, K_SCAN_PART, dim3(ntiles), dim3(SCAN_THREADS), 0, k_scan_part<Tin, Tout>, in, n, part);
    if (e) return e;
    e = launch(c, K_SCAN_TOP, dim3(1), dim3(SCAN_THREADS), 0, k_scan_top<Tout>, part, ntiles, out + n);
    if (e) return e;
    return launch(c, K_SCAN_APPLY, dim3(ntiles), dim3(SCAN_THREADS), 0, k_scan_apply<Tin, Tout>, in, n,
                  (const Tout*)part, out);
}

template <class K>
size_t sort_scratch_bytes(uint64_t n)
{
    constexpr size_t P = sizeof(K);
    const size_t T = div_up(n ? n : 1, OS_TILE);
    auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
    const size_t pingpong = al(n * sizeof(K)) + al(n * 4);
    const size_t rts = 2 * al(T * RADIX * 4);                      // counts, offsets
    const size_t one = al(P * T * RADIX * 4) + al((P + 1) * 4);    // tile states, tile counters, barrier
    const size_t fin = al(sizeof(SortPlan)) + al((n / (SMALL_SEG + 1) + 1) * 8);   // plan, long-group list
    return pingpong + al(P * RADIX * 4) + (rts > one ? rts : one) + fin + 1024;
}

// Prefix digits the plan may stop at: the fewest h with 2^(8h) >= n.
template <class K>
static uint32_t prefix_digits(uint64_t n)
{
    uint32_t h = 1;
    while (h < sizeof(K) && (8 * h >= 64 || (1ull << (8 * h)) < n)) h++;
    return h;
}

template <class K>
cudaError_t sort_pairs(Ctx& c, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, uint64_t n)
{
    if (n == 0) return cudaSuccess;
    // the payload is the input position: it is what makes (key, payload) a strict order for the
    // finish kernels, and positions must stay below 2^32 - 1
    if (vin != nullptr || n >= 0xFFFFFFFFull) return cudaErrorInvalidValue;
    constexpr int P = sizeof(K);
    Arena& A = c.h->arena;
    // one-sweep unless asked otherwise; 30-bit tile states need n < 2^30
    const bool onesweep = c.h->cfg.sort_variant != FLIX_SORT_REDUCE_SCAN && n < (1ull << 30);
    const uint32_t T = div_up(n, OS_TILE);
    uint32_t* bases = A.take<uint32_t>(P * RADIX);
    uint32_t* status = onesweep ? A.take<uint32_t>((size_t)P * T * RADIX) : nullptr;
    uint32_t* tile_ctr = onesweep ? A.take<uint32_t>(P + 1) : nullptr;   // + the tail's barrier word
    uint32_t* counts = onesweep ? nullptr : A.take<uint32_t>((size_t)T * RADIX);
    uint32_t* offsets = onesweep ? nullptr : A.take<uint32_t>((size_t)T * RADIX);
    K* tk = A.take<K>(n);
    uint32_t* tv = A.take<uint32_t>(n);
    SortPlan* plan = A.take<SortPlan>(1);
    const uint64_t list_cap = n / (SMALL_SEG + 1) + 1;
    uint64_t* list = A.take<uint64_t>(list_cap);
    if (!bases || !tk || !tv || !plan || !list || (onesweep ? (!status || !tile_ctr) : (!counts || !offsets)))
        return cudaErrorMemoryAllocation;
    // the digit counts, the tile states and the tile counters were taken one after another from the
    // arena: one fill zeroes them all
    cudaError_t e = onesweep ? fill_bytes(c, bases, 0,
                                          (size_t)(reinterpret_cast<char*>(tile_ctr + P + 1) -
                                                   reinterpret_cast<char*>(bases)))
                             : fill_bytes(c, bases, 0, P * RADIX * 4);
    if (e) return e;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.h->device);
    uint32_t hg = div_up(n, 256);
    if (hg > (uint32_t)nsm * 8) hg = nsm * 8;
    if ((e = launch(c, K_SORT_HIST, dim3(hg), dim3(256), 0, k_hist_all<K>, kin, n, bases))) return e;
    if ((e = launch(c, K_SORT_PLAN, dim3(1), dim3(RADIX), 0, k_sort_plan<K>, bases, n, prefix_digits<K>(n), plan)))
        return e;
    // The plan's pass count lives on the device; every possible pass is launched and those beyond
    // it return at once.  When profiling, the count is read back so that idle passes are timed
    // under their own name.
    uint32_t active = P;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((e = cudaStreamIsCapturing(c.st, &cap))) return e;
    if (c.h->prof_on && cap == cudaStreamCaptureStatusNone) {
        if (readback_at(c.h, c.st, 62, {{&plan->npass, 4}}) != FLIX_OK) return cudaErrorUnknown;
        active = (uint32_t)c.h->hpin[62];
    }
    const size_t smem = sweep_smem<K>();
    e = onesweep ? cudaFuncSetAttribute(k_sweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_sweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    // the plan takes at least the h prefix digits unless fewer digits vary; one-sweep runs the passes
    // after those in one cooperative launch, which returns at once when the plan leaves them out
    const uint32_t h_min = onesweep ? std::min<uint32_t>(prefix_digits<K>(n), P) : P;
    for (int p = 0; p < (int)h_min; p++) {
        const bool on = (uint32_t)p < active;
        // algorithmic bytes: the first pass reads keys only (payload = position)
        const double bytes = on ? (double)n * ((p == 0 ? sizeof(K) : sizeof(K) + 4) + sizeof(K) + 4) : 0.0;
        if (onesweep) {
            e = launch_b(c, on ? K_SORT_ONESWEEP : K_SORT_IDLE, bytes, dim3(T), dim3(OS_THREADS), smem,
                         k_sweep<K, true>, kin, kout, vout, tk, tv, n, p, (const SortPlan*)plan,
                         (const uint32_t*)bases, (const uint32_t*)nullptr, T, status + (size_t)p * T * RADIX,
                         tile_ctr + p, c.h->err);
        } else {
            e = launch(c, on ? K_SORT_UP : K_SORT_IDLE, dim3(T), dim3(UP_THREADS_S), 0, k_upsweep<K>, kin, kout, vout,
                       tk, tv, n, p, (const SortPlan*)plan, counts, T);
            if (!e)
                e = launch(c, on ? K_SORT_SCAN : K_SORT_IDLE, dim3(RADIX), dim3(256), 0, k_scan_digits,
                           (const uint32_t*)counts, T, p, (const SortPlan*)plan, (const uint32_t*)bases, offsets);
            if (!e)
                e = launch_b(c, on ? K_SORT_DOWN : K_SORT_IDLE, bytes, dim3(T), dim3(OS_THREADS), smem,
                             k_sweep<K, false>, kin, kout, vout, tk, tv, n, p, (const SortPlan*)plan,
                             (const uint32_t*)bases, (const uint32_t*)offsets, T, (uint32_t*)nullptr,
                             (uint32_t*)nullptr, c.h->err);
        }
        if (e) return e;
    }
    if (h_min < (uint32_t)P) {
        if ((e = cudaFuncSetAttribute(k_sweep_tail<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        int per_sm = 0;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_tail<K>, OS_THREADS, smem))) return e;
        // every block of a cooperative launch is resident at once, which the grid barrier needs
        const uint32_t wave = std::min<uint32_t>(T, (uint32_t)std::max(per_sm, 1) * (uint32_t)nsm);
        double bytes = 0.0;
        for (uint32_t p = h_min; p < active && p < (uint32_t)P; p++) bytes += (double)n * 2.0 * (sizeof(K) + 4);
        e = launch_coop(c, active > h_min ? K_SORT_ONESWEEP : K_SORT_IDLE, bytes, dim3(wave), dim3(OS_THREADS), smem,
                        k_sweep_tail<K>, kin, kout, vout, tk, tv, n, (int)h_min, (const SortPlan*)plan,
                        (const uint32_t*)bases, T, status, tile_ctr, tile_ctr + P, c.h->err);
        if (e) return e;
    }
    if ((e = launch(c, K_SORT_FINISH, dim3(div_up(n, FIN_TILE)), dim3(FIN_THREADS), 0, k_sort_finish<K>, kout, vout, n,
                    plan, list, list_cap, c.h->err)))
        return e;
    if ((e = cudaFuncSetAttribute(k_sort_finish_big<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    return launch(c, K_SORT_FINISH, dim3(nsm), dim3(OS_THREADS), smem, k_sort_finish_big<K>, kout, vout, tk, tv, n,
                  plan, (const uint64_t*)list, list_cap);
}

template size_t sort_scratch_bytes<uint32_t>(uint64_t);
template size_t sort_scratch_bytes<uint64_t>(uint64_t);
template cudaError_t sort_pairs<uint32_t>(Ctx&, const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint64_t);
template cudaError_t sort_pairs<uint64_t>(Ctx&, const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, uint64_t);
template size_t scan_scratch_bytes<uint32_t>(uint64_t);
template size_t scan_scratch_bytes<uint64_t>(uint64_t);
template cudaError_t scan_exclusive<uint32_t, uint32_t>(Ctx&, const uint32_t*, uint32_t*, uint64_t);
template cudaError_t scan_exclusive<uint32_t, uint64_t>(Ctx&, const uint32_t*, uint64_t*, uint64_t);
template cudaError_t scan_exclusive<uint64_t, uint64_t>(Ctx&, const uint64_t*, uint64_t*, uint64_t);
template cudaError_t scan_exclusive<uint8_t, uint32_t>(Ctx&, const uint8_t*, uint32_t*, uint64_t);

}  // namespace flix
