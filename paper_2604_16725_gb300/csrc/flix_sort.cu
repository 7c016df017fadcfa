// Batch sort (Sec. 3.3: each batch is sorted by key before buckets pull their operations; Tab. 1
// times it) and prefix-sum primitives.
//
// The sort is a stable least-significant-digit radix sort of (key, payload) pairs with 8-bit
// digits.  One read of the keys builds the digit histograms of every pass.  Each pass is one
// scatter kernel over 4096-item tiles (512 threads x 8 items, two blocks per SM): a tile ranks its
// items in shared memory with warp match/popc (stable: warp-striped items ranked in warp, item,
// lane order), learns where each digit's run of this tile starts in the output, and writes the
// locally sorted tile so that each digit's run is a contiguous store.  The start of each
// (digit, tile) run comes either from
//   - one-sweep (after the single-pass "Onesweep" radix sort of Adinets and Merrill, 2022): every
//     tile publishes its per-digit counts and looks back through the published states of earlier
//     tiles (an aggregate, or an inclusive prefix that ends the walk), reading 8 earlier tiles per
//     round trip; tiles take their index from an atomic counter in start order, so each tile
//     waited on has already started, and every wait is bounded (a wait that runs out sets an
//     error bit); or
//   - reduce-then-scan: an upsweep kernel counts each tile's digits, a scan kernel turns the counts
//     into run starts, and the scatter reads them.
// Both give the same (stable) order; the one-sweep variant saves one read of the keys per pass.
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

// Digit histograms of every pass from one read of the keys.
template <class K>
__global__ void __launch_bounds__(256) k_hist_all(const K* __restrict__ keys, uint64_t n, uint32_t* __restrict__ hist)
{
    constexpr int P = sizeof(K);
    __shared__ uint32_t sh[P * RADIX];
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        K k = keys[i];
#pragma unroll
        for (int p = 0; p < P; p++) atomicAdd(&sh[p * RADIX + digit_of(k, 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < P * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// In place: hist[p * RADIX + d] becomes the number of items whose pass-p digit is below d.
__global__ void __launch_bounds__(RADIX) k_digit_bases(uint32_t* __restrict__ hist)
{
    __shared__ uint32_t sw[RADIX / 32];
    uint32_t* h = hist + (size_t)blockIdx.x * RADIX;
    uint32_t tot;
    const uint32_t b = block_excl_scan<uint32_t, RADIX / 32>(h[threadIdx.x], sw, tot);
    h[threadIdx.x] = b;
}

// Reduce-then-scan: per-tile digit counts of one pass, counts[d * T + tile].
template <class K>
__global__ void __launch_bounds__(UP_THREADS_S) k_upsweep(const K* __restrict__ keys, uint64_t n, int shift,
                                                          uint32_t* __restrict__ counts, uint32_t T)
{
    __shared__ uint32_t sh[RADIX];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * OS_TILE;
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll 4
    for (int i = 0; i < UP_ITEMS; i++) {
        uint64_t pos = base + (uint64_t)i * UP_THREADS_S + threadIdx.x;
        uint32_t d = pos < n ? digit_of(keys[pos], shift) : RADIX;
        uint32_t peers = __match_any_sync(FULL, d);
        if (d < RADIX && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * T + blockIdx.x] = sh[threadIdx.x];
}

// Reduce-then-scan: offsets[d * T + t] = bases[d] + (items of digit d in tiles < t).
__global__ void __launch_bounds__(256) k_scan_digits(const uint32_t* __restrict__ counts, uint32_t T,
                                                    const uint32_t* __restrict__ bases, uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t sw[NWARPS];
    const uint32_t d = blockIdx.x;
    uint32_t carry = bases[d];
    for (uint32_t t0 = 0; t0 < T; t0 += 256) {
        uint32_t t = t0 + threadIdx.x;
        uint32_t c = t < T ? counts[(uint64_t)d * T + t] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan<uint32_t>(c, sw, tot);
        if (t < T) offsets[(uint64_t)d * T + t] = carry + ex;
        carry += tot;
    }
}

// One digit pass.  vin == nullptr: payload = position.  LOOKBACK selects one-sweep (status,
// tile_ctr) or reduce-then-scan (offsets).
template <class K, bool LOOKBACK>
__global__ void __launch_bounds__(OS_THREADS, 2) k_sweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout, uint64_t n,
                                                         int shift, const uint32_t* __restrict__ bases,
                                                         const uint32_t* __restrict__ offsets, uint32_t T,
                                                         uint32_t* __restrict__ status, uint32_t* __restrict__ tile_ctr,
                                                         uint32_t* __restrict__ err)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + OS_TILE);
    uint16_t* whist = reinterpret_cast<uint16_t*>(sv + OS_TILE);                // [OS_WARPS][RADIX]
    uint32_t* goff = reinterpret_cast<uint32_t*>(whist + OS_WARPS * RADIX);     // [RADIX]
    uint32_t* sw = goff + RADIX;                                                // [OS_WARPS]
    uint32_t* s_tile = sw + OS_WARPS;

    if (LOOKBACK && threadIdx.x == 0) *s_tile = atomicAdd(tile_ctr, 1u);
    for (int i = threadIdx.x; i < OS_WARPS * RADIX / 2; i += OS_THREADS) reinterpret_cast<uint32_t*>(whist)[i] = 0;
    __syncthreads();
    const uint32_t tile = LOOKBACK ? *s_tile : blockIdx.x;
    const uint64_t base = (uint64_t)tile * OS_TILE;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

    K key[OS_ITEMS];
    uint32_t val[OS_ITEMS];
    uint32_t rank[OS_ITEMS];
    const uint64_t wbase = base + (uint64_t)warp * 32 * OS_ITEMS;
#pragma unroll
    for (int i = 0; i < OS_ITEMS; i++) {
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        bool ok = pos < n;
        key[i] = ok ? kin[pos] : K(0);
        val[i] = ok ? (vin ? vin[pos] : static_cast<uint32_t>(pos)) : 0u;
    }
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < OS_ITEMS; i++) {
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        uint32_t d = pos < n ? digit_of(key[i], shift) : RADIX;
        uint32_t peers = __match_any_sync(FULL, d);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t prior = 0;
        if (lane == leader && d < RADIX) prior = whist[warp * RADIX + d];
        prior = __shfl_sync(FULL, prior, leader);
        rank[i] = prior + __popc(peers & lt);
        if (lane == leader && d < RADIX) whist[warp * RADIX + d] = (uint16_t)(prior + __popc(peers));
        __syncwarp();
    }
    __syncthreads();
    uint32_t cnt = 0;
    if (threadIdx.x < RADIX) {
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < OS_WARPS; w++) {
            uint32_t c = whist[w * RADIX + d];
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
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        if (pos < n) {
            uint32_t d = digit_of(key[i], shift);
            uint32_t r = whist[warp * RADIX + d] + rank[i];
            sk[r] = key[i];
            sv[r] = val[i];
        }
    }
    __syncthreads();
    const uint32_t tile_n = (uint32_t)((n - base) < (uint64_t)OS_TILE ? (n - base) : OS_TILE);
    for (uint32_t j = threadIdx.x; j < tile_n; j += OS_THREADS) {
        K k = sk[j];
        uint32_t o = goff[digit_of(k, shift)] + j;
        kout[o] = k;
        vout[o] = sv[j];
    }
}

template <class K>
size_t sweep_smem()
{
    return (size_t)OS_TILE * (sizeof(K) + 4) + (size_t)OS_WARPS * RADIX * 2 + (RADIX + OS_WARPS + 4) * 4;
}

// ---- exclusive scan ----------------------------------------------------------------------------

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

template <class Tin, class Tout>
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_part(const Tin* __restrict__ in, uint64_t n, Tout* __restrict__ part)
{
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

template <class Tout>
size_t scan_scratch_bytes(uint64_t n)
{
    return ((size_t)div_up(n ? n : 1, SCAN_TILE) * sizeof(Tout) + 511) & ~size_t(255);
}

template <class Tin, class Tout>
cudaError_t scan_exclusive(Ctx& c, const Tin* in, Tout* out, uint64_t n)
{
    if (n == 0) return cudaMemsetAsync(out, 0, sizeof(Tout), c.st);
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
    const size_t one = al(P * T * RADIX * 4) + al(P * 4);          // tile states, tile counters
    return pingpong + al(P * RADIX * 4) + (rts > one ? rts : one) + 1024;
}

template <class K>
cudaError_t sort_pairs(Ctx& c, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, uint64_t n)
{
    if (n == 0) return cudaSuccess;
    constexpr int P = sizeof(K);
    Arena& A = c.h->arena;
    // one-sweep unless asked otherwise; 30-bit tile states need n < 2^30
    const bool onesweep = c.h->cfg.sort_variant != FLIX_SORT_REDUCE_SCAN && n < (1ull << 30);
    const uint32_t T = div_up(n, OS_TILE);
    uint32_t* bases = A.take<uint32_t>(P * RADIX);
    uint32_t* status = onesweep ? A.take<uint32_t>((size_t)P * T * RADIX) : nullptr;
    uint32_t* tile_ctr = onesweep ? A.take<uint32_t>(P) : nullptr;
    uint32_t* counts = onesweep ? nullptr : A.take<uint32_t>((size_t)T * RADIX);
    uint32_t* offsets = onesweep ? nullptr : A.take<uint32_t>((size_t)T * RADIX);
    K* tk = A.take<K>(n);
    uint32_t* tv = A.take<uint32_t>(n);
    if (!bases || !tk || !tv || (onesweep ? (!status || !tile_ctr) : (!counts || !offsets)))
        return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(bases, 0, P * RADIX * 4, c.st);
    if (e) return e;
    if (onesweep) {
        if ((e = cudaMemsetAsync(status, 0, (size_t)P * T * RADIX * 4, c.st))) return e;
        if ((e = cudaMemsetAsync(tile_ctr, 0, P * 4, c.st))) return e;
    }
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.h->device);
    uint32_t hg = div_up(n, 256);
    if (hg > (uint32_t)nsm * 8) hg = nsm * 8;
    if ((e = launch(c, K_SORT_HIST, dim3(hg), dim3(256), 0, k_hist_all<K>, kin, n, bases))) return e;
    if ((e = launch(c, K_SORT_SCAN, dim3(P), dim3(RADIX), 0, k_digit_bases, bases))) return e;
    const size_t smem = sweep_smem<K>();
    e = onesweep ? cudaFuncSetAttribute(k_sweep<K, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                 : cudaFuncSetAttribute(k_sweep<K, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const K* sk = kin;
    const uint32_t* sv = vin;
    for (int p = 0; p < P; p++) {
        // the last pass writes kout; passes alternate between kout and the scratch pair
        const bool to_out = ((P - 1 - p) & 1) == 0;
        K* dk = to_out ? kout : tk;
        uint32_t* dv = to_out ? vout : tv;
        const int shift = 8 * p;
        const uint32_t* bp = bases + p * RADIX;
        if (onesweep) {
            e = launch(c, K_SORT_ONESWEEP, dim3(T), dim3(OS_THREADS), smem, k_sweep<K, true>, sk, sv, dk, dv, n, shift,
                       bp, (const uint32_t*)nullptr, T, status + (size_t)p * T * RADIX, tile_ctr + p, c.h->err);
        } else {
            e = launch(c, K_SORT_UP, dim3(T), dim3(UP_THREADS_S), 0, k_upsweep<K>, sk, n, shift, counts, T);
            if (!e)
                e = launch(c, K_SORT_SCAN, dim3(RADIX), dim3(256), 0, k_scan_digits, (const uint32_t*)counts, T, bp,
                           offsets);
            if (!e)
                e = launch(c, K_SORT_DOWN, dim3(T), dim3(OS_THREADS), smem, k_sweep<K, false>, sk, sv, dk, dv, n, shift,
                           bp, (const uint32_t*)offsets, T, (uint32_t*)nullptr, (uint32_t*)nullptr, c.h->err);
        }
        if (e) return e;
        sk = dk;
        sv = dv;
    }
    return cudaSuccess;
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
