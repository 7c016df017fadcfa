// Batch sort (Sec. 3.3: "sorting the query list"; Tab. 1 times it) and prefix-sum primitives.
//
// The sort is a stable least-significant-digit radix sort of (key, payload) pairs with 8-bit
// digits: one read of the keys builds the digit histograms of every pass; each pass then counts
// its digit per 4096-item tile (upsweep), scans the (digit, tile) counts, and scatters (downsweep).
// The downsweep ranks a tile in shared memory with warp match/popc (stable: warp-striped items,
// ranked in warp, item, lane order), then writes the locally sorted tile out so that each digit's
// run is a contiguous, coalesced store.
#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr uint32_t FULL = 0xFFFFFFFFu;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 16;
constexpr int SORT_TILE = SORT_THREADS * SORT_ITEMS;
constexpr int NWARPS = SORT_THREADS / 32;
constexpr int RADIX = 256;

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

// Exclusive scan of one value per thread over a 256-thread block; `total` gets the block sum.
// sw must hold NWARPS entries; the function ends with a barrier so sw can be reused.
template <class T>
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
        T t = lane < NWARPS ? sw[lane] : T(0);
#pragma unroll
        for (int o = 1; o < NWARPS; o <<= 1) {
            T y = __shfl_up_sync(FULL, t, o);
            if (lane >= o) t += y;
        }
        if (lane < NWARPS) sw[lane] = t;
    }
    __syncthreads();
    T wbase = w ? sw[w - 1] : T(0);
    total = sw[NWARPS - 1];
    __syncthreads();
    return wbase + x - v;
}

template <class K>
__device__ __forceinline__ uint32_t digit_of(K k, int shift) { return static_cast<uint32_t>(k >> shift) & 255u; }

// Digit histograms of every pass from one read of the keys.
template <class K>
__global__ void __launch_bounds__(256) k_hist_all(const K* __restrict__ keys, uint64_t n,
                                                 uint32_t* __restrict__ hist)
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

// Per-tile digit counts of one pass: counts[d * T + tile].
template <class K>
__global__ void __launch_bounds__(SORT_THREADS) k_upsweep(const K* __restrict__ keys, uint64_t n, int shift,
                                                          uint32_t* __restrict__ counts, uint32_t T)
{
    __shared__ uint32_t sh[RADIX];
    sh[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)blockIdx.x * SORT_TILE;
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll 4
    for (int i = 0; i < SORT_ITEMS; i++) {
        uint64_t pos = base + (uint64_t)i * SORT_THREADS + threadIdx.x;
        uint32_t d = pos < n ? digit_of(keys[pos], shift) : RADIX;
        uint32_t peers = __match_any_sync(FULL, d);
        if (d < RADIX && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&sh[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(uint64_t)threadIdx.x * T + blockIdx.x] = sh[threadIdx.x];
}

// offsets[d * T + t] = (items of digit < d) + (items of digit d in tiles < t).
__global__ void __launch_bounds__(256) k_scan_digits(const uint32_t* __restrict__ counts, uint32_t T,
                                                    const uint32_t* __restrict__ hist,
                                                    uint32_t* __restrict__ offsets)
{
    __shared__ uint32_t sw[NWARPS];
    const uint32_t d = blockIdx.x;
    uint32_t base;
    block_excl_scan<uint32_t>(threadIdx.x < d ? hist[threadIdx.x] : 0u, sw, base);
    uint32_t carry = base;
    for (uint32_t t0 = 0; t0 < T; t0 += 256) {
        uint32_t t = t0 + threadIdx.x;
        uint32_t c = t < T ? counts[(uint64_t)d * T + t] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan<uint32_t>(c, sw, tot);
        if (t < T) offsets[(uint64_t)d * T + t] = carry + ex;
        carry += tot;
    }
}

// One scatter pass.  vin == nullptr: payload = position.
template <class K>
__global__ void __launch_bounds__(SORT_THREADS) k_downsweep(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                            K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                            uint64_t n, int shift,
                                                            const uint32_t* __restrict__ offsets, uint32_t T)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    K* sk = reinterpret_cast<K*>(smem_raw);
    uint32_t* sv = reinterpret_cast<uint32_t*>(sk + SORT_TILE);
    uint32_t* whist = sv + SORT_TILE;          // [NWARPS][RADIX]: counts, then warp bases
    uint32_t* dstart = whist + NWARPS * RADIX;  // [RADIX]: tile-local start of each digit
    uint32_t* goff = dstart + RADIX;            // [RADIX]: global start of (digit, tile)
    uint32_t* sw = goff + RADIX;                // [NWARPS]

    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * SORT_TILE;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NWARPS * RADIX; i += SORT_THREADS) whist[i] = 0;

    K key[SORT_ITEMS];
    uint32_t val[SORT_ITEMS];
    uint32_t rank[SORT_ITEMS];
    const uint64_t wbase = base + (uint64_t)warp * 32 * SORT_ITEMS;
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        bool ok = pos < n;
        key[i] = ok ? kin[pos] : K(0);
        val[i] = ok ? (vin ? vin[pos] : static_cast<uint32_t>(pos)) : 0u;
    }
    __syncthreads();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        uint32_t d = pos < n ? digit_of(key[i], shift) : RADIX;
        uint32_t peers = __match_any_sync(FULL, d);
        uint32_t leader = __ffs(peers) - 1;
        uint32_t prior = 0;
        if (lane == leader && d < RADIX) prior = whist[warp * RADIX + d];
        prior = __shfl_sync(FULL, prior, leader);
        rank[i] = prior + __popc(peers & lt);
        if (lane == leader && d < RADIX) whist[warp * RADIX + d] = prior + __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    // per digit: exclusive prefix over warps, then over digits
    {
        const uint32_t d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < NWARPS; w++) {
            uint32_t c = whist[w * RADIX + d];
            whist[w * RADIX + d] = run;
            run += c;
        }
        uint32_t tot;
        uint32_t start = block_excl_scan<uint32_t>(run, sw, tot);
        dstart[d] = start;
        goff[d] = offsets[(uint64_t)d * T + tile];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SORT_ITEMS; i++) {
        uint64_t pos = wbase + (uint64_t)i * 32 + lane;
        if (pos < n) {
            uint32_t d = digit_of(key[i], shift);
            uint32_t r = dstart[d] + whist[warp * RADIX + d] + rank[i];
            sk[r] = key[i];
            sv[r] = val[i];
        }
    }
    __syncthreads();
    const uint32_t tile_n = (uint32_t)((n - base) < (uint64_t)SORT_TILE ? (n - base) : SORT_TILE);
    for (uint32_t j = threadIdx.x; j < tile_n; j += SORT_THREADS) {
        K k = sk[j];
        uint32_t d = digit_of(k, shift);
        uint32_t o = goff[d] + (j - dstart[d]);
        kout[o] = k;
        vout[o] = sv[j];
    }
}

template <class K>
size_t downsweep_smem()
{
    return (size_t)SORT_TILE * (sizeof(K) + sizeof(uint32_t)) + (size_t)(NWARPS * RADIX + 2 * RADIX + NWARPS) * 4;
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
    const size_t T = div_up(n ? n : 1, SORT_TILE);
    size_t b = 0;
    b += (sizeof(K) * RADIX * 4 + 255) & ~size_t(255);        // histograms
    b += 2 * ((T * RADIX * 4 + 255) & ~size_t(255));           // counts, offsets
    b += ((n * sizeof(K) + 255) & ~size_t(255)) + ((n * 4 + 255) & ~size_t(255));  // ping-pong buffer
    return b + 1024;
}

template <class K>
cudaError_t sort_pairs(Ctx& c, const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, uint64_t n)
{
    if (n == 0) return cudaSuccess;
    constexpr int P = sizeof(K);
    const uint32_t T = div_up(n, SORT_TILE);
    Arena& A = c.h->arena;
    uint32_t* hist = A.take<uint32_t>(P * RADIX);
    uint32_t* counts = A.take<uint32_t>((size_t)T * RADIX);
    uint32_t* offsets = A.take<uint32_t>((size_t)T * RADIX);
    K* tk = A.take<K>(n);
    uint32_t* tv = A.take<uint32_t>(n);
    if (!hist || !counts || !offsets || !tk || !tv) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaMemsetAsync(hist, 0, P * RADIX * 4, c.st);
    if (e) return e;
    int nsm = 148;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c.h->device);
    uint32_t hg = div_up(n, 256);
    if (hg > (uint32_t)nsm * 8) hg = nsm * 8;
    e = launch(c, K_SORT_HIST, dim3(hg), dim3(256), 0, k_hist_all<K>, kin, n, hist);
    if (e) return e;
    const size_t smem = downsweep_smem<K>();
    e = cudaFuncSetAttribute(k_downsweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e) return e;
    const K* sk = kin;
    const uint32_t* sv = vin;
    for (int p = 0; p < P; p++) {
        // the last pass writes kout; passes alternate between kout and the scratch pair
        const bool to_out = ((P - 1 - p) & 1) == 0;
        K* dk = to_out ? kout : tk;
        uint32_t* dv = to_out ? vout : tv;
        const int shift = 8 * p;
        e = launch(c, K_SORT_UP, dim3(T), dim3(SORT_THREADS), 0, k_upsweep<K>, sk, n, shift, counts, T);
        if (e) return e;
        e = launch(c, K_SORT_SCAN, dim3(RADIX), dim3(256), 0, k_scan_digits, (const uint32_t*)counts, T,
                   (const uint32_t*)(hist + p * RADIX), offsets);
        if (e) return e;
        e = launch(c, K_SORT_DOWN, dim3(T), dim3(SORT_THREADS), smem, k_downsweep<K>, sk, sv, dk, dv, n, shift,
                   (const uint32_t*)offsets, T);
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
