// flix_lookup_noalloc: the point-query path of flix_lookup with its scratch memory (sort buffers,
// digit counts, per-query buckets) taken from one fixed array compiled into the library instead of
// the handle's scratch arena, so the call itself allocates no device memory.
//
// Who needs it: callers that run where device allocation is unavailable or forbidden at call
// time -- code executing inside a pre-reserved memory budget (a serving process whose allocator
// has already handed all device memory to its own pools), real-time paths that may not block on
// cudaMalloc's implicit synchronisation, or hosts that install a custom allocator the library
// cannot see.  The handle itself (node pool, MKBA) is still created beforehand by flix_create.
//
// The fixed array is a file-scope __device__ variable: every GPU that loads the library reserves
// FLIX_NOALLOC_SCRATCH_BYTES on it until the process exits.  Host code cannot use the variable's
// name as a device address; the address is looked up once per device with cudaGetSymbolAddress
// the first time the entry point runs on that device (with that device current), so that first
// call must not happen while a stream is being captured.
//
// All calls share the one array and each call overwrites it; the kernels clear what must start
// at zero (the radix-sort histograms) themselves.  Calls whose work overlaps on the GPU (other
// streams, other threads, other handles on the same device) race on the array and must be
// serialised by the caller.
#include <mutex>

#include "flix_internal.cuh"

namespace flix {
namespace {

constexpr size_t kNoallocBytes = FLIX_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[kMaxDevices] = {};

// Device address of g_noalloc_scratch on device `dev` (looked up once, with `dev` current).
cudaError_t noalloc_address(int dev, void** out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        int cur = -1;
        cudaError_t e = cudaGetDevice(&cur);
        if (e != cudaSuccess) return e;
        if (cur != dev && (e = cudaSetDevice(dev)) != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (cur != dev) cudaSetDevice(cur);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

template <class K>
size_t noalloc_need(uint64_t n, uint64_t nb)
{
    return sort_scratch_bytes<K>(n) + al256(n * sizeof(K)) + al256(n * 4) * 2 + partition_scratch_bytes(nb, n);
}

template <class K>
int lookup_noalloc(flix_index* h, const K* keys, uint64_t n, K* vals_out, uint8_t* found, cudaStream_t st)
{
    const size_t need = noalloc_need<K>(n, h->nb);
    if (need > kNoallocBytes) {
        h->last_error = "flix_lookup_noalloc: " + std::to_string(n) + " keys on an index of " +
                        std::to_string(h->nb) + " buckets need " + std::to_string(need) +
                        " bytes of scratch; the fixed scratch array holds " + std::to_string(kNoallocBytes);
        return FLIX_EINVAL;
    }
    if (n == 0) return FLIX_OK;
    void* base = nullptr;
    cudaError_t e = noalloc_address(h->device, &base);
    if (e != cudaSuccess) {
        h->last_error = std::string("flix_lookup_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return FLIX_ECUDA;
    }
    // Run the flix_lookup kernels with the fixed array standing in for the handle's arena.  Per-launch
    // profiling events are not created during this call (creating them would allocate).
    Arena saved = h->arena;
    const bool prof = h->prof_on;
    h->arena.base = static_cast<char*>(base);
    h->arena.cap = kNoallocBytes;
    h->arena.used = 0;
    h->prof_on = false;
    Ctx c{h, st};
    K* sk = h->arena.take<K>(n);
    uint32_t* si = h->arena.take<uint32_t>(n);
    uint32_t* bk = h->arena.take<uint32_t>(n);
    e = cudaSuccess;
    if (!sk || !si || !bk) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = sort_pairs<K>(c, keys, nullptr, sk, si, n);
    if (e == cudaSuccess) e = partition<K>(c, static_cast<const K*>(h->mkba), h->nb, sk, n, nullptr, nullptr, bk);
    if (e == cudaSuccess) e = read_point<K>(c, FLIX_OP_LOOKUP, sk, si, n, bk, nullptr, nullptr, vals_out, found);
    h->arena = saved;
    h->prof_on = prof;
    if (e != cudaSuccess) {
        h->last_error = std::string("flix_lookup_noalloc: ") + cudaGetErrorString(e);
        cudaGetLastError();
        return FLIX_ECUDA;
    }
    return FLIX_OK;
}

}  // namespace
}  // namespace flix

extern "C" int flix_lookup_noalloc(flix_t h, const void* d_keys, uint64_t n, void* d_vals_out, uint8_t* d_found_or_null,
                                   void* stream)
{
    if (!h || (n && (!d_keys || !d_vals_out)) || n >= 0xFFFFF000ull) return FLIX_EINVAL;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (h->kw == 32)
        return flix::lookup_noalloc<uint32_t>(h, static_cast<const uint32_t*>(d_keys), n,
                                              static_cast<uint32_t*>(d_vals_out), d_found_or_null, st);
    return flix::lookup_noalloc<uint64_t>(h, static_cast<const uint64_t*>(d_keys), n,
                                          static_cast<uint64_t*>(d_vals_out), d_found_or_null, st);
}
