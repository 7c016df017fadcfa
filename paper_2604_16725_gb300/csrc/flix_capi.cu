// C ABI of the FliX index (declared in include/flix.h): handle, device memory, and the host-side
// orchestration of the kernels for each call.  Every step of every call runs in this library's
// kernels; the host only sizes launches, reads back a few words where the ABI says it
// synchronises, and manages memory.
#include <algorithm>
#include <mutex>
#include <cstdio>
#include <vector>

#include "flix_internal.cuh"

namespace flix {

const char* kKernelNames[K_NUM] = {
    "readback", "sort_hist", "sort_upsweep", "sort_scan", "sort_downsweep", "sort_onesweep", "sort_plan", "sort_pass_idle",
    "sort_finish",
    "scan_partials", "scan_top", "scan_apply",
    "partition", "read_point", "read_unsort", "range_count", "range_fill",
    "validate", "fold_flags", "fold_init", "fold_del", "fold_ins", "fold_emit", "fold_write",
    "update_count", "alloc_copy", "update_apply", "admit",
    "live_count", "gather", "cut_keys", "cut_meta", "dedupe", "stats", "fill", "split_chains", "merge_underfull",
    "update_heavy", "queue",
};

cudaError_t dev_malloc(const DevAlloc& da, void** p, size_t bytes)
{
    if (!da.alloc) return cudaMalloc(p, bytes);
    *p = da.alloc(bytes, da.ctx);
    return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}

void dev_free(const DevAlloc& da, void* p)
{
    if (!p) return;
    if (!da.free) {
        cudaFree(p);   // synchronises the device
        return;
    }
    cudaDeviceSynchronize();
    da.free(p, da.ctx);
}

cudaError_t Arena::ensure(size_t bytes)
{
    if (bytes <= cap) return cudaSuccess;
    size_t want = std::max(bytes, cap + cap / 2);
    want = (want + (1 << 20) - 1) & ~size_t((1 << 20) - 1);
    if (base) {
        dev_free(da, base);  // synchronises the device: no call still uses the arena
        base = nullptr;
        cap = 0;
    }
    cudaError_t e = dev_malloc(da, reinterpret_cast<void**>(&base), want);
    if (e) { base = nullptr; return e; }
    cap = want;
    used = 0;
    return cudaSuccess;
}

void Arena::release()
{
    dev_free(da, base);
    base = nullptr;
    cap = used = 0;
}

cudaEvent_t prof_event(flix_index* h)
{
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        h->ev_pool.push_back(e);
    }
    return h->ev_pool[h->ev_used++];
}

namespace {

__global__ void k_fill_desc(uint32_t* __restrict__ dst, uint64_t count, uint64_t top_value)
{
    grid_dep_enter();
    // dst[i] = top_value + count - 1 - i: the smallest id ends on top of the stack
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = (uint32_t)(top_value + count - 1 - i);
}

int fail(flix_index* h, cudaError_t e)
{
    if (h) {
        h->last_error = cudaGetErrorString(e);
        cudaGetLastError();
    }
    return e == cudaErrorMemoryAllocation ? FLIX_ENOMEM : FLIX_ECUDA;
}

#define CK(...)                                    \
    do {                                           \
        cudaError_t _e = (__VA_ARGS__);            \
        if (_e != cudaSuccess) return fail(h, _e); \
    } while (0)

size_t al(size_t b) { return (b + 255) & ~size_t(255); }

// Small read-backs go through a kernel that stores into the mapped pinned buffer hpin, not through
// a copy engine: a synchronising call then never waits behind bulk transfers that other streams
// have queued on the copy engines.
struct ReadItems {
    const void* src[8];
    uint32_t bytes[8];
    uint32_t n;
    uint32_t word0;
    uint64_t* dst;
};

__global__ void k_readback(ReadItems it)
{
    grid_dep_enter();
    for (uint32_t i = 0; i < it.n; i++) {
        const unsigned char* s = static_cast<const unsigned char*>(it.src[i]);
        uint64_t v = 0;
        for (uint32_t b = 0; b < it.bytes[i]; b++) v |= (uint64_t)s[b] << (8 * b);
        it.dst[it.word0 + i] = v;
    }
    __threadfence_system();
}

// Read up to 8 device values (4 or 8 bytes each, zero-extended) into h->hpin[word0 + i] and
// synchronise the stream.
int readback_impl(flix_index* h, cudaStream_t st, uint32_t word0,
                  std::initializer_list<std::pair<const void*, size_t>> items)
{
    ReadItems it{};
    for (auto& x : items) {
        if (it.n == 8) return fail(h, cudaErrorInvalidValue);
        it.src[it.n] = x.first;
        it.bytes[it.n] = (uint32_t)x.second;
        it.n++;
    }
    it.word0 = word0;
    it.dst = h->hpin_dev;
    Ctx c{h, st};
    CK(launch(c, K_READBACK, dim3(1), dim3(1), 0, k_readback, it));
    CK(cudaStreamSynchronize(st));
    return FLIX_OK;
}

int readback(flix_index* h, cudaStream_t st, std::initializer_list<std::pair<const void*, size_t>> items)
{
    return readback_impl(h, st, 0, items);
}

// Device error word: read, clear, report.
int check_err(flix_index* h, cudaStream_t st)
{
    int r = readback_impl(h, st, 63, {{h->err, 4}});
    if (r) return r;
    const uint32_t v = (uint32_t)h->hpin[63];
    if (v) {
        { Ctx c0{h, st}; CK(fill_bytes(c0, h->err, 0, 4)); }
        if (v == ERR_TIMEOUT) {
            h->last_error = "a bounded device-side wait gave up (persistent queue)";
            return FLIX_ETIMEDOUT;
        }
        h->last_error = "device consistency check failed (code " + std::to_string(v) + ")";
        return FLIX_EINTERNAL;
    }
    return FLIX_OK;
}

// The second key/value node array of the one-pass restructure (sized like the pool).
void pool_free_second(flix_index* h)
{
    dev_free(h->da, h->keys2);
    dev_free(h->da, h->vals2);
    h->keys2 = h->vals2 = nullptr;
    h->cap2 = 0;
    dev_free(h->da, h->mkba2);
    dev_free(h->da, h->head2);
    h->mkba2 = nullptr;
    h->head2 = nullptr;
    h->capb2 = 0;
}

void pool_free(flix_index* h)
{
    void* ptrs[] = {h->keys, h->vals, h->size, h->bound, h->next, h->tnode, h->mkba, h->head, h->free_ids};
    for (void* p : ptrs) dev_free(h->da, p);
    h->keys = h->vals = h->bound = h->mkba = nullptr;
    h->size = h->next = h->tnode = h->head = h->free_ids = nullptr;
    h->cap = 0;
    pool_free_second(h);
}

struct PoolArrays {
    void *keys, *vals, *bound, *mkba;
    uint32_t *size, *next, *tnode, *head, *free_ids;
};

cudaError_t pool_alloc_arrays(flix_index* h, uint64_t cap, PoolArrays& a)
{
    memset(&a, 0, sizeof(a));
    const size_t ks = h->ks;
    const DevAlloc& da = h->da;
    cudaError_t e;
    if ((e = dev_malloc(da, &a.keys, cap * h->NS * ks))) return e;
    if ((e = dev_malloc(da, &a.vals, cap * h->NS * ks))) return e;
    if ((e = dev_malloc(da, &a.bound, cap * ks))) return e;
    if ((e = dev_malloc(da, &a.mkba, cap * ks))) return e;
    if ((e = dev_malloc(da, reinterpret_cast<void**>(&a.size), cap * 4))) return e;
    if ((e = dev_malloc(da, reinterpret_cast<void**>(&a.next), cap * 4))) return e;
    if ((e = dev_malloc(da, reinterpret_cast<void**>(&a.tnode), cap * 4))) return e;
    if ((e = dev_malloc(da, reinterpret_cast<void**>(&a.head), cap * 4))) return e;
    if ((e = dev_malloc(da, reinterpret_cast<void**>(&a.free_ids), cap * 4))) return e;
    return cudaSuccess;
}

void pool_free_arrays(flix_index* h, PoolArrays& a)
{
    void* ptrs[] = {a.keys, a.vals, a.bound, a.mkba, a.size, a.next, a.tnode, a.head, a.free_ids};
    for (void* p : ptrs) dev_free(h->da, p);
}

void pool_adopt(flix_index* h, const PoolArrays& a, uint64_t cap)
{
    h->keys = a.keys; h->vals = a.vals; h->bound = a.bound; h->mkba = a.mkba;
    h->size = a.size; h->next = a.next; h->tnode = a.tnode; h->head = a.head; h->free_ids = a.free_ids;
    h->cap = cap;
}

// Fresh pool of `cap` nodes whose contents the caller rebuilds.
int pool_reset(flix_index* h, uint64_t cap)
{
    cudaDeviceSynchronize();
    pool_free(h);
    PoolArrays a;
    cudaError_t e = pool_alloc_arrays(h, cap, a);
    if (e) { pool_free_arrays(h, a); return fail(h, e); }
    pool_adopt(h, a, cap);
    return FLIX_OK;
}

// Grow the pool to new_cap nodes, keeping every node, bucket and free id; the new ids go on top of
// the free stack, smallest id on top.
int pool_grow(flix_index* h, cudaStream_t st, uint64_t new_cap)
{
    if (new_cap > 0xFFFFFFF0ull) return FLIX_ENOMEM;
    PoolArrays a;
    cudaError_t e = pool_alloc_arrays(h, new_cap, a);
    if (e) { pool_free_arrays(h, a); cudaGetLastError(); return FLIX_ENOMEM; }
    const uint64_t c = h->cap;
    const size_t ks = h->ks;
    CK(cudaMemcpyAsync(a.keys, h->keys, c * h->NS * ks, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.vals, h->vals, c * h->NS * ks, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.bound, h->bound, c * ks, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.mkba, h->mkba, h->nb * ks, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.size, h->size, c * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.next, h->next, c * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.tnode, h->tnode, c * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.head, h->head, h->nb * 4, cudaMemcpyDeviceToDevice, st));
    CK(cudaMemcpyAsync(a.free_ids, h->free_ids, h->free_top * 4, cudaMemcpyDeviceToDevice, st));
    const uint64_t added = new_cap - c;
    Ctx cx{h, st};
    CK(launch(cx, K_FILL, dim3(div_up(added, 256)), dim3(256), 0, k_fill_desc, a.free_ids + h->free_top, added, c));
    CK(cudaStreamSynchronize(st));
    pool_free(h);
    pool_adopt(h, a, new_cap);
    h->free_top += added;
    return FLIX_OK;
}

bool valid_ns(uint32_t ns) { return ns >= 2 && ns <= 128 && (ns % 2) == 0; }

uint64_t default_cap(flix_index* h, uint64_t nb)
{
    // an explicit pool size is honoured (it must at least hold one node per bucket)
    if (h->cfg.pool_nodes) return std::max<uint64_t>(h->cfg.pool_nodes, nb);
    return std::max<uint64_t>(2 * nb + 64, 1024);
}

// ------------------------------------------------------------------------------------------------
// Calls, templated on the key type
// ------------------------------------------------------------------------------------------------

template <class K>
int do_bulk_load(flix_index* h, const K* keys, const K* vals, uint64_t n, cudaStream_t st)
{
    Ctx c{h, st};
    const size_t ks = sizeof(K);
    CK(h->arena.ensure(sort_scratch_bytes<K>(n) + al(n * ks) * 3 + al(n * 4) * 3 + al(n * 4) + (1 << 20)));
    h->arena.reset();
    uint32_t* status = h->arena.take<uint32_t>(16);
    K* sk = h->arena.take<K>(n + 1);
    uint32_t* si = h->arena.take<uint32_t>(n + 1);
    K* ok = h->arena.take<K>(n + 1);
    K* ov = h->arena.take<K>(n + 1);
    CK(fill_bytes(c, status, 0, 64));
    if (n) {
        CK(validate_inserts<K>(c, nullptr, keys, n, status));
        CK(sort_pairs<K>(c, keys, nullptr, sk, si, n));
        CK(dedupe_sorted<K>(c, sk, si, vals, n, ok, ov, status + 1));
    }
    int r = readback(h, st, {{status, 4}, {status + 1, 4}});
    if (r) return r;
    uint32_t flag = (uint32_t)(h->hpin[0] & 0xFFFFFFFFu);
    uint64_t nd = n ? (h->hpin[1] & 0xFFFFFFFFu) : 0;
    if (flag & ERR_BADKEY) return FLIX_EINVAL;
    const uint64_t nb_new = nd ? (nd + h->p - 1) / h->p : 1;
    const uint64_t want = default_cap(h, nb_new);
    if (h->cap < nb_new || (h->cfg.pool_nodes == 0 && h->cap < want)) {
        // keep the scratch pair alive: the pool is separate memory
        int rr = pool_reset(h, want);
        if (rr) return rr;
    }
    CK(cut_buckets<K>(c, ok, ov, nd, nb_new));
    return check_err(h, st);
}

template <class K>
int do_read_point(flix_index* h, int mode, const K* keys, uint64_t n, K* keys_out, K* vals_out, uint8_t* found,
                  cudaStream_t st)
{
    if (n == 0) return FLIX_OK;
    Ctx c{h, st};
    CK(h->arena.ensure(sort_scratch_bytes<K>(n) + al(n * sizeof(K)) + al(n * 4) * 2 + partition_scratch_bytes(h->nb, n) +
                       read_point_scratch_bytes<K>(n) + (1 << 16)));
    h->arena.reset();
    K* sk = h->arena.take<K>(n);
    uint32_t* si = h->arena.take<uint32_t>(n);
    uint32_t* bk = h->arena.take<uint32_t>(n);
    CK(sort_pairs<K>(c, keys, nullptr, sk, si, n));
    CK(partition<K>(c, static_cast<const K*>(h->mkba), h->nb, sk, n, nullptr, nullptr, bk));
    CK(read_point<K>(c, mode, sk, si, n, bk, nullptr, keys_out, vals_out, found));
    return FLIX_OK;
}

template <class K>
int do_sort_only(flix_index* h, const K* keys, uint64_t n, K* keys_out, uint32_t* pos_out, cudaStream_t st)
{
    if (n == 0) return FLIX_OK;
    Ctx c{h, st};
    CK(h->arena.ensure(sort_scratch_bytes<K>(n) + (1 << 16)));
    h->arena.reset();
    CK(sort_pairs<K>(c, keys, nullptr, keys_out, pos_out, n));
    return check_err(h, st);
}

template <class K>
int do_range(flix_index* h, const K* lo, const K* hi, uint64_t n, uint64_t* roff, K* rk, K* rv, uint64_t rcap,
             uint64_t* h_total, cudaStream_t st)
{
    Ctx c{h, st};
    if (n == 0) {
        CK(fill_bytes(c, roff, 0, 8));
        if (h_total) *h_total = 0;
        return FLIX_OK;
    }
    CK(h->arena.ensure(sort_scratch_bytes<K>(n) + al(n * sizeof(K)) + al(n * 4) * 5 + al(n * 8) +
                       scan_scratch_bytes<uint64_t>(n) + partition_scratch_bytes(h->nb, n) + (1 << 16)));
    h->arena.reset();
    K* sk = h->arena.take<K>(n);
    uint32_t* si = h->arena.take<uint32_t>(n);
    uint32_t* sb = h->arena.take<uint32_t>(n);
    uint32_t* sn = h->arena.take<uint32_t>(n);
    uint32_t* sp = h->arena.take<uint32_t>(n);
    uint64_t* cnt = h->arena.take<uint64_t>(n);
    uint32_t* bk = h->arena.take<uint32_t>(n);
    CK(sort_pairs<K>(c, lo, nullptr, sk, si, n));
    CK(partition<K>(c, static_cast<const K*>(h->mkba), h->nb, sk, n, nullptr, nullptr, bk));
    CK(range_count<K>(c, sk, si, n, bk, nullptr, hi, sb, sn, sp, cnt));
    CK(scan_exclusive<uint64_t, uint64_t>(c, cnt, roff, n));
    int r = readback(h, st, {{roff + n, 8}});
    if (r) return r;
    const uint64_t total = h->hpin[0];
    if (h_total) *h_total = total;
    if (total > rcap) return FLIX_ENOMEM;
    if (total) CK(range_fill<K>(c, si, n, nullptr, sb, sn, sp, roff, rk, rv, false));
    return FLIX_OK;
}

// Scratch bytes of one batch of n ops on nb buckets.
template <class K>
size_t batch_scratch_bytes(uint64_t n, uint64_t nb)
{
    return sort_scratch_bytes<K>(n) + al(n * sizeof(K)) * 3 + al(n * 4) * 16 + al(n * 8) * 2 + al((nb + 1) * 4) * 2 +
           al((nb + 1) * 8) * 2 + al(nb + 1) + scan_scratch_bytes<uint64_t>(n) * 4 +
           scan_scratch_bytes<uint64_t>(nb + 1) * 2 + al(2 * n * 4 + 64) + partition_scratch_bytes(nb, n) * 2 +
           heavy_scratch_bytes(n) + (1 << 16);
}

size_t split_scratch_bytes(uint64_t nb);
template <class K>
int split_chains_impl(flix_index* h, uint32_t max_chain, const uint32_t* uoff, uint64_t* added, cudaStream_t st);

// Reads of a mixed batch (snapshot), then its updates.  hom_op != 0: homogeneous insert/delete.
// sync: read back the node demand and range total, decide admission (and pool growth) on the host
// and report errors as return codes.  !sync: no host round trip; the admit kernel decides on the
// device and writes d_status (flags, range total, need, free nodes before the batch).
template <class K>
int do_batch(flix_index* h, const uint8_t* ops, int hom_op, const K* keys, const K* aux, uint64_t n, K* keys_out,
             K* vals_out, uint8_t* found, uint64_t* roff_user, K* rk, K* rv, uint64_t rcap, uint64_t* h_rtotal,
             uint64_t* d_status, bool sync, cudaStream_t st)
{
    if (h_rtotal) *h_rtotal = 0;
    if (n == 0) {
        Ctx c0{h, st};
        if (roff_user) CK(fill_bytes(c0, roff_user, 0, 8));
        if (d_status) CK(fill_bytes(c0, d_status, 0, 4 * sizeof(uint64_t)));
        return FLIX_OK;
    }
    Ctx c{h, st};
    const uint64_t nb = h->nb;
    const bool mixed = hom_op == 0;
    const bool split_after = sync && h->cfg.split_chains_over;
    const size_t need_bytes = batch_scratch_bytes<K>(n, nb) + (split_after ? split_scratch_bytes(nb) : 0);
    if (sync) {
        CK(h->arena.ensure(need_bytes));
    } else if (h->arena.cap < need_bytes) {
        h->last_error = "scratch not reserved for a batch of " + std::to_string(n) + " ops (call flix_reserve)";
        return FLIX_ENOMEM;
    }
    h->arena.reset();
    Arena& A = h->arena;
    uint32_t* status = A.take<uint32_t>(16);
    K* sk = A.take<K>(n);
    uint32_t* si = A.take<uint32_t>(n);
    CK(fill_bytes(c, status, 0, 64));
    CK(validate_inserts<K>(c, mixed ? ops : nullptr, keys, mixed || hom_op == FLIX_OP_INSERT ? n : 0, status));
    CK(sort_pairs<K>(c, keys, nullptr, sk, si, n));
    // A mixed batch's reads (on st) and the preparation of its updates (fold, partition, count pass,
    // on the handle's side stream) both only read the pre-batch state, so they run side by side; the
    // side stream joins st before admission.  Scratch for both is taken here, on the host, in order.
    Ctx cu{h, mixed ? h->side_st : st};
    // on every return between the fork and the join (an error), the side stream still rejoins st, so
    // that no work of this call runs past it into the next call's use of the scratch
    struct Rejoin {
        flix_index* h;
        cudaStream_t st;
        bool armed = false;
        ~Rejoin()
        {
            if (!armed) return;
            cudaEventRecord(h->join_ev, h->side_st);
            cudaStreamWaitEvent(st, h->join_ev, 0);
        }
    } rejoin{h, st};
    if (mixed) {
        CK(cudaEventRecord(h->fork_ev, st));
        CK(cudaStreamWaitEvent(h->side_st, h->fork_ev, 0));
        rejoin.armed = true;
    }
    uint64_t* roff = roff_user;
    uint32_t *sb = nullptr, *sn = nullptr, *sp = nullptr;
    if (mixed) {
        uint32_t* bk = A.take<uint32_t>(n);
        CK(partition<K>(c, static_cast<const K*>(h->mkba), nb, sk, n, nullptr, nullptr, bk));
        CK(read_point<K>(c, 0, sk, si, n, bk, ops, keys_out, vals_out, found));
        if (!roff) roff = A.take<uint64_t>(n + 1);
        sb = A.take<uint32_t>(n);
        sn = A.take<uint32_t>(n);
        sp = A.take<uint32_t>(n);
        uint64_t* cnt = A.take<uint64_t>(n);
        CK(range_count<K>(c, sk, si, n, bk, ops, aux, sb, sn, sp, cnt));
        CK(scan_exclusive<uint64_t, uint64_t>(c, cnt, roff, n));
    }
    // updates: net effect per key, bucket partition, node demand
    K* ukey = A.take<K>(n);
    uint32_t* uop = A.take<uint32_t>(n);
    K* uval = A.take<K>(n);
    uint32_t* udev = status + 2;
    uint32_t* uoff = A.take<uint32_t>(nb + 1);
    uint64_t* nf = A.take<uint64_t>(nb + 1);
    uint64_t* nf_off = A.take<uint64_t>(nb + 1);
    uint8_t* allgone = A.take<uint8_t>(nb + 1);
    const uint64_t alloc_cap = 2 * n + 16;   // a batch of U distinct updates allocates at most 2U nodes
    uint32_t* alloc_ids = A.take<uint32_t>(alloc_cap);
    if (!ukey || !uop || !uval || !uoff || !nf || !nf_off || !allgone || !alloc_ids) return FLIX_ENOMEM;
    CK(fold_updates<K>(cu, sk, si, n, ops, hom_op, aux, ukey, uop, uval, udev));
    CK(partition<K>(cu, static_cast<const K*>(h->mkba), nb, ukey, n, udev, uoff, nullptr));
    const HeavyList hl = heavy_list(cu, n);
    if (!hl.list || !hl.n) return FLIX_ENOMEM;
    CK(update_count<K>(cu, ukey, uop, uval, uoff, nf, allgone, hl));
    CK(scan_exclusive<uint64_t, uint64_t>(cu, nf, nf_off, nb));
    if (mixed) {
        rejoin.armed = false;
        CK(cudaEventRecord(h->join_ev, h->side_st));
        CK(cudaStreamWaitEvent(st, h->join_ev, 0));
    }
    const uint64_t* nf_total = nf_off + nb;
    const uint64_t* rtot_dev = (mixed && roff) ? roff + n : nullptr;
    uint64_t need = 0, freed = 0, rtotal = 0, heavy_nodes = 1;   // async: the heavy kernel always runs
    if (sync) {
        int r = readback(h, st, {{status, 4}, {nf_total, 8}, {rtot_dev ? (const void*)rtot_dev : (const void*)status, 8},
                                 {&h->dstate->free_top, 8}, {hl.n, 4}});
        if (r) return r;
        const uint32_t flag = (uint32_t)(h->hpin[0] & 0xFFFFFFFFu);
        need = h->hpin[1] & 0xFFFFFFFFull;
        freed = h->hpin[1] >> 32;
        rtotal = rtot_dev ? h->hpin[2] : 0;
        h->free_top = h->hpin[3];
        heavy_nodes = h->hpin[4];
        if (flag & ERR_BADKEY) return FLIX_EINVAL;
        if (h_rtotal) *h_rtotal = rtotal;
        if (mixed && rtotal > rcap) return FLIX_ENOMEM;
        if (need > h->free_top) {
            if (!h->cfg.grow) return FLIX_ENOMEM;
            uint64_t nc = std::max<uint64_t>(h->cap * 2, h->cap + (need - h->free_top) + 1024);
            int g = pool_grow(h, st, nc);
            if (g) return g;
            CK(set_free_top(c, h->free_top));
        }
    }
    CK(admit(c, nf_total, status, rtot_dev, mixed ? rcap : 0, d_status));
    if (mixed && (!sync || rtotal)) CK(range_fill<K>(c, si, n, ops, sb, sn, sp, roff, rk, rv, true));
    CK(alloc_copy(c, h->free_ids, alloc_ids, alloc_cap));
    CK(update_apply<K>(c, ukey, uop, uval, uoff, nf_off, allgone, alloc_ids));
    if (heavy_nodes) CK(update_heavy<K>(c, ukey, uop, uval, nf_off, alloc_ids, hl));
    CK(commit(c));
    if (sync) h->free_top = h->free_top - need + freed;
    // chain maintenance in the buckets the batch touched: merge underfull neighbours (only if the
    // batch was admitted), then split chains that grew too long (synchronous batches only)
    if (h->cfg.merge_underfull) CK(merge_underfull<K>(c, uoff, 1, nullptr));
    if (split_after) {
        int r = split_chains_impl<K>(h, h->cfg.split_chains_over, uoff, nullptr, st);
        if (r) return r;
    }
    if (sync && h->cfg.merge_underfull) {
        int r = readback(h, st, {{&h->dstate->free_top, 8}});
        if (r) return r;
        h->free_top = h->hpin[0];
    }
    return FLIX_OK;
}

// Scratch for batches up to batch_max ops and at least free_nodes_min free nodes (synchronises).
template <class K>
int do_reserve(flix_index* h, uint64_t batch_max, uint64_t free_nodes_min, cudaStream_t st)
{
    Ctx c{h, st};
    CK(h->arena.ensure(batch_scratch_bytes<K>(batch_max, std::max<uint64_t>(h->cap, h->nb))));
    int r = readback(h, st, {{&h->dstate->free_top, 8}});
    if (r) return r;
    h->free_top = h->hpin[0];
    if (h->free_top < free_nodes_min) {
        int g = pool_grow(h, st, h->cap + (free_nodes_min - h->free_top) + 1024);
        if (g) return g;
        CK(set_free_top(c, h->free_top));
    }
    CK(cudaStreamSynchronize(st));
    return FLIX_OK;
}

// Makes the second key/value node arrays of the one-pass restructure as large as the pool.
int ensure_second(flix_index* h)
{
    if (h->cap2 == h->cap) return FLIX_OK;
    pool_free_second(h);
    CK(dev_malloc(h->da, &h->keys2, h->cap * h->NS * h->ks));
    CK(dev_malloc(h->da, &h->vals2, h->cap * h->NS * h->ks));
    h->cap2 = h->cap;
    return FLIX_OK;
}

// Makes the second MKBA and bucket-head arrays of the elastic split as large as the pool (a split
// never makes more buckets than there are nodes in chains).
int ensure_second_buckets(flix_index* h)
{
    if (h->capb2 == h->cap) return FLIX_OK;
    dev_free(h->da, h->mkba2);
    dev_free(h->da, h->head2);
    h->mkba2 = nullptr;
    h->head2 = nullptr;
    h->capb2 = 0;
    CK(dev_malloc(h->da, &h->mkba2, h->cap * h->ks));
    CK(dev_malloc(h->da, reinterpret_cast<void**>(&h->head2), h->cap * 4));
    h->capb2 = h->cap;
    return FLIX_OK;
}

size_t split_scratch_bytes(uint64_t nb) { return al((nb + 1) * 8) * 2 + scan_scratch_bytes<uint64_t>(nb + 1); }

// Elastic split of the buckets selected by uoff (all when null) whose chains exceed max_chain.  Takes
// its scratch from the arena as it stands (a batch calls it with its own scratch still in use).
template <class K>
int split_chains_impl(flix_index* h, uint32_t max_chain, const uint32_t* uoff, uint64_t* added, cudaStream_t st)
{
    Ctx c{h, st};
    const uint64_t nb = h->nb;
    uint64_t* cnt = h->arena.take<uint64_t>(nb + 1);
    uint64_t* boff = h->arena.take<uint64_t>(nb + 1);
    if (!cnt || !boff) return FLIX_ENOMEM;
    CK(split_count<K>(c, max_chain, uoff, cnt));
    CK(scan_exclusive<uint64_t, uint64_t>(c, cnt, boff, nb));
    int r = readback(h, st, {{boff + nb, 8}});
    if (r) return r;
    const uint64_t nb_new = h->hpin[0];
    if (added) *added = nb_new - nb;
    if (nb_new == nb) return check_err(h, st);
    if (nb_new > h->cap) return FLIX_EINTERNAL;
    r = ensure_second_buckets(h);
    if (r) return r;
    CK(split_write<K>(c, cnt, boff, static_cast<K*>(h->mkba2), h->head2));
    std::swap(h->mkba, h->mkba2);
    std::swap(h->head, h->head2);
    h->nb = nb_new;
    return check_err(h, st);
}

template <class K>
int do_split_chains(flix_index* h, uint32_t max_chain, uint64_t* added, cudaStream_t st)
{
    CK(h->arena.ensure(split_scratch_bytes(h->nb) + (1 << 16)));
    h->arena.reset();
    return split_chains_impl<K>(h, max_chain, nullptr, added, st);
}

template <class K>
int do_merge_underfull(flix_index* h, uint64_t* freed, cudaStream_t st)
{
    Ctx c{h, st};
    CK(h->arena.ensure(1 << 16));
    h->arena.reset();
    unsigned long long* cnt = h->arena.take<unsigned long long>(1);
    CK(fill_bytes(c, cnt, 0, 8));
    CK(merge_underfull<K>(c, nullptr, 0, cnt));
    int r = readback(h, st, {{cnt, 8}, {&h->dstate->free_top, 8}});
    if (r) return r;
    if (freed) *freed = h->hpin[0];
    h->free_top = h->hpin[1];
    return check_err(h, st);
}

// Restructure with the nodes put in chain order by their maxKeys (some chain is long).
template <class K>
int restructure_by_nodes(flix_index* h, cudaStream_t st)
{
    Ctx c{h, st};
    size_t extra = 0;
    for (int attempt = 0; attempt < 3; attempt++) {
        CK(h->arena.ensure(node_order_scratch_bytes<K>(h->cap) + extra + (1 << 16)));
        h->arena.reset();
        NodeOrder<K> no;
        int r = node_order<K>(c, no);
        if (r) return r;
        r = readback(h, st, {{no.noff + no.m, 8}});
        if (r) return r;
        const uint64_t n = h->hpin[0];
        const uint64_t nb_new = n ? (n + h->p - 1) / h->p : 1;
        if (h->cfg.restructure_in_one_pass && h->cap >= nb_new) {
            r = ensure_second(h);
            if (r) return r;
            CK(gather_nodes_cut<K>(c, no, nb_new, static_cast<K*>(h->keys2), static_cast<K*>(h->vals2)));
            std::swap(h->keys, h->keys2);
            std::swap(h->vals, h->vals2);
            CK(cut_buckets<K>(c, nullptr, nullptr, n, nb_new));
            return check_err(h, st);
        }
        K* tk = h->arena.take<K>(n + 1);
        K* tv = h->arena.take<K>(n + 1);
        if (!tk || !tv) {
            extra = al((n + 1) * sizeof(K)) * 2;
            continue;   // the arena moves: order the nodes again
        }
        CK(gather_nodes<K>(c, no, tk, tv));
        if (h->cap < nb_new) {
            CK(cudaStreamSynchronize(st));
            int rr = pool_reset(h, default_cap(h, nb_new));
            if (rr) return rr;
        }
        CK(cut_buckets<K>(c, tk, tv, n, nb_new));
        return check_err(h, st);
    }
    return FLIX_EINTERNAL;
}

template <class K>
int do_restructure(flix_index* h, cudaStream_t st)
{
    Ctx c{h, st};
    const uint64_t nb = h->nb;
    for (int attempt = 0; attempt < 3; attempt++) {
        CK(h->arena.ensure(al((nb + 1) * 8) * 2 + scan_scratch_bytes<uint64_t>(nb + 1) + (1 << 16)));
        h->arena.reset();
        uint64_t* cnt = h->arena.take<uint64_t>(nb + 1);
        uint64_t* goff = h->arena.take<uint64_t>(nb + 1);
        uint32_t* long_flag = h->arena.take<uint32_t>(1);
        CK(live_count<K>(c, cnt, long_flag));
        CK(scan_exclusive<uint64_t, uint64_t>(c, cnt, goff, nb));
        int r = readback(h, st, {{goff + nb, 8}, {long_flag, 4}});
        if (r) return r;
        if (h->hpin[1]) return restructure_by_nodes<K>(h, st);
        const uint64_t n = h->hpin[0];
        const size_t need = h->arena.used + al(n * sizeof(K)) * 2 + (1 << 16);
        if (need > h->arena.cap) {
            CK(h->arena.ensure(need + al((nb + 1) * 8) * 2));
            continue;  // the arena moved: recount
        }
        const uint64_t nb_new = n ? (n + h->p - 1) / h->p : 1;
        if (h->cfg.restructure_in_one_pass && h->cap >= nb_new) {
            // every live pair goes straight to its place in the second node array, which then
            // becomes the pool's key/value array
            r = ensure_second(h);
            if (r) return r;
            CK(gather_cut<K>(c, goff, n, nb_new, static_cast<K*>(h->keys2), static_cast<K*>(h->vals2)));
            std::swap(h->keys, h->keys2);
            std::swap(h->vals, h->vals2);
            CK(cut_buckets<K>(c, nullptr, nullptr, n, nb_new));
            return check_err(h, st);
        }
        K* tk = h->arena.take<K>(n + 1);
        K* tv = h->arena.take<K>(n + 1);
        CK(gather_live<K>(c, goff, tk, tv));
        if (h->cap < nb_new) {
            // the gathered pairs live in the arena, so the pool can be replaced
            CK(cudaStreamSynchronize(st));
            int rr = pool_reset(h, default_cap(h, nb_new));
            if (rr) return rr;
        }
        CK(cut_buckets<K>(c, tk, tv, n, nb_new));
        return check_err(h, st);
    }
    return FLIX_EINTERNAL;
}

template <class K>
int do_export(flix_index* h, K* dk, K* dv, uint64_t cap_out, uint64_t* h_n, cudaStream_t st)
{
    Ctx c{h, st};
    const uint64_t nb = h->nb;
    CK(h->arena.ensure(al((nb + 1) * 8) * 2 + scan_scratch_bytes<uint64_t>(nb + 1) + (1 << 16)));
    h->arena.reset();
    uint64_t* cnt = h->arena.take<uint64_t>(nb + 1);
    uint64_t* goff = h->arena.take<uint64_t>(nb + 1);
    uint32_t* long_flag = h->arena.take<uint32_t>(1);
    CK(live_count<K>(c, cnt, long_flag));
    CK(scan_exclusive<uint64_t, uint64_t>(c, cnt, goff, nb));
    int r = readback(h, st, {{goff + nb, 8}, {long_flag, 4}});
    if (r) return r;
    if (h->hpin[1]) {
        CK(h->arena.ensure(node_order_scratch_bytes<K>(h->cap) + (1 << 16)));
        h->arena.reset();
        NodeOrder<K> no;
        r = node_order<K>(c, no);
        if (r) return r;
        r = readback(h, st, {{no.noff + no.m, 8}});
        if (r) return r;
        if (h_n) *h_n = h->hpin[0];
        if (h->hpin[0] > cap_out) return FLIX_ENOMEM;
        CK(gather_nodes<K>(c, no, dk, dv));
    } else {
        if (h_n) *h_n = h->hpin[0];
        if (h->hpin[0] > cap_out) return FLIX_ENOMEM;
        CK(gather_live<K>(c, goff, dk, dv));
    }
    CK(cudaStreamSynchronize(st));
    return check_err(h, st);
}

template <class K>
int do_stats(flix_index* h, flix_stats_t* o, cudaStream_t st)
{
    Ctx c{h, st};
    CK(h->arena.ensure(1 << 16));
    h->arena.reset();
    uint64_t* s3 = h->arena.take<uint64_t>(4);
    CK(stats_kernel<K>(c, s3));
    int r = readback(h, st, {{s3, 8}, {s3 + 1, 8}, {s3 + 2, 8}, {&h->dstate->free_top, 8}, {s3 + 3, 8}});
    if (r) return r;
    memset(o, 0, sizeof(*o));
    o->buckets = h->nb;
    o->max_chain = h->hpin[0];
    o->live_keys = h->hpin[1];
    o->nodes_used = h->hpin[2];
    h->free_top = h->hpin[3];
    if (h->hpin[4]) {
        // a chain longer than the walk bound: count from the nodes in use instead
        CK(h->arena.ensure(node_order_scratch_bytes<K>(h->cap) + al(h->nb * 4) + al(h->cap * 4) + (1 << 16)));
        h->arena.reset();
        uint64_t* mx = h->arena.take<uint64_t>(1);
        NodeOrder<K> no;
        r = node_order<K>(c, no);
        if (r) return r;
        CK(chain_max_by_nodes<K>(c, no, mx));
        r = readback(h, st, {{mx, 8}, {no.noff + no.m, 8}});
        if (r) return r;
        o->max_chain = h->hpin[0];
        o->live_keys = h->hpin[1];
        o->nodes_used = no.m;
    }
    o->nodes_free = h->free_top;
    o->pool_nodes = h->cap;
    o->node_bytes = 2ull * h->NS * sizeof(K) + sizeof(K) + 8;
    o->used_bytes = o->nodes_used * o->node_bytes + h->nb * (sizeof(K) + 4);
    o->reserved_bytes = h->cap * (o->node_bytes + 4 + sizeof(K) + 4 + 4) + h->cap2 * h->NS * sizeof(K) * 2;
    return check_err(h, st);
}

template <class K>
int do_dump(flix_index* h, uint64_t* counts, K* mkba, uint32_t* chain_len, uint32_t* node_size, K* node_bound,
            K* keys, K* vals, cudaStream_t st)
{
    CK(cudaStreamSynchronize(st));
    const uint64_t cap = h->cap, nb = h->nb, NS = h->NS;
    std::vector<K> hk(cap * NS), hv(cap * NS), hb(cap), hm(nb);
    std::vector<uint32_t> hs(cap), hn(cap), hh(nb);
    CK(cudaMemcpy(hs.data(), h->size, cap * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hn.data(), h->next, cap * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hh.data(), h->head, nb * 4, cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hb.data(), h->bound, cap * sizeof(K), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hm.data(), h->mkba, nb * sizeof(K), cudaMemcpyDeviceToHost));
    const bool full = keys != nullptr;
    if (full) {
        CK(cudaMemcpy(hk.data(), h->keys, cap * NS * sizeof(K), cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(hv.data(), h->vals, cap * NS * sizeof(K), cudaMemcpyDeviceToHost));
    }
    uint64_t nn = 0, nk = 0;
    for (uint64_t b = 0; b < nb; b++) {
        uint32_t cl = 0;
        for (uint32_t x = hh[b]; x != NIL; x = hn[x]) {
            if (x >= cap || cl > cap) return FLIX_EINTERNAL;
            if (node_size) { node_size[nn] = hs[x]; node_bound[nn] = hb[x]; }
            if (full)
                for (uint32_t s = 0; s < hs[x]; s++) { keys[nk + s] = hk[x * NS + s]; vals[nk + s] = hv[x * NS + s]; }
            nn++;
            nk += hs[x];
            cl++;
        }
        if (chain_len) chain_len[b] = cl;
        if (mkba) mkba[b] = hm[b];
    }
    counts[0] = nb;
    counts[1] = nn;
    counts[2] = nk;
    return FLIX_OK;
}

#undef CK

__global__ void k_fill_bytes(uint32_t* __restrict__ dst, uint32_t pattern, uint64_t words, uint8_t* __restrict__ tail,
                             uint32_t tail_bytes, uint8_t value)
{
    grid_dep_enter();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = i0; i < words; i += stride) dst[i] = pattern;
    if (i0 < tail_bytes) tail[i0] = value;
}

__global__ void k_copy_words(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint32_t words)
{
    grid_dep_enter();
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < words) dst[i] = src[i];
}

}  // namespace

cudaError_t fill_bytes(Ctx& c, void* dst, uint8_t value, size_t bytes)
{
    if (bytes == 0) return cudaSuccess;
    // dst is at least 4-byte aligned (arena and allocations are 256-byte aligned); the tail is
    // filled byte by byte
    const uint64_t words = bytes / 4;
    const uint32_t tail = (uint32_t)(bytes - words * 4);
    const uint32_t pattern = 0x01010101u * value;
    uint32_t grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(div_up(words, 256), 1), 1216);
    return launch(c, K_FILL, dim3(grid), dim3(256), 0, k_fill_bytes, static_cast<uint32_t*>(dst), pattern, words,
                  static_cast<uint8_t*>(dst) + words * 4, tail, value);
}

cudaError_t copy_words(Ctx& c, void* dst, const void* src, uint32_t words)
{
    return launch(c, K_FILL, dim3(div_up(words, 256)), dim3(256), 0, k_copy_words, static_cast<uint32_t*>(dst),
                  static_cast<const uint32_t*>(src), words);
}

// Loads every kernel of the library on the current device (once per device per process), so that
// no call, and no replay of a captured graph, pays for loading a kernel at its first launch.
void preload_kernels()
{
    static std::mutex mu;
    static std::vector<int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lock(mu);
    for (int d : done)
        if (d == dev) return;
    cudaFuncAttributes a;
    cudaFuncGetAttributes(&a, k_fill_desc);
    cudaFuncGetAttributes(&a, k_readback);
    cudaFuncGetAttributes(&a, k_fill_bytes);
    cudaFuncGetAttributes(&a, k_copy_words);
    preload_sort_kernels();
    preload_read_kernels();
    preload_update_kernels();
    preload_build_kernels();
    preload_persist_kernels();
    done.push_back(dev);
}

int readback_at(flix_index* h, cudaStream_t st, uint32_t word0,
                std::initializer_list<std::pair<const void*, size_t>> items)
{
    return readback_impl(h, st, word0, items);
}

}  // namespace flix

using namespace flix;

#define CK(...)                                    \
    do {                                           \
        cudaError_t _e = (__VA_ARGS__);            \
        if (_e != cudaSuccess) return fail(h, _e); \
    } while (0)

#define DISPATCH(call32, call64) (h->kw == 32 ? (call32) : (call64))

static cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
static bool too_big(uint64_t n) { return n >= 0xFFFFF000ull; }

extern "C" {

void flix_config_default(flix_config* cfg, flix_keytype kt)
{
    memset(cfg, 0, sizeof(*cfg));
    cfg->key_type = kt;
    cfg->node_size = kt == FLIX_KEY_U32 ? 32 : 64;
    cfg->fill_pct = 50;
    cfg->grow = 1;
    cfg->pool_nodes = 0;
    cfg->sort_digit_bits = 8;
    cfg->restructure_in_one_pass = 1;
}

int flix_create(const flix_config* cfg, flix_t* out)
{
    if (!cfg || !out) return FLIX_EINVAL;
    *out = nullptr;
    if (cfg->key_type != FLIX_KEY_U32 && cfg->key_type != FLIX_KEY_U64) return FLIX_ETYPE;
    if (!valid_ns(cfg->node_size)) return FLIX_ETYPE;
    if (cfg->fill_pct == 0 || cfg->fill_pct > 100) return FLIX_EINVAL;
    if (cfg->sort_digit_bits != 0 && cfg->sort_digit_bits != 8) return FLIX_ENOTIMPL;
    if (cfg->sort_variant > FLIX_SORT_REDUCE_SCAN) return FLIX_EINVAL;
    if (cfg->bucket_threads != 0 && cfg->bucket_threads != 32) return FLIX_EINVAL;
    if (!cfg->dev_alloc != !cfg->dev_free) return FLIX_EINVAL;   // both or neither
    preload_kernels();
    flix_index* h = new flix_index();
    h->cfg = *cfg;
    h->kw = cfg->key_type == FLIX_KEY_U32 ? 32 : 64;
    h->ks = h->kw / 8;
    h->NS = cfg->node_size;
    h->p = std::max<uint32_t>(1, (uint32_t)(((uint64_t)h->NS * cfg->fill_pct) / 100));
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device);
    h->da.alloc = cfg->dev_alloc;
    h->da.free = cfg->dev_free;
    h->da.ctx = cfg->alloc_ctx;
    h->arena.da = h->da;
    cudaError_t e;
    if ((e = dev_malloc(h->da, reinterpret_cast<void**>(&h->err), 64)) || (e = cudaMemset(h->err, 0, 64)) ||
        (e = dev_malloc(h->da, reinterpret_cast<void**>(&h->dstate), sizeof(DevState))) ||
        (e = cudaMemset(h->dstate, 0, sizeof(DevState))) ||
        (e = cudaHostAlloc(&h->hpin, 64 * sizeof(uint64_t), cudaHostAllocMapped)) ||
        (e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->hpin_dev), h->hpin, 0)) ||
        (e = cudaEventCreateWithFlags(&h->qstage_ev, cudaEventDisableTiming)) ||
        (e = cudaStreamCreateWithFlags(&h->side_st, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&h->fork_ev, cudaEventDisableTiming)) ||
        (e = cudaEventCreateWithFlags(&h->join_ev, cudaEventDisableTiming))) {
        int r = fail(h, e);
        flix_destroy(h);
        return r;
    }
    // the empty index: one bucket with one empty node (maxBucket = KEY_MAX)
    int r = h->kw == 32 ? do_bulk_load<uint32_t>(h, nullptr, nullptr, 0, nullptr)
                        : do_bulk_load<uint64_t>(h, nullptr, nullptr, 0, nullptr);
    if (r) {
        flix_destroy(h);
        return r;
    }
    *out = h;
    return FLIX_OK;
}

int flix_destroy(flix_t h)
{
    if (!h) return FLIX_EINVAL;
    cudaDeviceSynchronize();
    pool_free(h);
    h->arena.release();
    dev_free(h->da, h->err);
    dev_free(h->da, h->dstate);
    if (h->hpin) cudaFreeHost(h->hpin);
    if (h->qstage_ev) cudaEventSynchronize(h->qstage_ev);
    if (h->qstage) cudaFreeHost(h->qstage);
    if (h->qstage_ev) cudaEventDestroy(h->qstage_ev);
    if (h->fork_ev) cudaEventDestroy(h->fork_ev);
    if (h->join_ev) cudaEventDestroy(h->join_ev);
    if (h->side_st) cudaStreamDestroy(h->side_st);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    delete h;
    return FLIX_OK;
}

int flix_bulk_load(flix_t h, const void* d_keys, const void* d_vals, uint64_t n, void* stream)
{
    if (!h || (n && (!d_keys || !d_vals)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_bulk_load<uint32_t>(h, (const uint32_t*)d_keys, (const uint32_t*)d_vals, n, S(stream)),
                    do_bulk_load<uint64_t>(h, (const uint64_t*)d_keys, (const uint64_t*)d_vals, n, S(stream)));
}

int flix_lookup(flix_t h, const void* d_keys, uint64_t n, void* d_vals_out, uint8_t* d_found, void* stream)
{
    if (!h || (n && (!d_keys || !d_vals_out)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_read_point<uint32_t>(h, FLIX_OP_LOOKUP, (const uint32_t*)d_keys, n, nullptr,
                                            (uint32_t*)d_vals_out, d_found, S(stream)),
                    do_read_point<uint64_t>(h, FLIX_OP_LOOKUP, (const uint64_t*)d_keys, n, nullptr,
                                            (uint64_t*)d_vals_out, d_found, S(stream)));
}

int flix_successor(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, void* d_vals_out, void* stream)
{
    if (!h || (n && (!d_keys || !d_keys_out || !d_vals_out)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_read_point<uint32_t>(h, FLIX_OP_SUCC, (const uint32_t*)d_keys, n, (uint32_t*)d_keys_out,
                                            (uint32_t*)d_vals_out, nullptr, S(stream)),
                    do_read_point<uint64_t>(h, FLIX_OP_SUCC, (const uint64_t*)d_keys, n, (uint64_t*)d_keys_out,
                                            (uint64_t*)d_vals_out, nullptr, S(stream)));
}

int flix_predecessor(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, void* d_vals_out, void* stream)
{
    if (!h || (n && (!d_keys || !d_keys_out || !d_vals_out)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_read_point<uint32_t>(h, FLIX_OP_PRED, (const uint32_t*)d_keys, n, (uint32_t*)d_keys_out,
                                            (uint32_t*)d_vals_out, nullptr, S(stream)),
                    do_read_point<uint64_t>(h, FLIX_OP_PRED, (const uint64_t*)d_keys, n, (uint64_t*)d_keys_out,
                                            (uint64_t*)d_vals_out, nullptr, S(stream)));
}

int flix_range(flix_t h, const void* d_lo, const void* d_hi, uint64_t n, uint64_t* d_offsets_out, void* d_keys_out,
               void* d_vals_out, uint64_t out_capacity, uint64_t* h_total_out, void* stream)
{
    if (!h || !d_offsets_out || (n && (!d_lo || !d_hi)) || too_big(n)) return FLIX_EINVAL;
    if (out_capacity && (!d_keys_out || !d_vals_out)) return FLIX_EINVAL;
    return DISPATCH(do_range<uint32_t>(h, (const uint32_t*)d_lo, (const uint32_t*)d_hi, n, d_offsets_out,
                                       (uint32_t*)d_keys_out, (uint32_t*)d_vals_out, out_capacity, h_total_out,
                                       S(stream)),
                    do_range<uint64_t>(h, (const uint64_t*)d_lo, (const uint64_t*)d_hi, n, d_offsets_out,
                                       (uint64_t*)d_keys_out, (uint64_t*)d_vals_out, out_capacity, h_total_out,
                                       S(stream)));
}

int flix_sort_pairs(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, uint32_t* d_pos_out, void* stream)
{
    if (!h || (n && (!d_keys || !d_keys_out || !d_pos_out)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_sort_only<uint32_t>(h, (const uint32_t*)d_keys, n, (uint32_t*)d_keys_out, d_pos_out, S(stream)),
                    do_sort_only<uint64_t>(h, (const uint64_t*)d_keys, n, (uint64_t*)d_keys_out, d_pos_out, S(stream)));
}

int flix_insert(flix_t h, const void* d_keys, const void* d_vals, uint64_t n, void* stream)
{
    if (!h || (n && (!d_keys || !d_vals)) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_batch<uint32_t>(h, nullptr, FLIX_OP_INSERT, (const uint32_t*)d_keys, (const uint32_t*)d_vals, n,
                                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, true,
                                       S(stream)),
                    do_batch<uint64_t>(h, nullptr, FLIX_OP_INSERT, (const uint64_t*)d_keys, (const uint64_t*)d_vals, n,
                                       nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, true,
                                       S(stream)));
}

int flix_delete(flix_t h, const void* d_keys, uint64_t n, void* stream)
{
    if (!h || (n && !d_keys) || too_big(n)) return FLIX_EINVAL;
    return DISPATCH(do_batch<uint32_t>(h, nullptr, FLIX_OP_DELETE, (const uint32_t*)d_keys, nullptr, n, nullptr,
                                       nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, true, S(stream)),
                    do_batch<uint64_t>(h, nullptr, FLIX_OP_DELETE, (const uint64_t*)d_keys, nullptr, n, nullptr,
                                       nullptr, nullptr, nullptr, nullptr, nullptr, 0, nullptr, nullptr, true, S(stream)));
}

int flix_apply(flix_t h, const uint8_t* d_ops, const void* d_keys, const void* d_aux, uint64_t n, void* d_keys_out,
               void* d_vals_out, uint8_t* d_found, uint64_t* d_range_off, void* d_range_keys, void* d_range_vals,
               uint64_t range_cap, uint64_t* h_range_total, void* stream)
{
    if (!h || (n && (!d_ops || !d_keys || !d_aux)) || too_big(n)) return FLIX_EINVAL;
    if (range_cap && (!d_range_keys || !d_range_vals)) return FLIX_EINVAL;
    return DISPATCH(
        do_batch<uint32_t>(h, d_ops, 0, (const uint32_t*)d_keys, (const uint32_t*)d_aux, n, (uint32_t*)d_keys_out,
                           (uint32_t*)d_vals_out, d_found, d_range_off, (uint32_t*)d_range_keys,
                           (uint32_t*)d_range_vals, range_cap, h_range_total, nullptr, true, S(stream)),
        do_batch<uint64_t>(h, d_ops, 0, (const uint64_t*)d_keys, (const uint64_t*)d_aux, n, (uint64_t*)d_keys_out,
                           (uint64_t*)d_vals_out, d_found, d_range_off, (uint64_t*)d_range_keys,
                           (uint64_t*)d_range_vals, range_cap, h_range_total, nullptr, true, S(stream)));
}

int flix_apply_async(flix_t h, const uint8_t* d_ops, const void* d_keys, const void* d_aux, uint64_t n,
                     void* d_keys_out, void* d_vals_out, uint8_t* d_found, uint64_t* d_range_off, void* d_range_keys,
                     void* d_range_vals, uint64_t range_cap, uint64_t* d_status, void* stream)
{
    if (!h || !d_status || (n && (!d_ops || !d_keys || !d_aux)) || too_big(n)) return FLIX_EINVAL;
    if (range_cap && (!d_range_keys || !d_range_vals)) return FLIX_EINVAL;
    return DISPATCH(
        do_batch<uint32_t>(h, d_ops, 0, (const uint32_t*)d_keys, (const uint32_t*)d_aux, n, (uint32_t*)d_keys_out,
                           (uint32_t*)d_vals_out, d_found, d_range_off, (uint32_t*)d_range_keys,
                           (uint32_t*)d_range_vals, range_cap, nullptr, d_status, false, S(stream)),
        do_batch<uint64_t>(h, d_ops, 0, (const uint64_t*)d_keys, (const uint64_t*)d_aux, n, (uint64_t*)d_keys_out,
                           (uint64_t*)d_vals_out, d_found, d_range_off, (uint64_t*)d_range_keys,
                           (uint64_t*)d_range_vals, range_cap, nullptr, d_status, false, S(stream)));
}

int flix_apply_queue(flix_t h, const flix_batch* h_batches, uint32_t count, uint32_t wait_us, uint64_t* d_flags_or,
                     void* stream)
{
    if (!h || (count && !h_batches)) return FLIX_EINVAL;
    return DISPATCH(apply_queue<uint32_t>(h, h_batches, count, wait_us, d_flags_or, S(stream)),
                    apply_queue<uint64_t>(h, h_batches, count, wait_us, d_flags_or, S(stream)));
}

int flix_reserve(flix_t h, uint64_t batch_max, uint64_t free_nodes_min, void* stream)
{
    if (!h || too_big(batch_max)) return FLIX_EINVAL;
    return DISPATCH(do_reserve<uint32_t>(h, batch_max, free_nodes_min, S(stream)),
                    do_reserve<uint64_t>(h, batch_max, free_nodes_min, S(stream)));
}

int flix_split_chains(flix_t h, uint32_t max_chain, uint64_t* h_added, void* stream)
{
    if (!h || max_chain == 0) return FLIX_EINVAL;
    return DISPATCH(do_split_chains<uint32_t>(h, max_chain, h_added, S(stream)),
                    do_split_chains<uint64_t>(h, max_chain, h_added, S(stream)));
}

int flix_merge_underfull(flix_t h, uint64_t* h_freed, void* stream)
{
    if (!h) return FLIX_EINVAL;
    return DISPATCH(do_merge_underfull<uint32_t>(h, h_freed, S(stream)),
                    do_merge_underfull<uint64_t>(h, h_freed, S(stream)));
}

int flix_restructure(flix_t h, void* stream)
{
    if (!h) return FLIX_EINVAL;
    return DISPATCH(do_restructure<uint32_t>(h, S(stream)), do_restructure<uint64_t>(h, S(stream)));
}

int flix_stats(flix_t h, flix_stats_t* out, void* stream)
{
    if (!h || !out) return FLIX_EINVAL;
    return DISPATCH(do_stats<uint32_t>(h, out, S(stream)), do_stats<uint64_t>(h, out, S(stream)));
}

int flix_export(flix_t h, void* d_keys, void* d_vals, uint64_t cap, uint64_t* h_n, void* stream)
{
    if (!h || (cap && (!d_keys || !d_vals))) return FLIX_EINVAL;
    return DISPATCH(do_export<uint32_t>(h, (uint32_t*)d_keys, (uint32_t*)d_vals, cap, h_n, S(stream)),
                    do_export<uint64_t>(h, (uint64_t*)d_keys, (uint64_t*)d_vals, cap, h_n, S(stream)));
}

int flix_dump_layout(flix_t h, uint64_t* h_counts, void* h_mkba, uint32_t* h_chain_len, uint32_t* h_node_size,
                     void* h_node_bound, void* h_keys, void* h_vals, void* stream)
{
    if (!h || !h_counts) return FLIX_EINVAL;
    const bool any = h_mkba || h_chain_len || h_node_size || h_node_bound || h_keys || h_vals;
    const bool all = h_mkba && h_chain_len && h_node_size && h_node_bound && h_keys && h_vals;
    if (any && !all) return FLIX_EINVAL;
    return DISPATCH(do_dump<uint32_t>(h, h_counts, (uint32_t*)h_mkba, h_chain_len, h_node_size, (uint32_t*)h_node_bound,
                                      (uint32_t*)h_keys, (uint32_t*)h_vals, S(stream)),
                    do_dump<uint64_t>(h, h_counts, (uint64_t*)h_mkba, h_chain_len, h_node_size, (uint64_t*)h_node_bound,
                                      (uint64_t*)h_keys, (uint64_t*)h_vals, S(stream)));
}

int flix_profile_enable(flix_t h, int enable)
{
    if (!h) return FLIX_EINVAL;
    h->prof_on = enable != 0;
    return FLIX_OK;
}

int flix_profile_reset(flix_t h)
{
    if (!h) return FLIX_EINVAL;
    cudaDeviceSynchronize();
    h->prof.clear();
    h->ev_used = 0;
    return FLIX_OK;
}

int flix_profile_read(flix_t h, uint32_t max_entries, char* h_names, uint64_t* h_launches, double* h_total_ms,
                      double* h_bytes, uint32_t* h_n_entries)
{
    if (!h) return FLIX_EINVAL;
    CK(cudaDeviceSynchronize());
    std::vector<uint64_t> cnt(K_NUM, 0);
    std::vector<double> ms(K_NUM, 0.0), by(K_NUM, 0.0);
    for (const ProfRec& r : h->prof) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, r.a, r.b));
        cnt[r.kid]++;
        ms[r.kid] += t;
        by[r.kid] += r.bytes;
    }
    uint32_t k = 0;
    for (int i = 0; i < K_NUM; i++) {
        if (!cnt[i]) continue;
        if (k < max_entries) {
            if (h_names) {
                memset(h_names + 48 * k, 0, 48);
                strncpy(h_names + 48 * k, kKernelNames[i], 47);
            }
            if (h_launches) h_launches[k] = cnt[i];
            if (h_total_ms) h_total_ms[k] = ms[i];
            if (h_bytes) h_bytes[k] = by[i];
        }
        k++;
    }
    if (h_n_entries) *h_n_entries = k < max_entries ? k : max_entries;
    return FLIX_OK;
}

uint64_t flix_launch_count(flix_t h) { return h ? h->launches : 0; }

const char* flix_strerror(int code)
{
    switch (code) {
        case FLIX_OK: return "ok";
        case FLIX_EINVAL: return "invalid argument (or reserved key KEY_MAX)";
        case FLIX_ENOMEM: return "out of memory or output capacity";
        case FLIX_ECUDA: return "CUDA runtime error";
        case FLIX_ETYPE: return "unsupported key type or node size";
        case FLIX_ETIMEDOUT: return "device wait timed out";
        case FLIX_EINTERNAL: return "internal consistency check failed";
        case FLIX_ENOTIMPL: return "not implemented";
        default: return "unknown error";
    }
}

const char* flix_last_error(flix_t h) { return h ? h->last_error.c_str() : ""; }

}  // extern "C"
