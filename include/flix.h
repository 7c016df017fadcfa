/*
 * flix.h -- C ABI of a GB300-native (sm_103a) implementation of FliX, the flipped-indexing GPU
 * ordered map (Kharal, Brown, Henneberg, Schuhknecht: "FliX: Flipped-Indexing for Scalable GPU
 * Queries and Updates", arXiv 2604.16725).
 *
 * Data layer (Sec. 3.2): buckets are chains of fixed-capacity nodes (node_size key/value slots plus
 * maxKey, size and a node-link); the MKBA holds every bucket's maxBucket.  There is no index layer:
 * every batch is radix-sorted by key and each bucket pulls the operations in its key range
 * (maxBucket_{i-1}, maxBucket_i] from the sorted batch (Sec. 3.3, Sec. 4.1), then applies them in
 * place (lookup and successor Sec. 3.3 / Sec. 6.5; insert with node split Sec. 4.3.2; delete with
 * compaction and node reclamation Sec. 4.4; restructuring Sec. 3.5).
 *
 * Conventions shared by every entry point:
 *  - Keys and values have the same width, fixed at creation: uint32 (FLIX_KEY_U32) or uint64
 *    (FLIX_KEY_U64).  KEY_MAX = all ones is reserved: it is the last bucket's maxBucket and the
 *    successor "none" key, so it cannot be stored.  VAL_NONE = all ones is the miss value.
 *  - Arrays named d_* are caller-owned DEVICE memory on the handle's GPU; arrays named h_* are
 *    caller-owned HOST memory.  Device arrays must stay valid until the stream reaches the call.
 *    The handle owns its node pool, MKBA and scratch memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Work is
 *    enqueued on it in order.  Calls that must return a size or an admission decision read a few
 *    bytes back and synchronise the stream (stated per call).
 *  - Batch semantics (Sec. 3.3 runs queries on a sorted batch; the paper only runs homogeneous
 *    batches): in a mixed batch every lookup, successor and range query sees the state BEFORE the
 *    batch; then the batch's inserts and deletes take effect in submission order.  Inserting a
 *    present key keeps its value (Sec. 3.2); deleting an absent key does nothing.
 *  - Errors are return codes (flix_status).  FLIX_EINVAL and FLIX_ENOMEM from an update or build
 *    leave the structure unchanged (the node demand is counted before anything is written).
 *  - One handle is used by one host thread and one stream at a time.
 */
#ifndef FLIX_H
#define FLIX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct flix_index* flix_t;

typedef enum {
    FLIX_OK = 0,
    FLIX_EINVAL = -1,      /* bad argument, or KEY_MAX in an insert/build key array */
    FLIX_ENOMEM = -2,      /* node pool or caller output capacity too small; nothing changed */
    FLIX_ECUDA = -3,       /* a CUDA runtime call failed (flix_last_error has the text) */
    FLIX_ETYPE = -4,       /* unsupported key type or node size */
    FLIX_ETIMEDOUT = -5,   /* a bounded device-side wait gave up */
    FLIX_EINTERNAL = -6,   /* a device-side consistency check failed */
    FLIX_ENOTIMPL = -7
} flix_status;

typedef enum { FLIX_KEY_U32 = 0, FLIX_KEY_U64 = 1 } flix_keytype;

/* Operation codes of mixed batches (flix_apply). */
enum {
    FLIX_OP_NOP = 0,
    FLIX_OP_LOOKUP = 1,    /* point query (Sec. 3.3) */
    FLIX_OP_SUCC = 2,      /* successor: smallest stored key >= key (Sec. 6.5) */
    FLIX_OP_RANGE = 3,     /* all pairs with lo <= key <= hi; lo = key, hi = aux (named in Sec. 2.1) */
    FLIX_OP_INSERT = 4,    /* insert (key, aux) if key is absent (Sec. 3.2, Sec. 4.3.2) */
    FLIX_OP_DELETE = 5,    /* physical delete (Sec. 3.2, Sec. 4.4) */
    FLIX_OP_PRED = 6       /* predecessor: largest stored key <= key (named in Sec. 2.1; the mirror
                              of the successor of Sec. 6.5) */
};

typedef struct {
    flix_keytype key_type;
    uint32_t node_size;    /* NS: slots per node, a power of two in [4, 128] (Sec. 5.3.1) */
    uint32_t fill_pct;     /* keys per node after a build or restructure, % of NS (Sec. 3.2: 50) */
    uint32_t grow;         /* nonzero: the node pool grows when an update needs more nodes */
    uint64_t pool_nodes;   /* initial node-pool capacity; 0 = sized by the first bulk load */
    uint32_t sort_digit_bits; /* radix digit width of the batch sort: 8 (default) */
    uint32_t sort_variant;    /* FLIX_SORT_*: how each radix pass finds its output offsets */
    uint32_t restructure_in_one_pass; /* nonzero: flix_restructure writes every live pair straight
                                 into its place in a second key/value node array, kept for later
                                 restructures (doubles the pool's key and value memory, halves
                                 the restructure's traffic); zero: gather to scratch, then cut */
    uint32_t split_chains_over; /* nonzero T: after every synchronous update batch, each bucket the
                                 batch touched whose chain is longer than T nodes is split into
                                 one bucket per node (flix_split_chains; asynchronous batches never
                                 change the bucket count).  0 (default): off */
    uint32_t merge_underfull; /* nonzero: after every update batch (synchronous or not), each bucket
                                 the batch touched merges underfull neighbours (flix_merge_underfull).
                                 0 (default): off */
    uint32_t bucket_threads;  /* threads that apply one bucket's updates (the paper's single-thread
                                 and tiled kernels, Sec. 4.2-4.3): 0 (default) one thread for a
                                 bucket whose chain is one node and that receives at most 8 updates
                                 which still fit the node, a warp (32 threads) for every other
                                 bucket; 32: a warp for every bucket.  Same layout either way */
    uint32_t reserved[2];
    /* Optional device allocator for every device buffer the handle owns (node pool, bucket arrays,
     * scratch, state words), e.g. a framework's caching allocator: dev_alloc(bytes, alloc_ctx)
     * returns memory of the current device aligned to at least 256 bytes, or NULL when it cannot;
     * dev_free(ptr, alloc_ctx) takes back a pointer dev_alloc returned.  The library synchronises
     * the device before every dev_free, so no kernel still uses the memory.  Both NULL (default):
     * cudaMalloc and cudaFree. */
    void* (*dev_alloc)(size_t bytes, void* alloc_ctx);
    void (*dev_free)(void* ptr, void* alloc_ctx);
    void* alloc_ctx;
} flix_config;

/* Batch-sort variants (same stable order, different speed): one-sweep passes with decoupled
 * look-back, or reduce-then-scan passes (a counting read, a scan, then the scatter). */
enum { FLIX_SORT_AUTO = 0, FLIX_SORT_ONESWEEP = 1, FLIX_SORT_REDUCE_SCAN = 2 };

typedef struct {
    uint64_t buckets;         /* number of buckets (MKBA entries) */
    uint64_t nodes_used;      /* nodes in bucket chains */
    uint64_t nodes_free;      /* nodes on the free list */
    uint64_t pool_nodes;      /* node-pool capacity */
    uint64_t live_keys;       /* stored pairs */
    uint64_t max_chain;       /* longest bucket chain, in nodes */
    uint64_t node_bytes;      /* bytes of one node: keys, values, maxKey, size, node-link */
    uint64_t used_bytes;      /* nodes_used * node_bytes + MKBA and bucket heads */
    uint64_t reserved_bytes;  /* device bytes held by the pool and the bucket arrays (and the
                                 second key/value arrays of the one-pass restructure) */
} flix_stats_t;

/* Fill *cfg with defaults for key type kt: node_size 32 (u32) or 64 (u64), fill 50%, grow on,
 * one-pass restructure on. */
void flix_config_default(flix_config* cfg, flix_keytype kt);

/* Create an empty index (one bucket with one empty node) on the current CUDA device.
 * Returns FLIX_ETYPE for an unsupported key type or node size, FLIX_EINVAL if only one of
 * dev_alloc and dev_free is given, FLIX_ECUDA if allocation fails. */
int flix_create(const flix_config* cfg, flix_t* out);

/* Free every device and host resource of h (synchronises the device). */
int flix_destroy(flix_t h);

/* Initial build (Sec. 3.2): sort the n pairs by key, keep the first pair of each duplicated key,
 * cut the sorted keys into groups of fill_pct*node_size, one single-node bucket per group; each
 * group's largest key becomes its maxBucket, the last bucket's is KEY_MAX.  Replaces the contents.
 * d_keys/d_vals: n keys and n values.  Synchronises (reads back the distinct count).
 * FLIX_EINVAL if a key is KEY_MAX (contents unchanged). */
int flix_bulk_load(flix_t h, const void* d_keys, const void* d_vals, uint64_t n, void* stream);

/* Point queries (Sec. 3.3): d_vals_out[i] = value of d_keys[i] or VAL_NONE; d_found_or_null[i] =
 * 1/0 if given.  Asynchronous. */
int flix_lookup(flix_t h, const void* d_keys, uint64_t n, void* d_vals_out, uint8_t* d_found_or_null,
                void* stream);

/* Bytes of the fixed device scratch array used by flix_lookup_noalloc. */
#define FLIX_NOALLOC_SCRATCH_BYTES (16u << 20)

/* flix_lookup without any device allocation during the call.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory when they query -- a process
 * whose allocator has already reserved the whole device for its own pools, a latency-bound path
 * that must not block on cudaMalloc's implicit device synchronisation, or a host with a custom
 * allocator this library cannot see.  Same arguments and results as flix_lookup.
 * Its scratch (sort buffers and bucket offsets) is one fixed array of FLIX_NOALLOC_SCRATCH_BYTES
 * compiled into the library; every GPU that loads the library holds it until the process exits.
 * A call needs about 31*n bytes (uint64 keys; 22*n for uint32) plus a few KB and 8 bytes per
 * 2048 buckets, so up to about 2^19 uint64 keys per call fit; a larger request returns
 * FLIX_EINVAL before launching anything (flix_last_error gives the sizes).  The first call on a
 * device looks up the array's device address on that device, so make it before any stream capture.
 * All calls share the array: calls whose work overlaps on the GPU (other streams, threads or
 * handles on the same device) race and must be serialised by the caller.  Asynchronous. */
int flix_lookup_noalloc(flix_t h, const void* d_keys, uint64_t n, void* d_vals_out, uint8_t* d_found_or_null,
                        void* stream);

/* Successor queries (Sec. 6.5: smallest stored key >= key): d_keys_out[i], d_vals_out[i], or
 * (KEY_MAX, VAL_NONE) when none exists.  Asynchronous. */
int flix_successor(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, void* d_vals_out,
                   void* stream);

/* Elastic bucket split (Sec. 3.4 names splitting buckets with long chains of nodes, which narrows
 * the key range each bucket covers).  Every bucket whose chain holds more than max_chain nodes
 * (max_chain >= 1) becomes one bucket per node, in chain order; each new bucket's maxBucket is its
 * node's maxKey, and the chain's last node keeps the old maxBucket.  No pair moves and no node is
 * allocated: only the MKBA and the bucket heads change (written to a second pair of bucket arrays,
 * allocated at the first split and sized like the pool, then swapped in).  *h_added (may be NULL)
 * receives the number of buckets added.  Synchronises.  FLIX_EINVAL if max_chain is 0. */
int flix_split_chains(flix_t h, uint32_t max_chain, uint64_t* h_added, void* stream);

/* Underfull-neighbour merge (Sec. 5.4.1 names merging underfull nodes during deletion as a possible
 * addition; Sec. 6.6 merges them into half-full nodes by restructuring).  In every bucket, walk the
 * chain: while the current node and the next hold at most NS/2 pairs together, the next node's
 * pairs are appended to the current node, which takes over its maxKey and node-link, and the next
 * node goes on the free list; otherwise the walk moves on.  *h_freed (may be NULL) receives the
 * number of nodes freed.  Synchronises. */
int flix_merge_underfull(flix_t h, uint64_t* h_freed, void* stream);

/* Predecessor queries (largest stored key <= key; the paper names predecessor in Sec. 2.1 without
 * defining it, and this is the mirror of Sec. 6.5's successor): d_keys_out[i], d_vals_out[i], or
 * (KEY_MAX, VAL_NONE) when none exists.  Asynchronous. */
int flix_predecessor(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, void* d_vals_out,
                     void* stream);

/* Range queries [d_lo[i], d_hi[i]] (inclusive; empty when lo > hi): pairs ascending per query,
 * concatenated in query order; d_offsets_out[n+1] (uint64) holds each query's start and the total.
 * d_keys_out/d_vals_out hold out_capacity pairs.  Synchronises to read the total into
 * *h_total_out; returns FLIX_ENOMEM (offsets written, pairs not) if it exceeds out_capacity. */
int flix_range(flix_t h, const void* d_lo, const void* d_hi, uint64_t n, uint64_t* d_offsets_out,
               void* d_keys_out, void* d_vals_out, uint64_t out_capacity, uint64_t* h_total_out,
               void* stream);

/* Insert n pairs (Sec. 4.3.2: merge into the first node with key <= maxKey, split full nodes into
 * halves).  Synchronises once (node-demand admission).  FLIX_EINVAL if a key is KEY_MAX,
 * FLIX_ENOMEM if the pool is short and grow is off; both leave the contents unchanged. */
int flix_insert(flix_t h, const void* d_keys, const void* d_vals, uint64_t n, void* stream);

/* Delete n keys (Sec. 4.4: compaction, emptied nodes leave their chain and are reused).
 * Synchronises once. */
int flix_delete(flix_t h, const void* d_keys, uint64_t n, void* stream);

/* Mixed batch of n ops (codes FLIX_OP_*), keys d_keys, per-op aux (insert value or range hi).
 * Reads see the pre-batch state.  Per op i:
 *   LOOKUP: d_vals_out[i] = value or VAL_NONE, d_found[i] = hit, d_keys_out[i] = key or KEY_MAX
 *   SUCC  : d_keys_out[i], d_vals_out[i] = successor pair or (KEY_MAX, VAL_NONE), d_found[i]
 *   PRED  : d_keys_out[i], d_vals_out[i] = predecessor pair or (KEY_MAX, VAL_NONE), d_found[i]
 *   others: (KEY_MAX, VAL_NONE, 0)
 * d_range_off[n+1]: exclusive prefix of range result counts (0 for non-range ops); the pairs go to
 * d_range_keys/d_range_vals (capacity range_cap).  Any output pointer may be NULL if the batch has
 * no op that writes it.  Synchronises (range total and node admission).  Errors as for
 * flix_insert and flix_range; on FLIX_ENOMEM for the range capacity the updates are not applied.
 * After its sort the batch's reads run on `stream` and the preparation of its updates on a stream
 * the handle owns; that stream rejoins `stream` (an event wait) before anything else is enqueued,
 * so all of the call's work is ordered before later work on `stream`, also when captured. */
int flix_apply(flix_t h, const uint8_t* d_ops, const void* d_keys, const void* d_aux, uint64_t n,
               void* d_keys_out, void* d_vals_out, uint8_t* d_found, uint64_t* d_range_off,
               void* d_range_keys, void* d_range_vals, uint64_t range_cap, uint64_t* h_range_total,
               void* stream);

/* flix_apply without any host synchronisation, for streams of batches and CUDA-graph capture (the
 * paper runs one batch per launch; this form keeps the whole batch on the device).  Same batch
 * semantics and outputs as flix_apply.  Admission is decided on the device: if an insert carries
 * KEY_MAX, the free nodes do not cover the batch's node demand, or the range pairs exceed range_cap,
 * the batch's updates and range pairs are not written (lookup and successor results still are).
 * d_status: caller-owned DEVICE uint64[4] written by the call: flags (1 reserved key, 2 node pool
 * short, 4 range capacity short), range pair total, nodes the batch needed, free nodes before it.
 * The handle's scratch must already hold a batch of n ops (flix_reserve); otherwise FLIX_ENOMEM is
 * returned before anything is launched.  The call never grows the pool.  Kernel parameters
 * capture the current bucket count and pool, so a captured graph must be re-captured after
 * flix_bulk_load, flix_restructure or pool growth. */
int flix_apply_async(flix_t h, const uint8_t* d_ops, const void* d_keys, const void* d_aux, uint64_t n,
                     void* d_keys_out, void* d_vals_out, uint8_t* d_found, uint64_t* d_range_off,
                     void* d_range_keys, void* d_range_vals, uint64_t range_cap, uint64_t* d_status,
                     void* stream);

/* One batch of a persistent queue (flix_apply_queue): the arrays of a flix_apply_async call, all
 * caller-owned device memory, plus an optional device word `ready`: when it is not NULL the kernel
 * waits for the word to become nonzero before it reads the batch (a producer can then fill the
 * batch while the kernel runs the ones before it). */
typedef struct {
    const uint8_t* ops;    /* n op codes FLIX_OP_* */
    const void* keys;      /* n keys */
    const void* aux;       /* n insert values or range upper bounds */
    uint64_t n;            /* at most FLIX_QUEUE_BATCH_MAX */
    void* keys_out;        /* n, as flix_apply (may be NULL when no op writes it) */
    void* vals_out;        /* n */
    uint8_t* found;        /* n */
    uint64_t* range_off;   /* n + 1 */
    void* range_keys;      /* range_cap */
    void* range_vals;      /* range_cap */
    uint64_t range_cap;
    uint64_t* status;      /* 4 words, as flix_apply_async; flags bit 8: not run (a wait gave up) */
    const uint32_t* ready; /* NULL, or a word the kernel waits on before it reads the batch */
} flix_batch;

#define FLIX_QUEUE_BATCH_MAX 2048u

/* A queue of count small mixed batches run in order by ONE persistent kernel (the batched form of
 * the paper's method: no launch per batch).  A cooperative grid of one wave of blocks takes the
 * batches one after another; each batch goes through the method's steps as phases separated by
 * grid barriers: its sort (Sec. 3.3) and same-key fold, the snapshot reads and every op's bucket,
 * the per-bucket update count and the range offsets, the admission (free nodes, range capacity,
 * reserved key), the range pairs, and the per-bucket merge, split and compaction (Sec. 4.3.2,
 * Sec. 4.4), one thread per touched bucket.  Each batch has exactly the semantics and outputs of
 * flix_apply_async (a rejected batch changes nothing; its reads are still written).  Every wait (a
 * batch's ready word, a grid barrier) gives up after wait_us microseconds: the queue then stops,
 * the batches not run get flag 8 in status[0], and the next synchronising call on the handle
 * returns FLIX_ETIMEDOUT.  h_batches is a HOST array of count descriptors (copied before the
 * launch).  Asynchronous; not for stream capture.  The chain split and underfull merge policies
 * are not applied on this path (FLIX_ENOTIMPL when one is configured).  Returns FLIX_EINVAL for a
 * batch larger than FLIX_QUEUE_BATCH_MAX.  d_flags_or (optional DEVICE word): every batch's status
 * flags are OR-ed into it. */
int flix_apply_queue(flix_t h, const flix_batch* h_batches, uint32_t count, uint32_t wait_us,
                     uint64_t* d_flags_or, void* stream);

/* Reserve scratch for batches of up to batch_max ops and grow the pool (if needed) so that at least
 * free_nodes_min nodes are free.  Synchronises.  FLIX_ENOMEM if the device cannot hold it. */
int flix_reserve(flix_t h, uint64_t batch_max, uint64_t free_nodes_min, void* stream);

/* Restructure (Sec. 3.5): flatten every chain, re-cut the live pairs into single-node buckets at
 * the build fill, reset the MKBA and the free list.  Synchronises. */
int flix_restructure(flix_t h, void* stream);

/* Statistics of h (synchronises). */
int flix_stats(flix_t h, flix_stats_t* out, void* stream);

/* All live pairs in key order into d_keys/d_vals (capacity cap); *h_n = count.  Synchronises.
 * FLIX_ENOMEM (nothing written) if the count exceeds cap. */
int flix_export(flix_t h, void* d_keys, void* d_vals, uint64_t cap, uint64_t* h_n, void* stream);

/* Layout dump in bucket and chain order, into HOST arrays (for tests and debugging).  With all
 * arrays NULL only h_counts[3] = {buckets, nodes in chains, live keys} is written.  Otherwise:
 * h_mkba[buckets], h_chain_len[buckets], h_node_size[nodes], h_node_bound[nodes] (maxKey),
 * h_keys[keys], h_vals[keys]; key-width arrays are uint32 or uint64 per the key type.
 * Synchronises. */
int flix_dump_layout(flix_t h, uint64_t* h_counts, void* h_mkba, uint32_t* h_chain_len,
                     uint32_t* h_node_size, void* h_node_bound, void* h_keys, void* h_vals,
                     void* stream);

/* Test hook: the batch sort alone (Sec. 3.3 sorts each batch by key before buckets pull their
 * operations; Tab. 1 times it).  d_keys_out[0..n) = the keys of d_keys ascending, d_pos_out[i] =
 * the input position of d_keys_out[i]; equal keys keep their input order (a stable sort, which
 * the same-key fold of an update batch depends on).  The index's contents are not used or changed;
 * scratch comes from the handle.  Device arrays, caller-owned; n < 2^32 - 4096.  Stream-ordered;
 * synchronises once at the end to report device errors.  Returns FLIX_EINVAL on null pointers. */
int flix_sort_pairs(flix_t h, const void* d_keys, uint64_t n, void* d_keys_out, uint32_t* d_pos_out,
                    void* stream);

/* Per-kernel timing.  While enabled, every kernel launch of h is bracketed by CUDA events on the
 * launch stream (and a batch sort reads its pass plan back, so that passes the plan leaves out are
 * listed as "sort_pass_idle").  flix_profile_read synchronises and returns up to max_entries rows:
 * kernel name (NUL-terminated, 48 bytes per row in h_names), launch count, total milliseconds and
 * total algorithmic bytes (the bytes the launches must move by definition, for kernels where the
 * host knows them, else 0).  Any output array may be NULL. */
int flix_profile_enable(flix_t h, int enable);
int flix_profile_reset(flix_t h);
int flix_profile_read(flix_t h, uint32_t max_entries, char* h_names, uint64_t* h_launches,
                      double* h_total_ms, double* h_bytes, uint32_t* h_n_entries);

/* Number of kernels h has launched since creation. */
uint64_t flix_launch_count(flix_t h);

/* Text of an error code, and the last CUDA error text recorded by h (never NULL). */
const char* flix_strerror(int code);
const char* flix_last_error(flix_t h);

#ifdef __cplusplus
}
#endif

#endif /* FLIX_H */
