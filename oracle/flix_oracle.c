/*
 * FliX CPU oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the smoke check and the benchmark's CPU-baseline leg load this library.  The
 * product (the CUDA library and its Python binding) never calls it and shares no code with it.
 *
 * It is deliberately plain and slow: sorted arrays, qsort, binary searches and linear merges, each
 * step written to be checked against the paper by eye.  Two parts:
 *
 *  1. The semantic ordered map (om_map_*): the result every FliX batch must reach.  A FliX batch is
 *     applied with snapshot semantics: lookups, successor and range queries see the state before the
 *     batch; then the batch's inserts and deletes are applied in submission order.  An insert of a
 *     present key leaves its value unchanged (Sec. 3.2: a key is inserted only if not already
 *     present); a delete removes the key physically (Sec. 3.2, no tombstones).  Successor is the
 *     smallest stored key k' >= k (Sec. 6.5).  A miss returns the all-ones "none" value (Sec. 3.3).
 *     Range [lo, hi] is inclusive and ascending; the paper names but does not define it (Sec. 2.1,
 *     Sec. 3.3), so this is the reading used throughout.
 *
 *  2. The structural model (om_model_*) of FliX's data layer, following Sec. 3.2-3.5 and Sec. 4:
 *     buckets are chains of fixed-capacity nodes (NS slots, metadata maxKey and size, a node-link);
 *     the MKBA holds each bucket's maxBucket; the initial build cuts the sorted keys into groups of
 *     p = fill * NS; each bucket pulls its sublist from the sorted update list by a binary search for
 *     maxBucket_{i-1} (Sec. 3.3, Sec. 4.1); an update goes to the first node of the chain whose
 *     maxKey >= k (Sec. 4.1); deletes compact the node by shifting survivors left by the number of
 *     earlier deletions (Sec. 4.4, Tab. 3); inserts merge the sublist into the node in key order
 *     (Sec. 4.3.2, Tab. 2); a node that overflows is split into halves (Sec. 3.2, Sec. 5.3.1);
 *     emptied nodes leave the chain and are reused (Sec. 4.4); restructuring flattens every chain
 *     into half-full single-node buckets and resets the MKBA (Sec. 3.5, Sec. 6.6).
 *
 *     Where the paper leaves the node layout after a multi-key overflow open, the model uses one
 *     canonical layout: a merged run of t keys stays one node if t <= NS; otherwise it becomes
 *     q = floor(t / s) nodes (s = NS/2, the even half of Sec. 5.3.1): q-1 nodes of s keys and a last
 *     node of the remaining t-(q-1)s keys.  Every piece but the last takes its own largest key as
 *     maxKey; the last keeps the old node's maxKey.  This reproduces Tab. 2.  An emptied node is
 *     unlinked unless the whole chain emptied, in which case the chain's first node stays as an empty
 *     node; when the chain's last node leaves, its maxKey (= maxBucket) passes to the new last node.
 *
 *     Two structural operations the paper proposes without fixing them (off unless asked for):
 *     the elastic split of a bucket with a long chain (Sec. 3.4), read here as one bucket per node
 *     of the chain with the node's maxKey as maxBucket, and the merge of underfull nodes during
 *     deletion (Sec. 5.4.1), read here as folding a chain's next node into the current one while
 *     both hold at most NS/2 pairs.  A policy runs both after every update batch on the buckets
 *     the batch touched (merge first, then split).
 *
 *  3. The same semantic map on all host cores (om_map_*_mt): the batch's reads split over threads by
 *     op ranges (each thread answers its ops on the unchanged snapshot), range offsets by one
 *     sequential scan, then the batch's net updates (the same per-key replay as om_map_update)
 *     merged into the sorted arrays by threads that each own a key range.  Same results as part 1;
 *     it is the timed CPU baseline, not a reference for the GPU.
 *
 * Keys and values are held as uint64 for both key widths kw in {32, 64}; KEY_MAX = 2^kw - 1 is not a
 * storable key (it is the last bucket's maxBucket and the successor "none" key) and VAL_NONE is
 * the all-ones value of the same width.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OP_NOP = 0, OP_LOOKUP = 1, OP_SUCC = 2, OP_RANGE = 3, OP_INSERT = 4, OP_DELETE = 5, OP_PRED = 6 };
/* Net effect of a key's update run (composition of its inserts and deletes in submission order). */
enum { EFF_NONE = 0, EFF_INS = 1, EFF_DEL = 2, EFF_UPS = 3 };

#define NIL (-1)

static uint64_t width_max(int kw) { return kw == 64 ? ~(uint64_t)0 : (((uint64_t)1 << kw) - 1); }

/* ------------------------------------------------------------------------------------------------
 * Small helpers
 * ---------------------------------------------------------------------------------------------- */

typedef struct {
    uint64_t key, val, pos;
    uint8_t op;
} orec;

static int cmp_key_pos(const void* a, const void* b)
{
    const orec* x = (const orec*)a;
    const orec* y = (const orec*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

/* first i in [0, n) with a[i] >= x, or n */
static size_t lower_bound_u64(const uint64_t* a, size_t n, uint64_t x)
{
    size_t lo = 0, hi = n;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* first i in [0, n) with a[i] > x, or n */
static size_t upper_bound_u64(const uint64_t* a, size_t n, uint64_t x)
{
    size_t lo = 0, hi = n;
    while (lo < hi) {
        size_t mid = lo + (hi - lo) / 2;
        if (a[mid] <= x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

/* Apply one key's update ops, in submission order, to its state (present, val). */
static void apply_run(const orec* r, size_t m, int* present, uint64_t* val)
{
    for (size_t i = 0; i < m; i++) {
        if (r[i].op == OP_INSERT) {
            if (!*present) { *present = 1; *val = r[i].val; }
        } else if (r[i].op == OP_DELETE) {
            *present = 0;
        }
    }
}

/* Net effect of a key's update run, whatever the key's prior state:
 *   ends absent                       -> EFF_DEL
 *   ends present, no delete in the run -> EFF_INS (first insert's value; a no-op if present)
 *   ends present after a delete        -> EFF_UPS (the value inserted after the last delete) */
static int run_effect(const orec* r, size_t m, uint64_t* val)
{
    int present = 0, deleted = 0;
    uint64_t v = 0;
    apply_run(r, m, &present, &v);          /* replayed from the absent state */
    for (size_t i = 0; i < m; i++)
        if (r[i].op == OP_DELETE) deleted = 1;
    if (!present) return EFF_DEL;
    *val = v;
    return deleted ? EFF_UPS : EFF_INS;
}

/* ------------------------------------------------------------------------------------------------
 * 1. Semantic ordered map
 * ---------------------------------------------------------------------------------------------- */

typedef struct {
    int kw;
    uint64_t kmax;
    uint64_t* k;
    uint64_t* v;
    size_t n;
} om_map;

om_map* om_map_create(int kw)
{
    if (kw != 32 && kw != 64) return NULL;
    om_map* m = (om_map*)calloc(1, sizeof(om_map));
    m->kw = kw;
    m->kmax = width_max(kw);
    return m;
}

void om_map_destroy(om_map* m)
{
    if (!m) return;
    free(m->k);
    free(m->v);
    free(m);
}

size_t om_map_size(const om_map* m) { return m->n; }

void om_map_export(const om_map* m, uint64_t* keys, uint64_t* vals)
{
    memcpy(keys, m->k, m->n * sizeof(uint64_t));
    memcpy(vals, m->v, m->n * sizeof(uint64_t));
}

/* Build from pairs: duplicates keep the first occurrence.  Returns -1 (unchanged) on KEY_MAX. */
int om_map_bulk_load(om_map* m, const uint64_t* keys, const uint64_t* vals, size_t n)
{
    for (size_t i = 0; i < n; i++)
        if (keys[i] >= m->kmax) return -1;
    orec* r = (orec*)malloc((n ? n : 1) * sizeof(orec));
    for (size_t i = 0; i < n; i++) { r[i].key = keys[i]; r[i].val = vals[i]; r[i].pos = i; r[i].op = OP_INSERT; }
    qsort(r, n, sizeof(orec), cmp_key_pos);
    free(m->k);
    free(m->v);
    m->k = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    m->v = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    size_t c = 0;
    for (size_t i = 0; i < n; i++) {
        if (i > 0 && r[i].key == r[i - 1].key) continue;
        m->k[c] = r[i].key;
        m->v[c] = r[i].val;
        c++;
    }
    m->n = c;
    free(r);
    return 0;
}

/* Reads of one batch against the current state.  Per op i (all outputs defined for every op):
 *   LOOKUP: out_val = value or VAL_NONE, out_found = hit, out_key = key if hit else KEY_MAX
 *   SUCC  : out_key = smallest stored key >= key (KEY_MAX if none), out_val its value (VAL_NONE),
 *           out_found = exists
 *   PRED  : out_key = largest stored key <= key (KEY_MAX if none), out_val its value (VAL_NONE),
 *           out_found = exists (the mirror of SUCC; the paper names predecessor without defining it)
 *   other : out_key = KEY_MAX, out_val = VAL_NONE, out_found = 0
 * range_off[n+1] (if non-NULL): exclusive prefix of the per-op range counts |{k : lo <= k <= hi}|
 * for RANGE ops (lo = key, hi = aux; empty when lo > hi) and 0 for all other ops. */
void om_map_read(const om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys,
                 const uint64_t* aux, uint64_t* out_val, uint8_t* out_found, uint64_t* out_key,
                 uint64_t* range_off)
{
    const uint64_t none = m->kmax;
    uint64_t acc = 0;
    if (range_off) range_off[0] = 0;
    for (size_t i = 0; i < n; i++) {
        uint64_t ok = none, ov = none;
        uint8_t of = 0;
        uint64_t cnt = 0;
        if (ops[i] == OP_LOOKUP) {
            size_t p = lower_bound_u64(m->k, m->n, keys[i]);
            if (p < m->n && m->k[p] == keys[i]) { ok = keys[i]; ov = m->v[p]; of = 1; }
        } else if (ops[i] == OP_SUCC) {
            size_t p = lower_bound_u64(m->k, m->n, keys[i]);
            if (p < m->n) { ok = m->k[p]; ov = m->v[p]; of = 1; }
        } else if (ops[i] == OP_PRED) {
            size_t p = upper_bound_u64(m->k, m->n, keys[i]);
            if (p > 0) { ok = m->k[p - 1]; ov = m->v[p - 1]; of = 1; }
        } else if (ops[i] == OP_RANGE) {
            if (keys[i] <= aux[i]) {
                size_t a = lower_bound_u64(m->k, m->n, keys[i]);
                size_t b = upper_bound_u64(m->k, m->n, aux[i]);
                cnt = b - a;
            }
        }
        if (out_key) out_key[i] = ok;
        if (out_val) out_val[i] = ov;
        if (out_found) out_found[i] = of;
        acc += cnt;
        if (range_off) range_off[i + 1] = acc;
    }
}

/* Range pairs of a batch, concatenated in op order at the offsets om_map_read produced. */
void om_map_range_fill(const om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys,
                       const uint64_t* aux, const uint64_t* range_off, uint64_t* rkeys, uint64_t* rvals)
{
    for (size_t i = 0; i < n; i++) {
        if (ops[i] != OP_RANGE || keys[i] > aux[i]) continue;
        size_t a = lower_bound_u64(m->k, m->n, keys[i]);
        size_t b = upper_bound_u64(m->k, m->n, aux[i]);
        uint64_t o = range_off[i];
        for (size_t j = a; j < b; j++, o++) { rkeys[o] = m->k[j]; rvals[o] = m->v[j]; }
    }
}

/* Inserts and deletes of one batch, applied in submission order.  Returns -1 (unchanged) if an
 * insert carries KEY_MAX.  Keys are independent, so the ops are grouped by key (stable, keeping
 * submission order inside a key) and each key's ops are replayed on that key's state. */
int om_map_update(om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys, const uint64_t* aux)
{
    size_t u = 0;
    for (size_t i = 0; i < n; i++) {
        if (ops[i] == OP_INSERT && keys[i] >= m->kmax) return -1;
        if (ops[i] == OP_INSERT || ops[i] == OP_DELETE) u++;
    }
    orec* r = (orec*)malloc((u ? u : 1) * sizeof(orec));
    u = 0;
    for (size_t i = 0; i < n; i++) {
        if (ops[i] != OP_INSERT && ops[i] != OP_DELETE) continue;
        r[u].key = keys[i];
        r[u].val = ops[i] == OP_INSERT ? aux[i] : 0;
        r[u].pos = i;
        r[u].op = ops[i];
        u++;
    }
    qsort(r, u, sizeof(orec), cmp_key_pos);
    uint64_t* nk = (uint64_t*)malloc((m->n + u + 1) * sizeof(uint64_t));
    uint64_t* nv = (uint64_t*)malloc((m->n + u + 1) * sizeof(uint64_t));
    size_t i = 0, j = 0, c = 0;
    while (i < m->n || j < u) {
        if (j >= u || (i < m->n && m->k[i] < r[j].key)) {
            nk[c] = m->k[i]; nv[c] = m->v[i]; c++; i++;
            continue;
        }
        size_t e = j;
        while (e < u && r[e].key == r[j].key) e++;
        int present = 0;
        uint64_t val = 0;
        if (i < m->n && m->k[i] == r[j].key) { present = 1; val = m->v[i]; i++; }
        apply_run(r + j, e - j, &present, &val);
        if (present) { nk[c] = r[j].key; nv[c] = val; c++; }
        j = e;
    }
    free(m->k);
    free(m->v);
    m->k = nk;
    m->v = nv;
    m->n = c;
    free(r);
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * 2. Structural model
 * ---------------------------------------------------------------------------------------------- */

/* Sec. 4.4 / Tab. 3: each node key is compared with the delete keys and marked; a survivor moves
 * left by the number of deletions among the slots before it.  shift[i] = -1 for a deleted slot.
 * Returns the new size. */
uint32_t om_delete_compact(const uint64_t* keys, uint32_t n, const uint64_t* dk, uint32_t m,
                           uint64_t* out, int32_t* shift)
{
    uint32_t del_count = 0;
    for (uint32_t i = 0; i < n; i++) {
        int marked = 0;
        for (uint32_t d = 0; d < m; d++)
            if (dk[d] == keys[i]) marked = 1;
        if (marked) {
            if (shift) shift[i] = -1;
            del_count++;
            continue;
        }
        if (shift) shift[i] = (int32_t)del_count;
        out[i - del_count] = keys[i];
    }
    return n - del_count;
}

/* Sec. 4.3.2 / Tab. 2: the sorted insert sublist is merged into the node's sorted keys; a key
 * already present is not inserted again.  Returns the merged size. */
uint32_t om_merge_insert(const uint64_t* keys, uint32_t n, const uint64_t* ins, uint32_t m, uint64_t* out)
{
    uint32_t i = 0, j = 0, c = 0;
    while (i < n || j < m) {
        if (j >= m || (i < n && keys[i] < ins[j])) out[c++] = keys[i++];
        else if (i < n && keys[i] == ins[j]) { out[c++] = keys[i++]; j++; }
        else out[c++] = ins[j++];
    }
    return c;
}

/* Canonical node layout of a merged run of t keys (see the header).  Writes the piece sizes and
 * returns the number of pieces q (0 when t == 0). */
uint32_t om_canonical_layout(uint64_t t, uint32_t NS, uint32_t* piece_sizes)
{
    if (t == 0) return 0;
    if (t <= NS) { if (piece_sizes) piece_sizes[0] = (uint32_t)t; return 1; }
    uint32_t s = NS / 2;
    uint64_t q = t / s;
    if (piece_sizes) {
        for (uint64_t r = 0; r + 1 < q; r++) piece_sizes[r] = s;
        piece_sizes[q - 1] = (uint32_t)(t - (q - 1) * s);
    }
    return (uint32_t)q;
}

typedef struct {
    int kw;
    uint64_t kmax;
    uint32_t NS, p;
    /* node pool */
    uint64_t cap, hw;
    uint64_t *keys, *vals;
    uint32_t* size;
    uint64_t* bound;
    int64_t* next;
    int64_t* free_stack;
    uint64_t nfree;
    /* buckets */
    uint64_t nb, nb_cap;
    uint64_t* mkba;
    int64_t* head;
    /* maintenance after every update batch (0: off) */
    uint64_t split_over;      /* elastic split of touched buckets with chains longer than this */
    int merge_underfull;      /* merge underfull neighbours in touched buckets */
} om_model;

static void model_grow(om_model* m, uint64_t want)
{
    if (want <= m->cap) return;
    uint64_t c = m->cap ? m->cap : 16;
    while (c < want) c *= 2;
    m->keys = (uint64_t*)realloc(m->keys, c * m->NS * sizeof(uint64_t));
    m->vals = (uint64_t*)realloc(m->vals, c * m->NS * sizeof(uint64_t));
    m->size = (uint32_t*)realloc(m->size, c * sizeof(uint32_t));
    m->bound = (uint64_t*)realloc(m->bound, c * sizeof(uint64_t));
    m->next = (int64_t*)realloc(m->next, c * sizeof(int64_t));
    m->free_stack = (int64_t*)realloc(m->free_stack, c * sizeof(int64_t));
    m->cap = c;
}

static int64_t node_alloc(om_model* m)
{
    if (m->nfree) return m->free_stack[--m->nfree];
    model_grow(m, m->hw + 1);
    return (int64_t)m->hw++;
}

static void node_free(om_model* m, int64_t id) { m->free_stack[m->nfree++] = id; }

static void buckets_resize(om_model* m, uint64_t nb)
{
    if (nb > m->nb_cap) {
        m->mkba = (uint64_t*)realloc(m->mkba, nb * sizeof(uint64_t));
        m->head = (int64_t*)realloc(m->head, nb * sizeof(int64_t));
        m->nb_cap = nb;
    }
    m->nb = nb;
}

om_model* om_model_create(int kw, uint32_t NS, uint32_t fill_pct)
{
    if ((kw != 32 && kw != 64) || NS < 2 || (NS & 1) || fill_pct == 0 || fill_pct > 100) return NULL;
    om_model* m = (om_model*)calloc(1, sizeof(om_model));
    m->kw = kw;
    m->kmax = width_max(kw);
    m->NS = NS;
    m->p = (uint32_t)(((uint64_t)NS * fill_pct) / 100);
    if (m->p < 1) m->p = 1;
    return m;
}

void om_model_destroy(om_model* m)
{
    if (!m) return;
    free(m->keys); free(m->vals); free(m->size); free(m->bound); free(m->next);
    free(m->free_stack); free(m->mkba); free(m->head);
    free(m);
}

/* Sec. 3.2: cut the sorted distinct pairs into groups of p keys, one single-node bucket per group;
 * maxBucket is the group's largest key, except the last bucket's, which is KEY_MAX so that keys
 * above the largest build key also have a bucket.  n == 0 gives one bucket with one empty node. */
static void model_cut(om_model* m, const uint64_t* k, const uint64_t* v, uint64_t n)
{
    m->hw = 0;
    m->nfree = 0;
    uint64_t nb = n ? (n + m->p - 1) / m->p : 1;
    buckets_resize(m, nb);
    model_grow(m, nb);
    for (uint64_t b = 0; b < nb; b++) {
        int64_t id = node_alloc(m);
        uint64_t lo = b * m->p, hi = lo + m->p < n ? lo + m->p : n;
        uint32_t sz = (uint32_t)(hi - lo);
        for (uint32_t s = 0; s < sz; s++) {
            m->keys[id * m->NS + s] = k[lo + s];
            m->vals[id * m->NS + s] = v[lo + s];
        }
        m->size[id] = sz;
        m->mkba[b] = (b + 1 == nb) ? m->kmax : k[hi - 1];
        m->bound[id] = m->mkba[b];
        m->next[id] = NIL;
        m->head[b] = id;
    }
}

int om_model_bulk_load(om_model* m, const uint64_t* keys, const uint64_t* vals, uint64_t n)
{
    for (uint64_t i = 0; i < n; i++)
        if (keys[i] >= m->kmax) return -1;
    orec* r = (orec*)malloc((n ? n : 1) * sizeof(orec));
    for (uint64_t i = 0; i < n; i++) { r[i].key = keys[i]; r[i].val = vals[i]; r[i].pos = i; r[i].op = 0; }
    qsort(r, n, sizeof(orec), cmp_key_pos);
    uint64_t* k = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t* v = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    uint64_t c = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (i > 0 && r[i].key == r[i - 1].key) continue;
        k[c] = r[i].key; v[c] = r[i].val; c++;
    }
    model_cut(m, k, v, c);
    free(r); free(k); free(v);
    return 0;
}

/* Apply one node's routed updates (sorted, distinct keys, net effects) and lay the result out.
 * Returns the number of output keys t; pieces are linked after `node`, the last piece's next is the
 * node's old next.  *tail receives the last piece (or NIL when t == 0). */
static uint64_t model_apply_node(om_model* m, int64_t node, const uint64_t* uk, const int* ue,
                                 const uint64_t* uv, uint64_t cnt, int64_t* tail)
{
    const uint32_t NS = m->NS;
    uint32_t sz = m->size[node];
    const uint64_t* nk = m->keys + node * NS;
    const uint64_t* nv = m->vals + node * NS;

    /* (i) deletes compact the node (Sec. 4.4); an upsert of a present key replaces its value. */
    uint64_t* dk = (uint64_t*)malloc((cnt + 1) * sizeof(uint64_t));
    uint32_t nd = 0;
    for (uint64_t j = 0; j < cnt; j++) if (ue[j] == EFF_DEL) dk[nd++] = uk[j];
    uint64_t* ck = (uint64_t*)malloc((NS + 1) * sizeof(uint64_t));
    uint64_t* cv = (uint64_t*)malloc((NS + 1) * sizeof(uint64_t));
    int32_t* shift = (int32_t*)malloc((NS + 1) * sizeof(int32_t));
    uint32_t c = om_delete_compact(nk, sz, dk, nd, ck, shift);
    for (uint32_t i = 0; i < sz; i++) if (shift[i] >= 0) cv[i - shift[i]] = nv[i];
    for (uint64_t j = 0; j < cnt; j++) {
        if (ue[j] != EFF_UPS) continue;
        for (uint32_t i = 0; i < c; i++) if (ck[i] == uk[j]) cv[i] = uv[j];
    }

    /* (ii) inserts (and upserts of absent keys) merge into the node in key order (Sec. 4.3.2). */
    uint64_t* ik = (uint64_t*)malloc((cnt + 1) * sizeof(uint64_t));
    uint64_t* iv = (uint64_t*)malloc((cnt + 1) * sizeof(uint64_t));
    uint32_t ni = 0;
    for (uint64_t j = 0; j < cnt; j++) {
        if (ue[j] != EFF_INS && ue[j] != EFF_UPS) continue;
        ik[ni] = uk[j]; iv[ni] = uv[j]; ni++;
    }
    uint64_t* rk = (uint64_t*)malloc((c + ni + 1) * sizeof(uint64_t));
    uint64_t* rv = (uint64_t*)malloc((c + ni + 1) * sizeof(uint64_t));
    uint64_t t = om_merge_insert(ck, c, ik, ni, rk);
    {   /* carry the values along the merge */
        uint32_t a = 0, b = 0;
        for (uint64_t o = 0; o < t; o++) {
            if (a < c && ck[a] == rk[o]) { rv[o] = cv[a]; a++; if (b < ni && ik[b] == rk[o]) b++; }
            else { rv[o] = iv[b]; b++; }
        }
    }

    /* (iii) canonical layout: the node keeps piece 0, new nodes take the rest. */
    uint64_t old_bound = m->bound[node];
    int64_t old_next = m->next[node];
    uint32_t* ps = (uint32_t*)malloc(((t / (NS / 2)) + 2) * sizeof(uint32_t));
    uint32_t q = om_canonical_layout(t, NS, ps);
    int64_t cur = node;
    uint64_t o = 0;
    for (uint32_t r = 0; r < q; r++) {
        if (r > 0) {
            int64_t nn = node_alloc(m);
            m->next[cur] = nn;
            cur = nn;
        }
        for (uint32_t s = 0; s < ps[r]; s++, o++) {
            m->keys[cur * NS + s] = rk[o];
            m->vals[cur * NS + s] = rv[o];
        }
        m->size[cur] = ps[r];
        m->bound[cur] = (r + 1 < q) ? rk[o - 1] : old_bound;
    }
    if (q > 0) m->next[cur] = old_next;
    *tail = q > 0 ? cur : NIL;
    if (q == 0) m->size[node] = 0;
    free(dk); free(ck); free(cv); free(shift); free(ik); free(iv); free(rk); free(rv); free(ps);
    return t;
}

/* One bucket applies its sublist (Sec. 4.1: walk node-links to the first node with k <= maxKey). */
static void model_apply_bucket(om_model* m, uint64_t b, const uint64_t* uk, const int* ue,
                               const uint64_t* uv, uint64_t cnt)
{
    int64_t node = m->head[b];
    int64_t prev = NIL;           /* last node kept so far in chain order */
    int64_t* dropped = (int64_t*)malloc((cnt + 2) * sizeof(int64_t));
    uint64_t nd = 0;
    int last_dropped = 0;
    uint64_t j = 0;
    while (j < cnt && node != NIL) {
        int64_t nx = m->next[node];
        uint64_t k = j;
        while (k < cnt && uk[k] <= m->bound[node]) k++;
        if (k == j) { prev = node; node = nx; continue; }
        int64_t tail;
        uint64_t t = model_apply_node(m, node, uk + j, ue + j, uv + j, k - j, &tail);
        if (t == 0) {
            if (prev == NIL) m->head[b] = nx; else m->next[prev] = nx;
            dropped[nd++] = node;
            last_dropped = (nx == NIL);
        } else {
            if (prev == NIL) m->head[b] = node; else m->next[prev] = node;
            prev = tail;
            last_dropped = 0;
        }
        j = k;
        node = nx;
    }
    if (m->head[b] == NIL) {
        /* the whole chain emptied: its first node stays as the bucket's only, empty node */
        int64_t keep = dropped[0];
        m->size[keep] = 0;
        m->bound[keep] = m->mkba[b];
        m->next[keep] = NIL;
        m->head[b] = keep;
        for (uint64_t i = 1; i < nd; i++) node_free(m, dropped[i]);
    } else {
        if (last_dropped) m->bound[prev] = m->mkba[b];   /* maxBucket passes to the new last node */
        for (uint64_t i = 0; i < nd; i++) node_free(m, dropped[i]);
    }
    free(dropped);
}

/* Underfull-node merge (the paper names it as a possible addition to deletion, Sec. 5.4.1, and
 * restructuring merges underfull nodes into half-full ones, Sec. 6.6).  Reading: walk the bucket's
 * chain; while the current node and the next one hold at most NS/2 pairs together, the next node's
 * pairs are appended to the current node (they are all larger), the current node takes over its
 * maxKey and node-link, and the next node is freed; otherwise the walk moves on to the next node.
 * The merged node is at most half full.  Returns the number of nodes freed. */
static uint64_t model_merge_underfull(om_model* m, uint64_t b)
{
    const uint32_t NS = m->NS;
    uint64_t freed = 0;
    int64_t a = m->head[b];
    while (a != NIL && m->next[a] != NIL) {
        int64_t x = m->next[a];
        if (m->size[a] + m->size[x] <= NS / 2) {
            for (uint32_t s = 0; s < m->size[x]; s++) {
                m->keys[a * NS + m->size[a] + s] = m->keys[x * NS + s];
                m->vals[a * NS + m->size[a] + s] = m->vals[x * NS + s];
            }
            m->size[a] += m->size[x];
            m->bound[a] = m->bound[x];
            m->next[a] = m->next[x];
            node_free(m, x);
            freed++;
        } else {
            a = x;
        }
    }
    return freed;
}

/* Elastic bucket split (Sec. 3.4: buckets with long chains of nodes may be split, which narrows the
 * key range each bucket covers).  Reading: a bucket whose chain holds more than T nodes (among the
 * flagged buckets; all of them when flags is NULL) becomes one bucket per node, in chain order, and
 * each new bucket's maxBucket is its node's maxKey (the chain's last node already carries the old
 * maxBucket).  No pair moves.  Returns the number of buckets added. */
static uint64_t model_split(om_model* m, uint64_t T, const uint8_t* flags)
{
    uint64_t nb2 = 0;
    for (uint64_t b = 0; b < m->nb; b++) {
        uint64_t L = 0;
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x]) L++;
        nb2 += ((!flags || flags[b]) && L > T) ? L : 1;
    }
    if (nb2 == m->nb) return 0;
    uint64_t* mk2 = (uint64_t*)malloc(nb2 * sizeof(uint64_t));
    int64_t* hd2 = (int64_t*)malloc(nb2 * sizeof(int64_t));
    uint64_t o = 0;
    for (uint64_t b = 0; b < m->nb; b++) {
        uint64_t L = 0;
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x]) L++;
        if ((!flags || flags[b]) && L > T) {
            int64_t x = m->head[b];
            while (x != NIL) {
                int64_t nx = m->next[x];
                hd2[o] = x;
                mk2[o] = m->bound[x];
                m->next[x] = NIL;
                o++;
                x = nx;
            }
        } else {
            hd2[o] = m->head[b];
            mk2[o] = m->mkba[b];
            o++;
        }
    }
    uint64_t added = nb2 - m->nb;
    free(m->mkba);
    free(m->head);
    m->mkba = mk2;
    m->head = hd2;
    m->nb = m->nb_cap = nb2;
    return added;
}

uint64_t om_model_split_chains(om_model* m, uint64_t T) { return model_split(m, T, NULL); }

uint64_t om_model_merge_underfull_all(om_model* m)
{
    uint64_t freed = 0;
    for (uint64_t b = 0; b < m->nb; b++) freed += model_merge_underfull(m, b);
    return freed;
}

void om_model_set_policy(om_model* m, uint64_t split_over, int merge_underfull)
{
    m->split_over = split_over;
    m->merge_underfull = merge_underfull;
}

/* Inserts and deletes of one batch: sort the update list, reduce each key's run to its net effect,
 * then every bucket pulls its sublist by binary search (Sec. 3.3, Sec. 4.1).  With the maintenance
 * policy on, every bucket whose sublist was non-empty then merges its underfull neighbours, and
 * after all buckets are done those touched buckets with chains longer than split_over are split.
 * Returns -1 (unchanged) if an insert carries KEY_MAX. */
int om_model_update(om_model* m, uint64_t n, const uint8_t* ops, const uint64_t* keys, const uint64_t* aux)
{
    uint64_t u = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (ops[i] == OP_INSERT && keys[i] >= m->kmax) return -1;
        if (ops[i] == OP_INSERT || ops[i] == OP_DELETE) u++;
    }
    orec* r = (orec*)malloc((u ? u : 1) * sizeof(orec));
    u = 0;
    for (uint64_t i = 0; i < n; i++) {
        if (ops[i] != OP_INSERT && ops[i] != OP_DELETE) continue;
        r[u].key = keys[i]; r[u].val = ops[i] == OP_INSERT ? aux[i] : 0; r[u].pos = i; r[u].op = ops[i];
        u++;
    }
    qsort(r, u, sizeof(orec), cmp_key_pos);
    uint64_t* uk = (uint64_t*)malloc((u + 1) * sizeof(uint64_t));
    uint64_t* uv = (uint64_t*)malloc((u + 1) * sizeof(uint64_t));
    int* ue = (int*)malloc((u + 1) * sizeof(int));
    uint64_t U = 0;
    for (uint64_t j = 0; j < u;) {
        uint64_t e = j;
        while (e < u && r[e].key == r[j].key) e++;
        uint64_t val = 0;
        int eff = run_effect(r + j, e - j, &val);
        uk[U] = r[j].key; uv[U] = val; ue[U] = eff; U++;
        j = e;
    }
    uint8_t* touched = (uint8_t*)calloc(m->nb ? m->nb : 1, 1);
    for (uint64_t b = 0; b < m->nb; b++) {
        uint64_t start = b == 0 ? 0 : upper_bound_u64(uk, U, m->mkba[b - 1]);
        uint64_t end = upper_bound_u64(uk, U, m->mkba[b]);
        if (start < end) {
            model_apply_bucket(m, b, uk + start, ue + start, uv + start, end - start);
            touched[b] = 1;
            if (m->merge_underfull) model_merge_underfull(m, b);
        }
    }
    if (m->split_over) model_split(m, m->split_over, touched);
    free(touched);
    free(r); free(uk); free(uv); free(ue);
    return 0;
}

uint64_t om_model_live_keys(const om_model* m)
{
    uint64_t n = 0;
    for (uint64_t b = 0; b < m->nb; b++)
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x]) n += m->size[x];
    return n;
}

uint64_t om_model_nodes_used(const om_model* m) { return m->hw - m->nfree; }
uint64_t om_model_buckets(const om_model* m) { return m->nb; }

uint64_t om_model_max_chain(const om_model* m)
{
    uint64_t mx = 0;
    for (uint64_t b = 0; b < m->nb; b++) {
        uint64_t c = 0;
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x]) c++;
        if (c > mx) mx = c;
    }
    return mx;
}

/* Sec. 3.5: flatten every chain into single-node buckets at the build fill and reset the MKBA.
 * Returns the number of nodes recovered (used before minus used after). */
int64_t om_model_restructure(om_model* m)
{
    uint64_t before = om_model_nodes_used(m);
    uint64_t n = om_model_live_keys(m);
    uint64_t* k = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    uint64_t* v = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    uint64_t c = 0;
    for (uint64_t b = 0; b < m->nb; b++)
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x])
            for (uint32_t s = 0; s < m->size[x]; s++) {
                k[c] = m->keys[x * m->NS + s];
                v[c] = m->vals[x * m->NS + s];
                c++;
            }
    model_cut(m, k, v, c);
    free(k); free(v);
    return (int64_t)before - (int64_t)om_model_nodes_used(m);
}

/* Reads through the structure.  Queries are sorted by key and each bucket pulls its sublist by a
 * binary search for maxBucket_{i-1} (Sec. 3.3); each query walks to the first node with
 * k <= maxKey.  Output conventions match om_map_read (LOOKUP, SUCC and PRED only). */
void om_model_read(const om_model* m, uint64_t n, const uint8_t* ops, const uint64_t* keys,
                   uint64_t* out_val, uint8_t* out_found, uint64_t* out_key)
{
    const uint64_t none = m->kmax;
    orec* r = (orec*)malloc((n ? n : 1) * sizeof(orec));
    for (uint64_t i = 0; i < n; i++) {
        r[i].key = keys[i]; r[i].pos = i; r[i].op = ops[i]; r[i].val = 0;
        out_key[i] = none; out_val[i] = none; out_found[i] = 0;
    }
    qsort(r, n, sizeof(orec), cmp_key_pos);
    uint64_t* sk = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) sk[i] = r[i].key;
    for (uint64_t b = 0; b < m->nb; b++) {
        uint64_t start = b == 0 ? 0 : upper_bound_u64(sk, n, m->mkba[b - 1]);
        uint64_t end = upper_bound_u64(sk, n, m->mkba[b]);
        for (uint64_t j = start; j < end; j++) {
            uint64_t q = r[j].key, i = r[j].pos;
            int64_t x = m->head[b];
            while (q > m->bound[x]) x = m->next[x];
            const uint64_t* nk = m->keys + x * m->NS;
            uint32_t sz = m->size[x];
            uint32_t p = (uint32_t)lower_bound_u64(nk, sz, q);
            if (r[j].op == OP_LOOKUP) {
                if (p < sz && nk[p] == q) { out_key[i] = q; out_val[i] = m->vals[x * m->NS + p]; out_found[i] = 1; }
            } else if (r[j].op == OP_SUCC) {
                /* the smallest stored key >= q: in this node, else the first key of the next
                 * non-empty node in chain and bucket order */
                uint64_t bb = b;
                while (p >= m->size[x]) {
                    p = 0;
                    x = m->next[x];
                    while (x == NIL) {
                        if (++bb >= m->nb) break;
                        x = m->head[bb];
                    }
                    if (x == NIL) break;
                }
                if (x != NIL) { out_key[i] = m->keys[x * m->NS + p]; out_val[i] = m->vals[x * m->NS + p]; out_found[i] = 1; }
            } else if (r[j].op == OP_PRED) {
                /* the largest stored key <= q: in this node below the first key > q, else the last
                 * key of the nearest non-empty node before it in chain and bucket order */
                uint32_t pu = (uint32_t)upper_bound_u64(nk, sz, q);
                int64_t px = NIL;
                uint32_t pp = 0;
                if (pu > 0) {
                    px = x;
                    pp = pu - 1;
                } else {
                    /* earlier nodes of this bucket's chain */
                    for (int64_t y = m->head[b]; y != x; y = m->next[y])
                        if (m->size[y] > 0) { px = y; pp = m->size[y] - 1; }
                    /* else the last non-empty node of an earlier bucket */
                    for (int64_t bb = (int64_t)b - 1; px == NIL && bb >= 0; bb--)
                        for (int64_t y = m->head[bb]; y != NIL; y = m->next[y])
                            if (m->size[y] > 0) { px = y; pp = m->size[y] - 1; }
                }
                if (px != NIL) { out_key[i] = m->keys[px * m->NS + pp]; out_val[i] = m->vals[px * m->NS + pp]; out_found[i] = 1; }
            }
        }
    }
    free(r); free(sk);
}

/* Layout dump in bucket and chain order.  With NULL arrays only the counts are written:
 * counts[0] = buckets, counts[1] = nodes in chains, counts[2] = live keys. */
void om_model_dump(const om_model* m, uint64_t* counts, uint64_t* mkba, uint32_t* chain_len,
                   uint32_t* node_size, uint64_t* node_bound, uint64_t* keys, uint64_t* vals)
{
    uint64_t nn = 0, nk = 0;
    for (uint64_t b = 0; b < m->nb; b++) {
        uint32_t c = 0;
        for (int64_t x = m->head[b]; x != NIL; x = m->next[x]) {
            if (node_size) { node_size[nn] = m->size[x]; node_bound[nn] = m->bound[x]; }
            if (keys)
                for (uint32_t s = 0; s < m->size[x]; s++) {
                    keys[nk + s] = m->keys[x * m->NS + s];
                    vals[nk + s] = m->vals[x * m->NS + s];
                }
            nn++;
            nk += m->size[x];
            c++;
        }
        if (chain_len) chain_len[b] = c;
        if (mkba) mkba[b] = m->mkba[b];
    }
    counts[0] = m->nb;
    counts[1] = nn;
    counts[2] = nk;
}

/* Invariant check.  Returns 0 when all hold, else the number of the first violated invariant:
 *  1 MKBA strictly increasing, last entry KEY_MAX
 *  2 every chain non-empty, node bounds strictly increasing, last node bound == maxBucket
 *  3 keys strictly increasing inside a node and inside (previous bound, bound]
 *  4 0 <= size <= NS, and a size-0 node only as a bucket's only node
 *  5 nodes in chains + free nodes == nodes ever allocated
 *  6 (only if build_shape) every node holds exactly p keys except the last bucket's (1..p) */
int om_model_check(const om_model* m, int build_shape)
{
    uint64_t in_chains = 0;
    for (uint64_t b = 0; b < m->nb; b++) {
        if (b > 0 && !(m->mkba[b - 1] < m->mkba[b])) return 1;
        if (b + 1 == m->nb && m->mkba[b] != m->kmax) return 1;
        int64_t x = m->head[b];
        if (x == NIL) return 2;
        int have_lo = b > 0;
        uint64_t lo = b > 0 ? m->mkba[b - 1] : 0;
        uint64_t chain = 0;
        int64_t last = NIL;
        for (; x != NIL; x = m->next[x]) {
            chain++;
            in_chains++;
            if (chain > m->hw) return 2;
            uint32_t sz = m->size[x];
            if (sz > m->NS) return 4;
            if (last != NIL && !(m->bound[last] < m->bound[x])) return 2;
            for (uint32_t s = 0; s < sz; s++) {
                uint64_t k = m->keys[x * m->NS + s];
                if (have_lo && !(k > lo)) return 3;
                if (!(k <= m->bound[x])) return 3;
                if (s > 0 && !(m->keys[x * m->NS + s - 1] < k)) return 3;
            }
            lo = m->bound[x];
            have_lo = 1;
            last = x;
        }
        if (m->bound[last] != m->mkba[b]) return 2;
        if (chain > 1)
            for (x = m->head[b]; x != NIL; x = m->next[x])
                if (m->size[x] == 0) return 4;
        if (build_shape) {
            if (chain != 1) return 6;
            uint32_t sz = m->size[m->head[b]];
            if (b + 1 < m->nb ? sz != m->p : (sz > m->p || (m->nb > 1 && sz == 0))) return 6;
        }
    }
    if (in_chains + m->nfree != m->hw) return 5;
    return 0;
}

/* ------------------------------------------------------------------------------------------------
 * 3. Batch-synchronous map on all host cores
 * ---------------------------------------------------------------------------------------------- */

typedef struct {
    const om_map* m;
    size_t lo, hi;
    const uint8_t* ops;
    const uint64_t *keys, *aux;
    uint64_t *out_val, *out_key, *cnt;
    uint8_t* out_found;
    const uint64_t* range_off;
    uint64_t *rkeys, *rvals;
} mt_read_job;

static void* mt_read_part(void* arg)
{
    mt_read_job* j = (mt_read_job*)arg;
    const size_t n = j->hi - j->lo;
    uint64_t* off = (uint64_t*)malloc((n + 1) * sizeof(uint64_t));
    om_map_read(j->m, n, j->ops + j->lo, j->keys + j->lo, j->aux + j->lo, j->out_val ? j->out_val + j->lo : NULL,
                j->out_found ? j->out_found + j->lo : NULL, j->out_key ? j->out_key + j->lo : NULL, off);
    for (size_t i = 0; i < n; i++) j->cnt[j->lo + i] = off[i + 1] - off[i];
    free(off);
    return NULL;
}

static void* mt_fill_part(void* arg)
{
    mt_read_job* j = (mt_read_job*)arg;
    om_map_range_fill(j->m, j->hi - j->lo, j->ops + j->lo, j->keys + j->lo, j->aux + j->lo, j->range_off + j->lo,
                      j->rkeys, j->rvals);
    return NULL;
}

static int clamp_threads(int t) { return t < 1 ? 1 : (t > 256 ? 256 : t); }

/* om_map_read on nthreads threads (same outputs); range_off is required. */
void om_map_read_mt(const om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys, const uint64_t* aux,
                    uint64_t* out_val, uint8_t* out_found, uint64_t* out_key, uint64_t* range_off, int nthreads)
{
    const int T = clamp_threads(nthreads);
    pthread_t th[256];
    mt_read_job jb[256];
    uint64_t* cnt = (uint64_t*)malloc((n ? n : 1) * sizeof(uint64_t));
    for (int t = 0; t < T; t++) {
        mt_read_job j = {m, n * t / T, n * (t + 1) / T, ops, keys, aux, out_val, out_key, cnt, out_found, NULL, NULL, NULL};
        jb[t] = j;
        pthread_create(&th[t], NULL, mt_read_part, &jb[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
    range_off[0] = 0;
    for (size_t i = 0; i < n; i++) range_off[i + 1] = range_off[i] + cnt[i];
    free(cnt);
}

/* om_map_range_fill on nthreads threads. */
void om_map_range_fill_mt(const om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys, const uint64_t* aux,
                          const uint64_t* range_off, uint64_t* rkeys, uint64_t* rvals, int nthreads)
{
    const int T = clamp_threads(nthreads);
    pthread_t th[256];
    mt_read_job jb[256];
    for (int t = 0; t < T; t++) {
        mt_read_job j = {m, n * t / T, n * (t + 1) / T, ops, keys, aux, NULL, NULL, NULL, NULL, range_off, rkeys, rvals};
        jb[t] = j;
        pthread_create(&th[t], NULL, mt_fill_part, &jb[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
}

typedef struct {
    const om_map* m;
    const orec* r;
    size_t rlo, rhi;      /* this thread's update records (whole key runs) */
    size_t mlo, mhi;      /* the map slots with keys in its key range */
    uint64_t *nk, *nv;    /* output arrays (NULL: count only) */
    size_t out0, cnt;
} mt_merge_job;

/* The merge of one key range: map slots [mlo, mhi) and update records [rlo, rhi), each key's run
 * replayed on that key's prior state (as om_map_update). */
static void* mt_merge_part(void* arg)
{
    mt_merge_job* j = (mt_merge_job*)arg;
    const om_map* m = j->m;
    size_t i = j->mlo, k = j->rlo, c = 0;
    while (i < j->mhi || k < j->rhi) {
        if (k >= j->rhi || (i < j->mhi && m->k[i] < j->r[k].key)) {
            if (j->nk) { j->nk[j->out0 + c] = m->k[i]; j->nv[j->out0 + c] = m->v[i]; }
            c++; i++;
            continue;
        }
        size_t e = k;
        while (e < j->rhi && j->r[e].key == j->r[k].key) e++;
        int present = 0;
        uint64_t val = 0;
        if (i < j->mhi && m->k[i] == j->r[k].key) { present = 1; val = m->v[i]; i++; }
        apply_run(j->r + k, e - k, &present, &val);
        if (present) {
            if (j->nk) { j->nk[j->out0 + c] = j->r[k].key; j->nv[j->out0 + c] = val; }
            c++;
        }
        k = e;
    }
    j->cnt = c;
    return NULL;
}

/* om_map_update on nthreads threads (same result). */
int om_map_update_mt(om_map* m, size_t n, const uint8_t* ops, const uint64_t* keys, const uint64_t* aux,
                     int nthreads)
{
    size_t u = 0;
    for (size_t i = 0; i < n; i++) {
        if (ops[i] == OP_INSERT && keys[i] >= m->kmax) return -1;
        if (ops[i] == OP_INSERT || ops[i] == OP_DELETE) u++;
    }
    orec* r = (orec*)malloc((u ? u : 1) * sizeof(orec));
    u = 0;
    for (size_t i = 0; i < n; i++) {
        if (ops[i] != OP_INSERT && ops[i] != OP_DELETE) continue;
        r[u].key = keys[i];
        r[u].val = ops[i] == OP_INSERT ? aux[i] : 0;
        r[u].pos = i;
        r[u].op = ops[i];
        u++;
    }
    qsort(r, u, sizeof(orec), cmp_key_pos);
    const int T = clamp_threads(nthreads);
    pthread_t th[256];
    mt_merge_job jb[256];
    /* thread t owns the update records from split t (moved forward to a key boundary) and the map
     * keys below the next thread's first record key */
    size_t split[257];
    for (int t = 0; t <= T; t++) {
        size_t s = u * (size_t)t / (size_t)T;
        while (s > 0 && s < u && r[s].key == r[s - 1].key) s++;
        split[t] = s;
    }
    for (int t = 1; t <= T; t++)
        if (split[t] < split[t - 1]) split[t] = split[t - 1];
    for (int t = 0; t < T; t++) {
        mt_merge_job j;
        memset(&j, 0, sizeof(j));
        j.m = m;
        j.r = r;
        j.rlo = split[t];
        j.rhi = split[t + 1];
        j.mlo = t == 0 ? 0 : (split[t] < u ? lower_bound_u64(m->k, m->n, r[split[t]].key) : m->n);
        j.mhi = t + 1 == T ? m->n : (split[t + 1] < u ? lower_bound_u64(m->k, m->n, r[split[t + 1]].key) : m->n);
        jb[t] = j;
        pthread_create(&th[t], NULL, mt_merge_part, &jb[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
    size_t total = 0;
    for (int t = 0; t < T; t++) { jb[t].out0 = total; total += jb[t].cnt; }
    uint64_t* nk = (uint64_t*)malloc((total + 1) * sizeof(uint64_t));
    uint64_t* nv = (uint64_t*)malloc((total + 1) * sizeof(uint64_t));
    for (int t = 0; t < T; t++) {
        jb[t].nk = nk;
        jb[t].nv = nv;
        pthread_create(&th[t], NULL, mt_merge_part, &jb[t]);
    }
    for (int t = 0; t < T; t++) pthread_join(th[t], NULL);
    free(m->k);
    free(m->v);
    m->k = nk;
    m->v = nv;
    m->n = total;
    free(r);
    return 0;
}
