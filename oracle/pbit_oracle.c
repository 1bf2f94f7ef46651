/*
 * pbit_oracle.c -- the Pbit oracle: a plain, slow, single-threaded CPU
 * restatement of the paper's list sort over real pointer nodes.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the package smoke check and the benchmark's
 * CPU-baseline leg do.  It shares no code, header, table or helper with the
 * CUDA library.
 *
 * What it follows (section names of the paper "Pbit and other list sorting
 * algorithms", D. S. Planeta):
 *   - node layout {next pointer, data}          Sec. "Structure of data representing a node"
 *   - the split loop: walk the list once, push each node onto the front of
 *     the bucket selected by the K-bit digit (data >> M) & (Omega-1), after
 *     M has been decreased by K                 Sec. "Implementation in C++", Sec. "Cutting bits off"
 *   - every bucket sorted the same way on the bits left while any are left,
 *     then the leaf buckets concatenated with merge(A, B)
 *                                               Sec. "Implementation in C++", Sec. 5.1 "Function merge"
 *   - ascending order: the output assembled from its far end, bucket Omega-1
 *     first, each lower bucket hung in front  Sec. "Differences between sorting in descending and ascending order"
 *   - descending order: bucket 0 first (same section)
 *   - signed keys: split into negatives and non-negatives by pushing onto two
 *     lists, sort both, concatenate           Sec. "Negative numbers sorting", Sec. "Complete Pbit implementation"
 *   - the merge-step counter (always n) and the split counter (n*M/K)
 *                                               Sec. 5.1 (instrumented merge), Sec. 3 (f(n) = (M/K)n + n)
 *
 * Readings taken where the paper is silent or inconsistent:
 *   - data is held as a 64-bit unsigned word whatever the key width; the
 *     digit (data >> M) & (Omega-1) only ever looks at bits below the key
 *     width, so the result equals that of the narrower TYPE.
 *   - the push-to-front split reverses the order of equal digits at every
 *     level, so the literal code keeps equal keys in list order only when the
 *     number of reversals (M/K, plus one for the signed split) is even.  The
 *     oracle reproduces the literal code exactly; the stable-sort definition
 *     used for the other cases lives in oracle.py.
 *   - the recursion is carried out with an explicit stack of lists still to
 *     be sorted (same visiting order), and the bucket table comes from the
 *     heap, so K up to 16 (Omega = 65536) and M up to 64 need no deep call
 *     stack.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct onode {
    struct onode *next;
    uint64_t data;
} onode;

typedef struct {
    unsigned K;
    uint64_t omega;
    int descending;
    uint64_t splits;      /* nodes pushed by split loops          */
    uint64_t merges;      /* nodes visited by merge (Sec. 5.1)    */
    uint64_t depth;       /* deepest recursion level reached      */
    int oom;
} ostate;

/* merge(A, B): walk to the last node of A and hang B behind it (Sec. 5.1). */
static onode *omerge(onode *A, onode *B, ostate *st)
{
    if (A == NULL)
        return B;
    onode *t = A;
    st->merges++;
    while (t->next) {
        t = t->next;
        st->merges++;
    }
    t->next = B;
    return A;
}

/*
 * Work that is still to be done: a list whose low `bits` bits are not yet
 * sorted (bits == 0: a finished leaf bucket, ready to be concatenated).
 */
typedef struct {
    onode *list;
    unsigned bits;
    uint64_t level;
} owork;

typedef struct {
    owork *item;
    size_t count, cap;
} ostack;

static int ostack_push(ostack *s, onode *list, unsigned bits, uint64_t level)
{
    if (s->count == s->cap) {
        size_t cap = s->cap ? 2 * s->cap : 256;
        owork *p = (owork *)realloc(s->item, cap * sizeof(owork));
        if (p == NULL)
            return 0;
        s->item = p;
        s->cap = cap;
    }
    s->item[s->count].list = list;
    s->item[s->count].bits = bits;
    s->item[s->count].level = level;
    s->count++;
    return 1;
}

/*
 * Sort list L on its low M bits and put the result in front of the list P
 * (the paper's third argument, the part of the output already built behind
 * it); returns the head of the combined list.
 *
 * The method (Sec. "The idea of sorting using Pbit", Sec. "Implementation in
 * C++"): take the K bits just below the bits already used (M is lowered by K
 * before the shift), and distribute the nodes over Omega = 2^K buckets by
 * that digit, each node going to the FRONT of its bucket; then sort every
 * bucket on the remaining bits the same way; a bucket with no bits left is a
 * finished piece and is concatenated with merge(A, B) (Sec. 5.1).  The output
 * is assembled from its far end: for ascending order the highest bucket is
 * finished first and each lower one is hung in front of it (Sec.
 * "Differences between sorting in descending and ascending order"; for
 * descending order bucket 0 is finished first).
 *
 * Instead of recursing, the lists still to be handled wait on an explicit
 * stack; the buckets of one split are pushed so that the one to be finished
 * first is on top, which visits them in the same order as the recursion.
 */
static onode *opbit(onode *L, unsigned M, onode *P, ostate *st)
{
    ostack todo = {NULL, 0, 0};
    onode **bucket = (onode **)malloc((size_t)st->omega * sizeof(onode *));
    if (bucket == NULL || !ostack_push(&todo, L, M, 1)) {
        st->oom = 1;
        free(bucket);
        free(todo.item);
        return P;
    }
    while (todo.count > 0) {
        owork w = todo.item[--todo.count];
        if (w.list == NULL)
            continue;
        if (w.bits == 0) {  /* a leaf bucket: concatenate it in front of P */
            P = omerge(w.list, P, st);
            continue;
        }
        if (w.level > st->depth)
            st->depth = w.level;
        const unsigned rest = w.bits - st->K;  /* bits left after this digit */
        memset(bucket, 0, (size_t)st->omega * sizeof(onode *));
        onode *node = w.list;
        while (node != NULL) {
            onode *following = node->next;
            const uint64_t digit = (node->data >> rest) & (st->omega - 1);
            node->next = bucket[digit];  /* to the front of its bucket */
            bucket[digit] = node;
            st->splits++;
            node = following;
        }
        /* the bucket finished first goes on the stack last */
        for (uint64_t j = 0; j < st->omega; ++j) {
            const uint64_t b = st->descending ? st->omega - 1 - j : j;
            if (!ostack_push(&todo, bucket[b], rest, w.level + 1)) {
                st->oom = 1;
                free(bucket);
                free(todo.item);
                return P;
            }
        }
    }
    free(bucket);
    free(todo.item);
    return P;
}

static uint64_t load_key(const void *key, int64_t stride, int key_bytes, int64_t v)
{
    const unsigned char *p = (const unsigned char *)key + v * stride;
    switch (key_bytes) {
    case 1: return *(const uint8_t *)p;
    case 2: { uint16_t x; memcpy(&x, p, 2); return x; }
    case 4: { uint32_t x; memcpy(&x, p, 4); return x; }
    default: { uint64_t x; memcpy(&x, p, 8); return x; }
    }
}

/*
 * Walk the list from root and write the node ids in list order.  Returns the
 * length, -1 if an index is out of range, -2 if more than max_len nodes are
 * seen (a cycle or a list longer than expected).
 */
int64_t pbit_oracle_list_order(int64_t pool_size, const int32_t *next, int64_t next_stride,
                               int32_t root, int32_t *order, int64_t max_len)
{
    int64_t len = 0;
    int32_t v = root;
    while (v != -1) {
        if (v < 0 || v >= pool_size)
            return -1;
        if (len >= max_len)
            return -2;
        order[len++] = v;
        v = *(const int32_t *)((const unsigned char *)next + (int64_t)v * next_stride);
    }
    return len;
}

/*
 * Sort the list starting at root with the literal Pbit.
 *   next_in / next_stride : pool of int32 successor indices, -1 = NULL
 *   key / key_stride      : keys (key_bytes = 1, 2, 4 or 8), unsigned or
 *                           two's complement when is_signed
 *   M, K                  : bits sorted, bits per digit (K divides M)
 *   next_out              : pool_size int32, receives the relinked successors
 *                           (nodes off the list keep next_in's value)
 *   counters[4]           : splits, merge steps, max recursion depth, length
 * Returns 0, or -1 bad arguments, -2 malformed list, -3 out of memory.
 */
int pbit_oracle_sort(int64_t pool_size, const int32_t *next_in, int64_t next_stride,
                     const void *key, int64_t key_stride, int key_bytes, int32_t root,
                     int M, int K, int is_signed, int descending, int32_t *next_out,
                     int32_t *root_out, uint64_t *counters)
{
    if (K < 1 || K > 16 || M < 1 || M > 8 * key_bytes || M % K != 0)
        return -1;
    if (is_signed && M != 8 * key_bytes)
        return -1;
    for (int64_t v = 0; v < pool_size; ++v)
        next_out[v] = *(const int32_t *)((const unsigned char *)next_in + v * next_stride);
    int32_t *order = (int32_t *)malloc((size_t)(pool_size > 0 ? pool_size : 1) * sizeof(int32_t));
    onode *nodes = (onode *)malloc((size_t)(pool_size > 0 ? pool_size : 1) * sizeof(onode));
    if (!order || !nodes) {
        free(order);
        free(nodes);
        return -3;
    }
    int64_t len = pbit_oracle_list_order(pool_size, next_in, next_stride, root, order, pool_size);
    if (len < 0) {
        free(order);
        free(nodes);
        return -2;
    }
    /* build the linked structure of real nodes, in list order */
    onode *L = NULL;
    for (int64_t r = len - 1; r >= 0; --r) {
        onode *nd = &nodes[order[r]];
        nd->data = load_key(key, key_stride, key_bytes, order[r]);
        nd->next = L;
        L = nd;
    }
    ostate st;
    memset(&st, 0, sizeof st);
    st.K = (unsigned)K;
    st.omega = (uint64_t)1 << K;
    st.descending = descending;
    onode *P;
    if (!is_signed) {
        P = opbit(L, (unsigned)M, NULL, &st);
    } else {
        /* sign split of the complete implementation: two push-built lists */
        uint64_t sign = (uint64_t)1 << (M - 1);
        onode *neg = NULL, *nonneg = NULL;
        while (L) {
            onode *t = L;
            L = L->next;
            if (t->data & sign) {
                t->next = neg;
                neg = t;
            } else {
                t->next = nonneg;
                nonneg = t;
            }
        }
        if (!descending)
            P = opbit(neg, (unsigned)M, opbit(nonneg, (unsigned)M, NULL, &st), &st);
        else
            P = opbit(nonneg, (unsigned)M, opbit(neg, (unsigned)M, NULL, &st), &st);
    }
    int rc = st.oom ? -3 : 0;
    if (rc == 0) {
        for (onode *p = P; p; p = p->next)
            next_out[p - nodes] = p->next ? (int32_t)(p->next - nodes) : -1;
        *root_out = P ? (int32_t)(P - nodes) : -1;
    }
    if (counters) {
        counters[0] = st.splits;
        counters[1] = st.merges;
        counters[2] = st.depth;
        counters[3] = (uint64_t)len;
    }
    free(order);
    free(nodes);
    return rc;
}

/*
 * One split step only (the loop of Sec. "Implementation in C++") at bit
 * position M-K on the list from root, for inspecting the buckets of the
 * worked example of Sec. 3.  bucket_of[r] receives the digit of the node at
 * list rank r, bucket_seq receives, bucket by bucket from 0 to Omega-1, the
 * node ids in the order the split leaves them inside each bucket, and
 * bucket_len[b] the size of bucket b.  Returns the list length or < 0.
 */
int64_t pbit_oracle_split_once(int64_t pool_size, const int32_t *next, const void *key,
                               int key_bytes, int32_t root, int M, int K, int32_t *bucket_seq,
                               int64_t *bucket_len)
{
    if (K < 1 || K > 16 || M < K || M > 8 * key_bytes)
        return -1;
    int32_t *order = (int32_t *)malloc((size_t)(pool_size > 0 ? pool_size : 1) * sizeof(int32_t));
    onode *nodes = (onode *)malloc((size_t)(pool_size > 0 ? pool_size : 1) * sizeof(onode));
    uint64_t omega = (uint64_t)1 << K;
    onode **tab = (onode **)calloc((size_t)omega, sizeof(onode *));
    if (!order || !nodes || !tab) {
        free(order);
        free(nodes);
        free(tab);
        return -3;
    }
    int64_t len = pbit_oracle_list_order(pool_size, next, 4, root, order, pool_size);
    if (len >= 0) {
        onode *L = NULL;
        for (int64_t r = len - 1; r >= 0; --r) {
            onode *nd = &nodes[order[r]];
            nd->data = load_key(key, key_bytes, key_bytes, order[r]);
            nd->next = L;
            L = nd;
        }
        unsigned m = (unsigned)(M - K);
        while (L) {
            onode *i = L;
            onode **in = tab + ((L->data >> m) & (omega - 1));
            L = L->next;
            i->next = *in;
            *in = i;
        }
        int64_t w = 0;
        for (uint64_t b = 0; b < omega; ++b) {
            int64_t c = 0;
            for (onode *p = tab[b]; p; p = p->next) {
                bucket_seq[w++] = (int32_t)(p - nodes);
                ++c;
            }
            bucket_len[b] = c;
        }
    }
    free(order);
    free(nodes);
    free(tab);
    return len;
}
