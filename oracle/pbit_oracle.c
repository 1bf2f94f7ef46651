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
 *   - recursion into every bucket while M > 0, otherwise concatenation of the
 *     leaf buckets with merge(A, B)             Sec. "Implementation in C++", Sec. 5.1 "Function merge"
 *   - ascending order: buckets visited from Omega-1 down to 0, each result
 *     becoming the "end marker" P of the next  Sec. "Differences between sorting in descending and ascending order"
 *   - descending order: buckets visited 0 .. Omega-1 (same section)
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
 *   - bucket tables are taken from the heap instead of the stack so that K up
 *     to 16 (Omega = 65536) does not exhaust the thread stack.
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

/* One recursive Pbit call on list L with M unsorted top bits and end marker P. */
static onode *opbit(onode *L, unsigned M, onode *P, ostate *st, uint64_t level)
{
    if (L == NULL)
        return P;
    if (level > st->depth)
        st->depth = level;
    M -= st->K;
    onode **tab = (onode **)calloc((size_t)st->omega, sizeof(onode *));
    if (tab == NULL) {
        st->oom = 1;
        return P;
    }
    /* split: every node goes to the front of the bucket named by its digit */
    while (L) {
        onode *i = L;
        onode **in = tab + ((L->data >> M) & (st->omega - 1));
        L = L->next;
        i->next = *in;
        *in = i;
        st->splits++;
    }
    if (!st->descending) {
        for (int64_t b = (int64_t)st->omega - 1; b >= 0; --b)
            P = M ? opbit(tab[b], M, P, st, level + 1) : omerge(tab[b], P, st);
    } else {
        for (int64_t b = 0; b < (int64_t)st->omega; ++b)
            P = M ? opbit(tab[b], M, P, st, level + 1) : omerge(tab[b], P, st);
    }
    free(tab);
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
        P = opbit(L, (unsigned)M, NULL, &st, 1);
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
            P = opbit(neg, (unsigned)M, opbit(nonneg, (unsigned)M, NULL, &st, 1), &st, 1);
        else
            P = opbit(nonneg, (unsigned)M, opbit(neg, (unsigned)M, NULL, &st, 1), &st, 1);
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
