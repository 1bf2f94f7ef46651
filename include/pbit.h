/*
 * pbit.h -- C ABI of the GB300 Pbit list sort.
 *
 * Pbit ("Pbit and other list sorting algorithms", D. S. Planeta) sorts a
 * singly-linked list of {next, data} nodes by splitting it on K-bit digits of
 * the key, most significant digit first, recursing into every bucket and
 * finally concatenating the sorted fragments (Sec. "The idea of sorting using
 * Pbit", Sec. "Implementation in C++", Sec. 5.1 "Function merge").  This
 * library computes the same result -- the list relinked in ascending order of
 * the low M bits of the key, equal keys kept in list order -- with GPU
 * kernels: list ranking, MSD digit passes, shared-memory finishing of small
 * buckets and a relink (next[s[i]] = s[i+1]).
 *
 * Conventions shared by every call
 *   - A node pool is caller-owned DEVICE memory: int32 successor indices
 *     (-1 = NULL) and keys of 1, 2, 4 or 8 bytes (unsigned unless
 *     PBIT_SIGNED).  SoA: next_stride_bytes = 4, key_stride_bytes = key
 *     width.  AoS {int32 next; uint32 key}: both strides 8, key = next + 4.
 *     Strides must be multiples of the element width.
 *   - next[] is relinked IN PLACE; key[] is only read.
 *   - 1 <= K <= 16, K divides M, 1 <= M <= 8 * key width; otherwise
 *     PBIT_EINVAL.  K is the paper's digit width (Sec. "The length of bit
 *     pattern"): unless the tune sets another, each GPU MSD pass splits on K
 *     bits (K <= 8) or on half of a K-bit level (K > 8).  The result does not
 *     depend on K or on the GPU's digit width: only the number of passes does.
 *   - Before anything is written to next[], the list shape is validated (every
 *     index in range, no cycle, exactly n nodes reachable from the root).  On
 *     any error next[] is left untouched and no root is written.
 *   - Calls are stream-ordered on the given stream (a cudaStream_t passed as
 *     void*, NULL = legacy default stream); calls that return a status read it
 *     back and therefore synchronize that stream.
 *   - The library never throws, and the sort calls never allocate device
 *     memory: the caller passes a workspace of pbit_workspace_size() bytes
 *     (256-byte aligned device memory).  Workspaces must not be shared by
 *     calls that may run concurrently.
 */
#ifndef PBIT_H
#define PBIT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PBIT_OK = 0,
    PBIT_EINVAL = 1,   /* bad argument (M, K, sizes, strides, pointers)           */
    PBIT_ENOMEM = 2,   /* workspace too small / server arena exhausted            */
    PBIT_EBADLIST = 3, /* cycle, wrong length, index out of range, bad root       */
    PBIT_ETIMEOUT = 4, /* a bounded device wait gave up                            */
    PBIT_ECUDA = 5,    /* a CUDA runtime call failed                               */
    PBIT_EAGAIN = 6,   /* server: request not admitted (queue full / over budget)  */
    PBIT_EPENDING = 7  /* server: request still running                            */
} pbit_status;

typedef enum { PBIT_U8 = 1, PBIT_U16 = 2, PBIT_U32 = 4, PBIT_U64 = 8 } pbit_key_type;

/* pool flags */
#define PBIT_SIGNED 1     /* keys are two's complement (needs M = 8 * width)     */
#define PBIT_DESCENDING 2 /* largest key first; equal keys still in list order   */
#define PBIT_DOUBLY 4     /* pool has prev[]: it is rebuilt after the relink     */
#define PBIT_FLOAT 8      /* keys are IEEE-754 binary32/binary64 (width 4 or 8)   */

typedef struct {
    int32_t *next;            /* device: successor index, -1 = NULL              */
    int64_t next_stride_bytes;/* 4 (SoA) or 8 (AoS)                                */
    const void *key;          /* device: keys                                      */
    int64_t key_stride_bytes; /* key width (SoA) or 8 (AoS)                        */
    int32_t key_type;         /* pbit_key_type                                     */
    int32_t flags;            /* PBIT_SIGNED | PBIT_DESCENDING | PBIT_DOUBLY ...   */
    int64_t pool_size;        /* number of nodes in the pool, < 2^31               */
    int32_t *prev;            /* device, only with PBIT_DOUBLY: predecessor index  */
    int64_t prev_stride_bytes;/* only with PBIT_DOUBLY                              */
} pbit_pool;

/* Tuning knobs; any field <= 0 takes the built-in / autotuned default. */
typedef struct {
    int32_t digit_bits;   /* GPU digit width per MSD pass, 1..8 bits (2^bits     */
                          /* buckets); <= 0: the call's K when K <= 8, else two  */
                          /* passes of ceil(K/2) bits per K-bit level (K = 16:   */
                          /* two 8-bit passes).  The result is the same for any */
                          /* width: it only changes the number of passes         */
    int32_t smem_cutoff;  /* buckets <= this many nodes are finished in smem     */
    int32_t ruler_stride; /* list ranking: one ruler per this many nodes (2^k)   */
    int32_t gather_pack;  /* 0: by size, 1: off, 2: on -- pack {next, key} per   */
                          /* node before the ranking walk (one random access     */
                          /* per hop instead of two)                             */
} pbit_tune;

/* Human-readable name of a status code (static string). */
const char *pbit_status_string(int status);

/*
 * Workspace bytes needed to sort up to `pool_size` nodes in `num_lists` lists
 * with keys of `key_type`, for the given tune (NULL = defaults).
 * Returns PBIT_OK or PBIT_EINVAL.
 */
pbit_status pbit_workspace_size(int64_t pool_size, int32_t num_lists, int32_t key_type,
                                const pbit_tune *tune, size_t *bytes);

/*
 * Sort ONE list (Sec. "Complete Pbit implementation": Pbit(L) returning the
 * new head).  The list starts at `root` and must contain exactly `n` nodes,
 * and n must equal pool->pool_size (every pool node is on the list).
 * root = -1 with n = 0 returns -1 (an empty list, as in the paper).
 * On PBIT_OK, *new_root_host (HOST memory) receives the index of the first
 * node of the sorted list.  Synchronizes `stream`.
 */
pbit_status pbit_sort_list(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                           int32_t *new_root_host, const pbit_tune *tune, void *ws,
                           size_t ws_bytes, void *stream);

/*
 * Sort `num_lists` independent lists sharing one pool in one segmented launch
 * sequence.  d_offsets (DEVICE, num_lists+1 int64, non-decreasing, last <=
 * pool_size): list i owns the nodes [d_offsets[i], d_offsets[i+1]) and must
 * contain every one of them; d_roots (DEVICE, num_lists int32) are the heads
 * (-1 for an empty list).  d_new_roots (DEVICE, num_lists int32) receives the
 * sorted heads.  Nodes outside every range are never touched.  tune = NULL
 * takes the autotuned choice for this size.  Synchronizes `stream`.
 */
pbit_status pbit_sort_lists_batched(const pbit_pool *pool, int32_t num_lists,
                                    const int32_t *d_roots, const int64_t *d_offsets, int32_t M,
                                    int32_t K, int32_t *d_new_roots, const pbit_tune *tune,
                                    void *ws, size_t ws_bytes, void *stream);

/*
 * Sort ONE list whose pool lives in HOST memory (pageable or pinned): the
 * pool is copied to the device part of the workspace, sorted there, and
 * next[] (and prev[] with PBIT_DOUBLY) copied back; key[] is only read.
 * Same contract as pbit_sort_list otherwise; host_pool's pointers are host
 * pointers.  The workspace (device) must hold pbit_workspace_size_host()
 * bytes.  For a list sorted through the relink windows, next[] is copied back
 * one window at a time on a stream the call creates (and destroys before it
 * returns), each window as soon as the kernel that writes it has run on
 * `stream`; without windows (short lists) or if that stream cannot be
 * created, one copy on `stream` after the sort.  Either way every copy has
 * completed when the call returns.  Synchronizes `stream`.
 */
pbit_status pbit_workspace_size_host(const pbit_pool *host_pool, const pbit_tune *tune, size_t *bytes);
pbit_status pbit_sort_list_host(const pbit_pool *host_pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                int32_t *new_root_host, const pbit_tune *tune, void *ws, size_t ws_bytes,
                                void *stream);

/*
 * pbit_sort_list without a workspace, for callers that cannot allocate device
 * memory (a process whose allocator has given all device memory to a
 * framework's pool, a loop where an allocation and the synchronization it
 * implies cannot be afforded, a wrapper whose API has no room for a
 * workspace).  The paper has no counterpart: this is a library convenience.
 *   - The scratch space is a fixed 8 MiB array in the library's device
 *     image; every GPU that loads the library holds it until the process
 *     exits.  Lists longer than 65536 nodes are rejected with PBIT_ENOMEM
 *     (nothing is written).
 *   - The call allocates nothing: no device memory, no pinned host memory,
 *     no CUDA event or stream.  It records no per-kernel profile
 *     (pbit_profile_read returns no entries after it); pbit_last_launch_count
 *     counts its launches.
 *   - Warm-up: the CUDA runtime loads kernels and the scratch array onto a
 *     device lazily, at their first use, and that load takes device memory.
 *     The first call on a device also looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.  So, on each device,
 *     for each key type and K in use, make one call with a list of more than
 *     4096 nodes and one with a shorter list (the two take different
 *     kernels) before the caller's
 *     allocator reserves the device's memory and before any stream capture on
 *     that device; from then on the calls take no device memory.  (Setting
 *     CUDA_MODULE_LOADING=EAGER in the environment loads every kernel when the
 *     process starts instead.)
 *   - All calls share the one array, which keeps the last call's contents;
 *     each call clears what it needs cleared.  Calls whose GPU work overlaps
 *     (other threads, other streams) race on the array: serialize them.
 * Same arguments, validation and result as pbit_sort_list (device pool,
 * pool_size == n, next[] relinked in place, *new_root_host on PBIT_OK);
 * synchronizes `stream`.
 */
pbit_status pbit_sort_list_noalloc(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                   int32_t *new_root_host, void *stream);

/*
 * Number of kernel launches the last sort call on this thread enqueued (for
 * benchmarks that report launches; 0 before any call).
 */
int64_t pbit_last_launch_count(void);

/*
 * Stage check (testing; not part of the method): runs the single-list
 * pipeline of pbit_sort_list (always the general path, never the one-kernel
 * path for short lists) only up to one stage and copies that stage's output
 * to the caller's device arrays, leaving next[] untouched.
 *   stage 1: the ranking -- d_idx[r] = the node at position r of the list
 *            (from the root), d_key[r] = its sort key (for unsigned ascending
 *            keys: key mod 2^M), the walk the paper's split loop makes along
 *            L->next (Sec. "Implementation in C++");
 *   stage 2: the first MSD pass -- the ranked nodes stably partitioned by
 *            bits [M-D, M) of their sort keys, D = the GPU digit width the
 *            call's K gives (K for K <= 8), buckets in ascending digit order:
 *            one level of the paper's split (Sec. "The idea of sorting using
 *            Pbit").  The list takes this pass whatever its length (a sort
 *            would finish short lists and small buckets in shared memory
 *            instead); a list of one node is refused with PBIT_EINVAL.  When
 *            bits [M-D, M) are equal in every key, the first iteration only
 *            moves the list on to its top varying bit, and when M <= D the
 *            pass writes the final order instead: d_idx / d_key are then
 *            unspecified.
 * d_idx holds n int32; d_key holds n keys of the pool's key width.  Same
 * argument checks, workspace and errors as pbit_sort_list, plus PBIT_EINVAL
 * for another stage; synchronizes `stream`.
 */
pbit_status pbit_debug_stage(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K, int32_t stage,
                             void *ws, size_t ws_bytes, int32_t *d_idx, void *d_key, void *stream);

/*
 * Self-test of the bounded device wait (failure detection; not part of the
 * method, which has no waits: the paper's sort is sequential).  One CTA
 * waits on a shared-memory mbarrier that nothing ever completes, through the
 * same bounded-wait routine with which the MSD pass waits for its tile
 * copies, polling at most `iterations` times (1 .. 2^24; the 2 s limit of
 * every device wait also applies).  When the wait gives up the kernel records
 * PBIT_ETIMEOUT in a device status word and returns, as the pass does; the
 * call reads the word back.  Expected result: PBIT_ETIMEOUT, with the CUDA
 * context still usable.  PBIT_EINVAL: `iterations` out of range (checked
 * before any CUDA call); PBIT_ECUDA: a CUDA call failed.  Allocates and frees
 * 4 bytes of device memory; synchronizes `stream` (a cudaStream_t, NULL = the
 * legacy default stream).
 */
pbit_status pbit_selftest_bounded_wait(int64_t iterations, void *stream);

/*
 * Per-kernel device timing (instrumentation; not part of the method).  While
 * enabled on a thread, every sort call on that thread records a CUDA event
 * after each kernel on its stream; pbit_profile_read() then returns, for the
 * last call, one entry per kernel kind: launches, summed device time in ms
 * (time between consecutive events) and the algorithmic bytes that kind of
 * kernel must move (reads + writes of its inputs and outputs).  Returns the
 * number of entries written, or -1 on a CUDA error.
 */
typedef struct {
    char name[24];
    int32_t launches;
    double ms;
    double bytes;
} pbit_kernel_stat;
void pbit_profile_enable(int32_t on);
int32_t pbit_profile_read(pbit_kernel_stat *out, int32_t max);

/* ------------------------------------------------------------ CUDA graphs
 * A sort call captured once as a CUDA graph and replayed.  The launch
 * sequence of a sort depends only on pool_size, num_lists, the key type, M
 * and the tune, never on the data: every replay re-reads next[], key[],
 * d_roots and d_offsets, so one graph sorts any lists laid out in the same
 * pool (different list orders, keys, or list lengths in d_offsets).  The
 * graph keeps the pointers it was created with: the pool, d_roots, d_offsets,
 * d_new_roots and the workspace must stay allocated, at the same addresses,
 * until pbit_graph_destroy.  Creating a graph enqueues no GPU work (the
 * capture runs on a private stream); the graph belongs to the device current
 * at creation.  Replays on one graph share its workspace: do not let two of
 * them overlap.
 */
typedef struct pbit_graph pbit_graph;
/* Capture pbit_sort_lists_batched(pool, num_lists, d_roots, d_offsets, M, K,
 * d_new_roots, tune, ws, ws_bytes) (same arguments and contract). */
pbit_status pbit_graph_create_batched(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                      const int64_t *d_offsets, int32_t M, int32_t K, int32_t *d_new_roots,
                                      const pbit_tune *tune, void *ws, size_t ws_bytes, pbit_graph **out);
/* Capture pbit_sort_list(pool, root, n, M, K, ...): root and n are fixed in
 * the graph; the new root is returned by pbit_graph_result. */
pbit_status pbit_graph_create_single(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                     const pbit_tune *tune, void *ws, size_t ws_bytes, pbit_graph **out);
/* Enqueue one replay on `stream` (asynchronous: no status read-back). */
pbit_status pbit_graph_launch(pbit_graph *g, void *stream);
/* Synchronize `stream` and return the status of the last replay enqueued on
 * it before this call; a single-list graph also writes *new_root_host. */
pbit_status pbit_graph_result(pbit_graph *g, void *stream, int32_t *new_root_host);
/* Number of nodes (memsets and kernels) in the graph. */
int64_t pbit_graph_node_count(const pbit_graph *g);
void pbit_graph_destroy(pbit_graph *g);

/* --------------------------------------------------------------- autotuner
 * Times the sort of the caller's batch under each candidate tune
 * (digit width 4/8 x shared-memory cutoff 128/256/512 x ruler stride
 * 16/32/64/128; `reps`
 * timed runs each after one warm-up, median kept) and returns the fastest in
 * *best (and its median time in *best_ms).  Candidates whose workspace
 * exceeds ws_bytes are skipped; pbit_autotune_workspace_size gives room for
 * all of them.  The pool is restored to its input state before every trial
 * and at the end (a temporary device copy of next[] / prev[] is allocated
 * for the call), so on return the lists are NOT sorted.  The choice is
 * remembered for this device, key type and size class (ceil log2 of
 * pool_size and of num_lists): later calls with tune == NULL on a pool of
 * that class take it whenever their workspace is large enough for it
 * (pbit_workspace_size with tune == NULL then returns room for it).  If the
 * environment variable PBIT_TUNE_FILE names a file, choices are appended to
 * it and read back from it by later processes.  Synchronizes `stream`.
 */
pbit_status pbit_autotune_workspace_size(int64_t pool_size, int32_t num_lists, int32_t key_type, size_t *bytes);
pbit_status pbit_autotune_batched(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                  const int64_t *d_offsets, int32_t M, int32_t K, int32_t *d_new_roots, void *ws,
                                  size_t ws_bytes, int32_t reps, void *stream, pbit_tune *best, float *best_ms);

/* ------------------------------------------------------------------ serving
 * A server owns a device arena of mem_budget_bytes on `device` and a
 * scheduler thread.  Requests queue in arrival order; the scheduler forms a
 * batch from the head of the queue plus compatible queued requests (same key
 * type, flags, M and K) and launches it as soon as one of its `streams` CUDA
 * streams is free and the batch's workspace fits in the free part of the
 * arena (first fit; the workspace returns to the arena when the batch
 * completes).  So the workspaces of the batches in flight never exceed the
 * budget, requests that arrive while others run on the GPU are admitted as
 * streams and memory free up (continuous batching), and a large request
 * waits only until enough memory is free (no later request overtakes the
 * head of the queue).  `tune` (NULL = defaults; copied) applies to every
 * batch, e.g. its digit width.  The caller owns each request's pool (device
 * memory) and keeps it alive until poll returns something other than
 * PBIT_EPENDING.
 */
typedef struct pbit_server pbit_server;

pbit_status pbit_serve_create(pbit_server **out, size_t mem_budget_bytes, int32_t device,
                              int32_t streams, int32_t max_batch, const pbit_tune *tune);
/* Queue one request; *ticket identifies it.  PBIT_EAGAIN if the request's
 * workspace alone exceeds the budget (it could never run); PBIT_EINVAL on bad
 * arguments. */
pbit_status pbit_serve_submit(pbit_server *s, const pbit_pool *pool, int32_t root, int64_t n,
                              int32_t M, int32_t K, uint64_t *ticket);
/* PBIT_EPENDING while queued or running; otherwise the request's final status,
 * with *new_root set on PBIT_OK.  A finished ticket may be polled again. */
pbit_status pbit_serve_poll(pbit_server *s, uint64_t ticket, int32_t *new_root);
/* Block until the ticket finishes (or timeout_ms elapses: PBIT_EPENDING). */
pbit_status pbit_serve_wait(pbit_server *s, uint64_t ticket, int32_t *new_root,
                            int64_t timeout_ms);
/* Host steady-clock times (ns) of a ticket's submission and of the moment
 * the scheduler saw it finish (0 while pending).  PBIT_EINVAL for an
 * unknown ticket. */
pbit_status pbit_serve_times(pbit_server *s, uint64_t ticket, int64_t *submit_ns, int64_t *done_ns);
/* Forget a finished ticket (its record is freed; polling it then returns
 * PBIT_EINVAL).  PBIT_EPENDING if it has not finished. */
pbit_status pbit_serve_release(pbit_server *s, uint64_t ticket);
/* Server counters: [0] submitted, [1] completed, [2] batches launched,
 * [3] max requests in one batch, [4] peak workspace bytes in flight. */
void pbit_serve_stats(pbit_server *s, int64_t *out5);
void pbit_serve_destroy(pbit_server *s);

#ifdef __cplusplus
}
#endif
#endif /* PBIT_H */
