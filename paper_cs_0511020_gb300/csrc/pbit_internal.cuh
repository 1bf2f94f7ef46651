// pbit_internal.cuh -- device-side layout and helpers shared by the kernels of
// the GB300 Pbit list sort.  Host orchestration is in engine.cu.
#pragma once
#include <type_traits>
#include <utility>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/pbit.h"

namespace pbit {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Internal status values beyond the ABI's pbit_status (never returned).
constexpr int kStOverflow = 100;  // a capacity computed on the host was exceeded

// ----------------------------------------------------------------- layouts
// One list as the kernels see it.  Node ids are "local" (0..n-1); the pool
// index of local node v is id_base + v; its sorted position lies in
// [out_base, out_base + n) of the order buffers.
struct ListDesc {
    int32_t *next;
    const unsigned char *key;
    int32_t *prev;
    int64_t next_stride;  // bytes
    int64_t key_stride;   // bytes
    int64_t prev_stride;  // bytes
    int32_t n;
    int32_t root;      // local root, -1 for an empty list
    int32_t id_base;
    int32_t out_base;
};

// A contiguous run of the order buffers that still has to be sorted on the
// key bits [0, hi); an active segment is split in the next pass on [lo, hi).
// buf = which of the two order buffers currently holds it.
struct Seg {
    int32_t start;
    int32_t len;
    int16_t lo;
    int16_t hi;
    int32_t buf;
    int32_t row;  // first row of its per-tile digit counts (tcnt)
    int32_t final;  // 1: keys are all equal; the pass writes it straight to F
};

// A small run (at most the finish capacity): sorted on bits [0, hi) by one
// warp and written to the final buffer.  buf = order buffer parity that
// holds it (low bit of mode_buf).
struct Fin {
    int32_t start;
    int32_t len;
    int32_t hi;
    int32_t mode_buf;  // (mode << 8) | buf
};

constexpr int kMaxIters = 64;
// Buckets of (cutoff, kMidCap] nodes are finished by one CTA each in shared
// memory instead of going through further global passes.
constexpr int kMidCap = 4096;
constexpr int kMidSmallCap = 2560;  // buckets up to this size: a CTA finish sized for them (more CTAs per SM)
constexpr int kMidSpan = 16;
// Lists of at most kSmallList nodes are sorted by one kernel, one CTA each.
constexpr int kSmallList = 4096;  // ... when at most this many of their key bits vary (4 windows)

// Elements per MSD pass tile (4- and 8-bit passes alike) and tiles per scan
// chunk: the plan kernels count tiles and chunks in these units.
constexpr int kPassTile = 2048;
// List positions per emit block (one block = one statistics tile of a list
// that starts at position 0).
constexpr int kEmitLog2 = 11;
constexpr int kEmitBlock = 1 << kEmitLog2;
static_assert(kEmitBlock == kPassTile, "an emit block is one pass tile");
constexpr int kScanChunk = 256;

// Work counters that many CTAs hit at once sit on their own 128-byte lines
// (an atomic on a line is serialized in one L2 slice).
struct alignas(128) HotCounter {
    int32_t v;
    int32_t pad[31];
};

struct Counters {
    HotCounter chunk_next;     // bump allocator of ranking chunks
    HotCounter task_next;      // work counter of the ranking walk
    HotCounter fin_ctr;        // work counter of the CTA finish
    HotCounter fin_ctr2;       // work counter of the CTA finish of the deferred (largest) buckets
    HotCounter rel_ctr;        // work counter of the relink partition
    int32_t n_virt;            // total nodes over all lists
    int32_t fin_count;
    int32_t mid_count;         // buckets finished by one CTA each
    int32_t defer_count;       // of those, left by the smaller CTA finish for the larger one
    int32_t act_count[2];
    int32_t pend_count[2];
    int32_t num_tiles[2];
    int32_t stat_tiles[2];
    int32_t brows[2];          // tcnt rows handed to the previous pass's buckets
    int32_t num_chunks[2];     // scan chunks of the pass
    // element counts for the per-kernel algorithmic-byte accounting
    long long pass_elems[kMaxIters];
    long long pass_final_elems[kMaxIters];
    long long stat_elems[kMaxIters];
    long long fin_sort_elems;
    long long fin_copy_elems;
    int32_t tile_ctr[kMaxIters];
    int32_t stat_ctr[kMaxIters];
    int32_t pad[16];
};

// Everything a kernel needs, passed by value.
struct Ctx {
    // problem
    int32_t num_lists;
    int32_t key_bytes;
    int32_t M;
    int32_t D;          // GPU digit width per pass (1..8; above 4: the 256-bucket passes)
    int32_t log2S;      // ruler stride S = 1 << log2S
    int32_t cutoff;     // buckets <= cutoff are finished in shared memory
    int32_t flags;      // PBIT_SIGNED | PBIT_DESCENDING | PBIT_FLOAT | PBIT_DOUBLY
    int32_t CH;         // ranking chunk entries
    int32_t shared_pool;       // all lists in one pool (blocked relink possible)
    int32_t force_pass;        // stage check: lists skip the finishes and take a global pass
    int64_t desc_next_stride;  // next[] stride of that pool
    int64_t ncap;       // capacity of the order buffers (pool size)
    int32_t R0;         // hash-ruler tasks
    int32_t Rcap;       // R0 + num_lists
    int64_t chunk_cap;
    int64_t seg_cap;    // active/pending segments per pass
    int64_t fin_cap;
    int64_t tile_cap;   // tiles per pass
    // arrays
    ListDesc *desc;
    int32_t *out_base;  // num_lists + 1 prefix (device copy of desc[].out_base)
    Counters *ctr;
    int32_t *status;
    int32_t *root_task;
    int32_t *task_list;
    int32_t *task_len;
    int32_t *task_succ;
    int64_t *wy[2];     // wy[0]: per task (succ << 32) | suffix length; wy[1]: per task
                        // (walk << 32) | nodes before it in its walk
    int64_t *sw[2];     // per ruler walk: (succ walk << 32) | nodes, pointer-jumping ping-pong
    int32_t Scap;       // ruler walks: ceil(Rcap / 32) + 1 + num_lists
    int32_t *chunk_task;
    int32_t *chunk_j0;
    int32_t *chunk_data;        // chunk_cap x CH node ids (virtual positions)
    unsigned char *chunk_key;   // chunk_cap x CH sort keys
    // emit: the chunks grouped by the block of kEmitBlock list positions
    // they fill (a chunk that runs into the next block is listed in both)
    int2 *chunk_pc;             // chunk_cap: {first list position, entries} (-1, 0: unused)
    int32_t *blk_cnt;           // blk_cap: chunks per block, then the fill cursors
    int32_t *blk_start;         // blk_cap + 1: first list entry of each block
    int2 *blk_list;             // 2 x chunk_cap: {chunk, (first position - block start + 32) | entries << 12}
    int64_t blk_cap;
    int32_t emit_hist;          // 1: the emit also counts the first 256-bucket pass's digits per tile
    unsigned char *keyb[2];
    int32_t *idxb[2];
    int32_t *F;
    // {next, sort key} packed per node in list-position order (8 bytes, 16
    // for 64-bit keys) so the ranking walk makes one random access per hop;
    // nullptr = the walk gathers next[] and key[] separately.  Aliases
    // keyb[1] / idxb[1] / F, which are idle until the first pass.
    unsigned char *pack;
    Seg *act[2];
    uint32_t *act_hist[2];      // seg_cap x 16 : histogram of the pass window (D > 4: seg_cap x 256
                                // bucket starts within the segment)
    int32_t *act_tile_base[2];  // seg_cap + 1
    int32_t *act_chunk_base[2]; // seg_cap + 1 : first scan chunk of the segment
    int32_t *act_nrow_base[2];  // seg_cap + 1 : first tcnt row of its buckets in the next pass
    uint32_t *tcnt[2];          // row_cap x 16 (D > 4: 256) : digit counts per pass tile -> exclusive prefixes
    uint32_t *ctot;             // scan_cap x 16 (D > 4: 256) : per scan chunk totals -> exclusive prefixes
    int64_t row_cap;
    int64_t scan_cap;
    unsigned long long *band[2];// seg_cap x 16
    unsigned long long *bor[2];
    Seg *pend[2];
    int32_t *pend_tile_base[2];
    unsigned long long *pand[2];
    unsigned long long *por[2];
    int4 *plan_cnt;             // seg_cap per-segment counts -> offsets
    int32_t *plan_mid;          // seg_cap per-segment mid-bucket counts -> offsets
    Fin *fin;
    Fin *mid;                   // mid_cap buckets of (cutoff, kMidCap] nodes: one CTA each
    int32_t *mid_defer;         // mid_cap: indices into mid of the buckets above kMidSmallCap nodes
    int64_t mid_cap;
    int32_t *rel_cursor;        // blocked relink: pairs per node block
    int32_t *new_roots;
};

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ void set_status(int32_t *st, int code) { atomicCAS(st, 0, code); }

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
    // MurmurHash3 finaliser (public domain, A. Appleby)
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// Position of the hash ruler of ruler block j (virtual positions [jS, jS+S)).
__device__ __forceinline__ int32_t ruler_of_block(int32_t j, int32_t log2S, int32_t n_virt) {
    int32_t base = j << log2S;
    int32_t blk = min(1 << log2S, n_virt - base);
    uint32_t h = fmix32((uint32_t)j * 0x9E3779B1u + 0x0511020u);
    int32_t off = (blk == (1 << log2S)) ? (int32_t)(h & ((1u << log2S) - 1)) : (int32_t)(h % (uint32_t)blk);
    return base + off;
}

__device__ __forceinline__ bool is_ruler(int32_t p, int32_t log2S, int32_t n_virt) {
    return ruler_of_block(p >> log2S, log2S, n_virt) == p;
}

// largest i in [0, n) with a[i] <= x (a non-decreasing, a[0] <= x)
__device__ __forceinline__ int32_t upper_index(const int32_t *a, int32_t n, int32_t x) {
    int32_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(a + mid) <= x)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ----------------------------------------------------------------- scans
__host__ __device__ constexpr int tiles_of(int64_t len, int64_t tile) { return (int)((len + tile - 1) / tile); }

// ---------------------------------------------------------------- scans
// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
__device__ __forceinline__ int block_excl_scan(int v, int *total, int *sh /* >= 33 ints */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < nw) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(kFull, s, o);
            if (lane >= o)
                s += y;
        }
        if (lane < nw)
            sh[lane] = s;  // inclusive warp totals
        if (lane == 31)
            sh[32] = s;
    }
    __syncthreads();
    int base = (wid > 0) ? sh[wid - 1] : 0;
    *total = sh[32];
    int r = base + x - v;
    __syncthreads();
    return r;
}

// Exclusive scan over the block, one value per thread, with one barrier:
// every warp scans its values, lane 31 posts the warp's total, and after the
// barrier each thread adds the totals of the warps before its own.  sh (one
// int per warp) must not be written again until the block has passed
// another barrier.
__device__ __forceinline__ int block_excl_scan_1bar(int v, int *total, int *sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o)
            x += y;
    }
    if (lane == 31)
        sh[wid] = x;
    __syncthreads();
    int before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
        const int t = sh[w];
        before += w < wid ? t : 0;
        tot += t;
    }
    *total = tot;
    return before + x - v;
}

// Stable rank of one lane's element among the elements of its 32-element
// group and of the warp's earlier groups that carry the same digit.  tab is
// the warp's table in shared memory, one {peer mask, running count} pair per
// digit, all masks zero on entry.  Each valid lane ORs its bit into its
// digit's mask; after the warp has synchronised the mask holds exactly the
// lanes with that digit (its peers).  Every peer reads the pair, and the
// lowest peer writes it back with the mask cleared and the count advanced by
// the number of peers; the lowest peers of one group hold distinct digits.
// Memory order = group, lane, so the rank is stable.  All lanes of the warp
// call it together; invalid lanes take part without an element.
__device__ __forceinline__ uint32_t warp_rank_by_or(uint2 *tab, unsigned dig, bool valid, unsigned lane_bit,
                                                    unsigned lt) {
    if (valid)
        atomicOr(&tab[dig].x, lane_bit);
    __syncwarp();
    const uint2 e = tab[dig];
    const unsigned below = e.x & lt;
    __syncwarp();  // every peer has read the pair before it is rewritten
    if (valid && below == 0)
        tab[dig] = make_uint2(0u, e.y + (uint32_t)__popc(e.x));
    __syncwarp();
    return e.y + (uint32_t)__popc(below);
}


// Keys up to 32 bits are handled in 32-bit words (digit shifts, AND/OR).
template <typename KeyT>
struct KeyWord {
    using U = typename std::conditional<sizeof(KeyT) <= 4, uint32_t, unsigned long long>::type;
};

template <typename KeyT>
__device__ __forceinline__ unsigned digit_of(KeyT k, int lo, unsigned mask) {
    return (unsigned)((typename KeyWord<KeyT>::U)k >> lo) & mask;
}

template <typename KeyT>
__device__ __forceinline__ KeyT load_key_raw(const unsigned char *p) {
    return *reinterpret_cast<const KeyT *>(p);
}

// Order-preserving transform of a key into the unsigned sort key of M bits.
template <typename KeyT>
__device__ __forceinline__ KeyT sort_key(KeyT k, int flags, int M) {
    constexpr int W = 8 * sizeof(KeyT);
    const KeyT sign = (KeyT)((KeyT)1 << (W - 1));
    if (flags & PBIT_FLOAT)
        k = (k & sign) ? (KeyT)~k : (KeyT)(k ^ sign);
    else if (flags & PBIT_SIGNED)
        k = (KeyT)(k ^ sign);
    if (flags & PBIT_DESCENDING)
        k = (KeyT)~k;
    if (M < W)
        k = (KeyT)(k & (KeyT)(((KeyT)1 << M) - 1));
    return k;
}

// ------------------------------------------------------------- launches
// Kernels of a sort are launched with programmatic stream serialization: a
// kernel may be scheduled while its predecessor drains (measured on this GPU:
// about 1.4 us per dependent launch instead of 4), so every kernel first
// waits for its predecessor's completion and memory (griddep_wait) before it
// touches anything an earlier kernel wrote.  Where a kernel does not follow
// another kernel the wait returns at once.
__device__ __forceinline__ void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Kernels enqueued by this host thread through launch_pdl (a sort call
// reports the difference across its enqueue as its launch count).
inline thread_local int64_t g_enqueued_launches = 0;

// Host side: when set, called after the blocked relink has enqueued on s the
// last kernel that writes next[] of pool nodes [lo, hi) (the host-buffer call
// starts copying that part of next[] back while the other windows are
// applied).
struct RelinkWindowHook {
    void (*fn)(void *arg, int64_t lo, int64_t hi, cudaStream_t s) = nullptr;
    void *arg = nullptr;
};
inline thread_local RelinkWindowHook g_relink_hook;

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    ++g_enqueued_launches;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Per-thread asynchronous global -> shared copies (4 or 8 bytes, aligned to
// their size); a thread waits for its own copies, a barrier then publishes
// them to the others.
template <int kBytes>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    static_assert(kBytes == 4 || kBytes == 8, "cp.async size");
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(smem);
    if constexpr (kBytes == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sa), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_group1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D bulk copy global -> shared (the TMA engine), completing on `bar`.
// dst, src and bytes must all be multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Every device-side wait gives up after this long and reports PBIT_ETIMEOUT.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

// Bounded wait on an mbarrier phase; false if the time or iteration limit
// was reached.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, long long limit) {
    const uint64_t t0 = globaltimer_ns();
    for (long long i = 0; i < limit; ++i) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((i & 255) == 255 && globaltimer_ns() - t0 > kWaitLimitNs)
            return false;
    }
    return false;
}

// ---------------------------------------------------------- launch helpers
struct Launch {
    int sms;
};

// Per-kernel event markers (profiling mode of engine.cu; no-ops otherwise):
// call after every launch with the kernel's name.
void prof_mark(const char *name, cudaStream_t s);

// kernel entry points (defined in rank.cu / msd.cu / finish.cu)
void launch_setup(const Ctx &c, const int64_t *d_offsets, const int32_t *d_roots, int mode,
                  const ListDesc *host_desc_tmpl, cudaStream_t s, int sms);
void launch_pack(const Ctx &c, cudaStream_t s, int sms);
void launch_walk(const Ctx &c, cudaStream_t s, int sms);
void launch_small(const Ctx &c, cudaStream_t s, int sms);  // every list <= kSmallList nodes
void launch_relink_direct(const Ctx &c, cudaStream_t s, int sms);
void launch_wyllie(const Ctx &c, cudaStream_t s, int sms, int rounds);
void launch_validate_emit(const Ctx &c, cudaStream_t s, int sms);
void launch_plan_init(const Ctx &c, cudaStream_t s);
void launch_iteration(const Ctx &c, int it, cudaStream_t s, int sms);   // D <= 4 here, else:
void launch_iteration8(const Ctx &c, int it, cudaStream_t s, int sms);  // windows of 5..8 bits (msd8.cu)
void launch_finish_relink(const Ctx &c, cudaStream_t s, int sms);
void launch_check_done(const Ctx &c, int iters, cudaStream_t s);
int finish_capacity();
bool relink_blocked(const Ctx &c);
int relink_bucket_bits(const Ctx &c);
int relink_max_buckets();
int pass_tile();
int stat_tile();
int digit_bits();       // widest window of the 16-bucket passes (4)
int wide_digit_bits();  // widest window of the 256-bucket passes (8)
int max_digit_bits();
int scan_rows();
int row_pad();

}  // namespace pbit
