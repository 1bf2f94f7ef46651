// engine.h -- host-side pieces of the sort engine shared by the C ABI
// (engine.cu) and the request server (serve.cu).
#pragma once
#include <vector>

#include "pbit_internal.cuh"

namespace pbit {

// Pools larger than this (next + key bytes) are packed before the walk
// (measured: the pack pays for itself from about 2^18 nodes on, even while
// the pool fits in L2).
constexpr int64_t kPackAutoBytes = 2ll << 20;

struct Tune {
    int digit_bits;  // GPU digit width per pass, 1..8 (0 only in workspace size queries)
    int cutoff;
    int log2S;
    int pack;  // 0 = by size, 1 = off, 2 = on (see Ctx::pack)
};

struct Sizes {
    int64_t ncap;
    int32_t L;
    int kb;
    Tune tune;
    int CH;
    int64_t R0, Rcap, chunk_cap, seg_cap, fin_cap, tile_cap, mid_cap;
    bool pack;
};

struct Memset {
    void *p;
    int v;
    size_t bytes;
};

// The memsets a sort call issues before its kernels (fixed capacity: a call
// makes no host allocation).
struct MemsetList {
    static constexpr int kCap = 48;
    Memset items[kCap];
    int count = 0;
    bool push(const Memset &m) {
        if (count == kCap)
            return false;
        items[count++] = m;
        return true;
    }
};

int device_sms();
// K: the call's digit width (0 = not known: digit_bits stays 0 unless the
// tune sets it, and workspace_bytes covers every width).
bool resolve_tune(const pbit_tune *t, int64_t pool_size, int kb, int K, Tune *out);
size_t workspace_bytes(int64_t ncap, int32_t L, int kb, Tune t, int sms);
Sizes compute_sizes(int64_t ncap, int32_t L, int kb, const Tune &t, int sms);
size_t bind(const Sizes &z, unsigned char *ws, Ctx *c, MemsetList *ms);
// small_lists: every list has at most kSmallList nodes (known on the host):
// one kernel sorts each list in shared memory instead of the whole pipeline.
// stop_after: 0 = the whole sort; 1 = stop after the ranking (list order in
// buffer 0); 2 = stop after the first MSD iteration (its output in buffer 1).
pbit_status enqueue_sort(const Ctx &c, const MemsetList &ms, int mode, const ListDesc *tmpl,
                         const int64_t *d_offsets, const int32_t *d_roots, int M, cudaStream_t s, int sms,
                         int64_t *launches, bool small_lists = false, int stop_after = 0);
pbit_status map_status(int st);
bool check_pool(const pbit_pool *p, int M, int K);
bool prof_set(bool on);  // per-thread event profiling on/off; returns the previous state
// Drop this thread's recorded profile, so pbit_profile_read reports nothing
// until the next profiled call.
void prof_forget();
// This thread's launch count of its last sort call (pbit_last_launch_count).
int64_t *last_launches_slot();
ListDesc pool_template(const pbit_pool *p);

// Enqueue a sort of a pool with list ranges (d_offsets) or of one list
// (d_offsets == nullptr: single_root, single_n); no synchronization.
pbit_status enqueue_pool(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                         const int64_t *d_offsets, int single_root, int64_t single_n, int M, int K,
                         int32_t *d_new_roots, const pbit_tune *tune, void *ws, size_t ws_bytes,
                         cudaStream_t s, Ctx *out, int stop_after = 0);

// Byte ranges of a pool: the next[] region, and the key[] / prev[] regions
// when they do not lie inside it (AoS keeps the key inside the node).
struct PoolSpan {
    size_t next_bytes, key_bytes, prev_bytes;
    bool key_inside;
    ptrdiff_t key_off;
};
PoolSpan pool_span(const pbit_pool *p);

// Tuned choices per (device, key width, size class), filled by the autotuner
// and optionally persisted in the file named by PBIT_TUNE_FILE.
bool tune_cache_lookup(int64_t pool_size, int32_t num_lists, int kb, pbit_tune *out);
void tune_cache_store(int64_t pool_size, int32_t num_lists, int kb, const pbit_tune &t, float ms);

}  // namespace pbit
