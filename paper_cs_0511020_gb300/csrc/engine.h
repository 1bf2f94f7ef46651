// engine.h -- host-side pieces of the sort engine shared by the C ABI
// (engine.cu) and the request server (serve.cu).
#pragma once
#include <vector>

#include "pbit_internal.cuh"

namespace pbit {

struct Tune {
    int digit_bits;
    int cutoff;
    int log2S;
};

struct Sizes {
    int64_t ncap;
    int32_t L;
    int kb;
    Tune tune;
    int CH;
    int64_t R0, Rcap, chunk_cap, seg_cap, fin_cap, tile_cap;
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
bool resolve_tune(const pbit_tune *t, int64_t pool_size, int kb, Tune *out);
Sizes compute_sizes(int64_t ncap, int32_t L, int kb, const Tune &t, int sms);
size_t bind(const Sizes &z, unsigned char *ws, Ctx *c, MemsetList *ms);
pbit_status enqueue_sort(const Ctx &c, const MemsetList &ms, int mode, const ListDesc *tmpl,
                         const int64_t *d_offsets, const int32_t *d_roots, int M, cudaStream_t s, int sms,
                         int64_t *launches);
pbit_status map_status(int st);
bool check_pool(const pbit_pool *p, int M, int K);
bool prof_set(bool on);  // per-thread event profiling on/off; returns the previous state
ListDesc pool_template(const pbit_pool *p);

}  // namespace pbit
