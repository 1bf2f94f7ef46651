// engine.cu -- host orchestration and the C ABI of include/pbit.h.
//
// One sort call = one stream-ordered sequence:
//   memsets -> setup -> pack -> walk -> ruler walks + pointer jumping
//   -> validate + emit -> plan_init
//   -> ceil(M/D) x [seg_stats, plan_pending, tile_scan, chunk_scan, pass,
//                   plan_count, plan_scan, plan_write]
//   -> check -> CTA finish (mid buckets) -> warp finish (small buckets)
//   -> relink -> status read-back;
// or, when every list has at most kSmallList nodes (known on the host),
//   memsets -> setup -> one-CTA-per-list sort -> direct relink.
// Kernels are launched with programmatic stream serialization (launch_pdl).
// The workspace is carved into fixed regions whose sizes depend only on the
// pool size, the number of lists, the key width and the tune; no call
// allocates device memory.
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include <nvtx3/nvToolsExt.h>

#include "engine.h"
#include "pbit_internal.cuh"

namespace pbit {

static thread_local int64_t g_last_launches = 0;

// ------------------------------------------------------------ profiling
// When enabled, every launch site records an event after its kernel; the
// time between consecutive events is charged to the kernel named there.
struct ProfState {
    bool on = false;
    std::vector<cudaEvent_t> pool;
    size_t used = 0;
    std::vector<std::pair<const char *, cudaEvent_t>> marks;
    cudaEvent_t start = nullptr;
    Counters ctr;
    bool have_ctr = false;
    int64_t n = 0, rcap = 0, scap = 0, rounds = 0;
    int kb = 4;
    bool blocked_relink = false;
    bool emit_hist = false;  // the emit counted the first pass's digits (its time is the emit's)
    bool pack = false;
    bool small = false;
};
static thread_local ProfState g_prof;

static cudaEvent_t prof_event() {
    if (g_prof.used == g_prof.pool.size()) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess)
            return nullptr;
        g_prof.pool.push_back(e);
    }
    return g_prof.pool[g_prof.used++];
}

void prof_mark(const char *name, cudaStream_t s) {
    if (!g_prof.on)
        return;
    cudaEvent_t e = prof_event();
    if (e && cudaEventRecord(e, s) == cudaSuccess)
        g_prof.marks.emplace_back(name, e);
}

bool prof_set(bool on) {
    const bool was = g_prof.on;
    g_prof.on = on;
    return was;
}

void prof_forget() {
    g_prof.marks.clear();
    g_prof.used = 0;
    g_prof.start = nullptr;
    g_prof.have_ctr = false;
}

int64_t *last_launches_slot() { return &g_last_launches; }

static void prof_begin(cudaStream_t s) {
    if (!g_prof.on)
        return;
    g_prof.used = 0;
    g_prof.marks.clear();
    g_prof.have_ctr = false;
    g_prof.start = prof_event();
    if (g_prof.start)
        cudaEventRecord(g_prof.start, s);
}

static inline size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// NVTX range over a scope: a profiler attached to the process shows when each
// stage's launches were enqueued (no cost without one).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

int device_sms() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return 148;
    static std::mutex mu;
    static std::unordered_map<int, int> cache;
    std::lock_guard<std::mutex> g(mu);
    auto it = cache.find(dev);
    if (it != cache.end())
        return it->second;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        sms = 148;
    cache[dev] = sms;
    return sms;
}

// GPU digit width of a call whose tune does not set one: the paper's K
// (Sec. "The length of bit pattern"), K bits per pass up to 8, and a level of
// more than 8 bits as two passes of ceil(K/2) bits (K = 16: two 8-bit passes).
static int digit_width_for_K(int K) { return K <= max_digit_bits() ? K : (K + 1) / 2; }

bool resolve_tune(const pbit_tune *t, int64_t pool_size, int kb, int K, Tune *out) {
    Tune r;
    r.digit_bits = K > 0 ? digit_width_for_K(K) : 0;  // 0: not known (workspace size queries)
    r.cutoff = finish_capacity();
    // Ruler stride: denser rulers for smaller pools, so there are enough
    // sub-walks to fill the GPU and the longest one stays short (measured:
    // stride 8 is fastest up to 2^23 nodes, 16 at 2^24-2^25, 32 above).
    r.log2S = pool_size <= (1ll << 23) ? 3 : (pool_size <= (1ll << 25) ? 4 : 5);
    r.pack = 0;
    if (t) {
        if (t->digit_bits > max_digit_bits())
            return false;
        if (t->digit_bits > 0)
            r.digit_bits = t->digit_bits;
        if (t->smem_cutoff > 0) {
            if (t->smem_cutoff > finish_capacity())
                return false;
            r.cutoff = t->smem_cutoff;
        }
        if (t->ruler_stride > 0) {
            int s = t->ruler_stride, l = 0;
            while ((1 << l) < s)
                ++l;
            if ((1 << l) != s || l < 1 || l > 12)
                return false;
            r.log2S = l;
        }
        if (t->gather_pack < 0 || t->gather_pack > 2)
            return false;
        r.pack = t->gather_pack;
    }
    (void)kb;
    *out = r;
    return true;
}

Sizes compute_sizes(int64_t ncap, int32_t L, int kb, const Tune &t, int sms) {
    Sizes z;
    z.ncap = ncap;
    z.L = L;
    z.kb = kb;
    z.tune = t;
    z.CH = 32;
    const int64_t S = 1ll << t.log2S;
    z.R0 = (ncap + S - 1) / S;
    z.Rcap = z.R0 + L;
    // slack: every walk warp may hold one partly used super-chunk of 64 chunks
    // (for the largest grid launch_walk uses: 8 CTAs of 8 warps per SM)
    const int64_t walk_blocks = std::min<int64_t>((int64_t)sms * 8, std::max<int64_t>(1, ((z.Rcap + 31) / 32 + 7) / 8));
    const int64_t walk_warps = walk_blocks * 8;
    z.chunk_cap = (ncap + z.CH - 1) / z.CH + z.Rcap + 64 * walk_warps + 64;
    z.seg_cap = ncap / (t.cutoff + 1) + 2;
    const int64_t iters = (8 * kb + t.digit_bits - 1) / t.digit_bits;
    // small buckets are disjoint and non-empty: at most one per node
    z.fin_cap = std::min<int64_t>(L + (int64_t)(1 << t.digit_bits) * iters * z.seg_cap, ncap + L) + 16;
    z.tile_cap = ncap / pass_tile() + z.seg_cap + 2;
    z.mid_cap = ncap / (t.cutoff + 1) + L + 16;  // disjoint buckets of more than cutoff nodes
    // A random gather costs a whole DRAM sector or more: the pack turns the
    // walk's two gathers per hop into one.
    z.pack = t.pack == 2 || (t.pack == 0 && ncap * (4 + kb) > kPackAutoBytes);
    return z;
}

// Carve the workspace.  With ws == nullptr only the size is computed.
size_t bind(const Sizes &z, unsigned char *ws, Ctx *c, MemsetList *ms) {
    size_t off = 0;
    auto take = [&](size_t bytes) -> unsigned char * {
        unsigned char *p = ws ? ws + off : nullptr;
        off += up256(bytes);
        return p;
    };
    auto zero = [&](void *p, int v, size_t bytes) {
        if (ms && p && !ms->push(Memset{p, v, bytes}))
            ms->count = -1;  // capacity exceeded: enqueue_sort refuses
    };
    Ctx x;
    std::memset(&x, 0, sizeof x);
    x.num_lists = z.L;
    x.key_bytes = z.kb;
    x.D = z.tune.digit_bits;
    x.log2S = z.tune.log2S;
    x.cutoff = z.tune.cutoff;
    x.CH = z.CH;
    x.ncap = z.ncap;
    x.R0 = (int32_t)z.R0;
    x.Rcap = (int32_t)z.Rcap;
    x.chunk_cap = z.chunk_cap;
    x.seg_cap = z.seg_cap;
    x.fin_cap = z.fin_cap;
    x.mid_cap = z.mid_cap;
    x.tile_cap = z.tile_cap;
    // 16-bucket passes use 16 counters per row for every window up to 4 bits;
    // the 256-bucket passes 256, and they need neither a second parity of
    // rows and histograms (each iteration counts its own tiles afresh) nor
    // per-bucket AND/OR
    const bool wide = z.tune.digit_bits > digit_bits();
    const int bins = wide ? 1 << wide_digit_bits() : 1 << digit_bits();

    x.ctr = (Counters *)take(sizeof(Counters));
    zero(x.ctr, 0, sizeof(Counters));
    x.status = (int32_t *)take(64);
    zero(x.status, 0, 64);
    x.new_roots = (int32_t *)take(4 * (size_t)(z.L > 16 ? z.L : 16));  // list heads (single/served calls)
    x.desc = (ListDesc *)take(sizeof(ListDesc) * (size_t)z.L);
    x.out_base = (int32_t *)take(4 * (size_t)(z.L + 1));
    x.root_task = (int32_t *)take(4 * (size_t)z.L);
    x.task_list = (int32_t *)take(4 * (size_t)z.Rcap);
    x.task_len = (int32_t *)take(4 * (size_t)z.Rcap);
    zero(x.task_len, 0, 4 * (size_t)z.Rcap);
    x.task_succ = (int32_t *)take(4 * (size_t)z.Rcap);
    zero(x.task_succ, 0xff, 4 * (size_t)z.Rcap);
    for (int b = 0; b < 2; ++b)
        x.wy[b] = (int64_t *)take(8 * (size_t)z.Rcap);
    x.Scap = (int32_t)((z.Rcap + 31) / 32 + 1 + z.L);  // grid walks, one gap, root walks
    for (int b = 0; b < 2; ++b)
        x.sw[b] = (int64_t *)take(8 * (size_t)x.Scap);
    x.chunk_task = (int32_t *)take(4 * (size_t)z.chunk_cap);
    zero(x.chunk_task, 0xff, 4 * (size_t)z.chunk_cap);
    x.chunk_j0 = (int32_t *)take(4 * (size_t)z.chunk_cap);
    x.chunk_data = (int32_t *)take(4 * (size_t)z.chunk_cap * z.CH);
    x.chunk_key = take((size_t)z.kb * z.chunk_cap * z.CH);
    x.blk_cap = (z.ncap + kEmitBlock - 1) / kEmitBlock + 1;
    x.chunk_pc = (int2 *)take(8 * (size_t)z.chunk_cap);
    x.blk_cnt = (int32_t *)take(4 * (size_t)x.blk_cap);
    zero(x.blk_cnt, 0, 4 * (size_t)x.blk_cap);
    x.blk_start = (int32_t *)take(4 * (size_t)(x.blk_cap + 1));
    x.blk_list = (int2 *)take(16 * (size_t)z.chunk_cap);
    // keyb[1], idxb[1] and F are adjacent: the ranking's pack array spans
    // them (n * (kb + 8) bytes >= n * 8, and >= n * 16 when kb == 8)
    for (int b = 0; b < 2; ++b) {
        x.keyb[b] = take((size_t)z.ncap * z.kb + 64);
        x.idxb[b] = (int32_t *)take((size_t)z.ncap * 4 + 64);
    }
    x.F = (int32_t *)take((size_t)z.ncap * 4 + 64);
    x.pack = z.pack ? x.keyb[1] : nullptr;
    // rows: the 16-bucket passes hold next-pass rows (tiles + 16 per bucket
    // list) besides the statistics rows; the 256-bucket passes only one row
    // per statistics tile of the pending segments (each longer than the cutoff)
    x.row_cap = wide ? z.ncap / pass_tile() + z.seg_cap + 64 : 2 * (z.ncap / pass_tile()) + 18 * z.seg_cap + 64;
    // scan chunks: only segments of more than one tile have them
    x.scan_cap = z.ncap / ((int64_t)pass_tile() * scan_rows()) + std::min<int64_t>(z.seg_cap, z.ncap / pass_tile()) + 2;
    for (int b = 0; b < 2; ++b) {
        x.act[b] = (Seg *)take(sizeof(Seg) * (size_t)z.seg_cap);
        x.act_hist[b] = (wide && b == 1) ? x.act_hist[0] : (uint32_t *)take(4 * (size_t)z.seg_cap * bins);
        x.act_tile_base[b] = (int32_t *)take(4 * (size_t)(z.seg_cap + 1));
        x.act_chunk_base[b] = (int32_t *)take(4 * (size_t)(z.seg_cap + 1));
        x.act_nrow_base[b] = (int32_t *)take(4 * (size_t)(z.seg_cap + 1));
        x.tcnt[b] = (wide && b == 1) ? x.tcnt[0] : (uint32_t *)take(4 * (size_t)x.row_cap * bins);
        if (!wide) {
            x.band[b] = (unsigned long long *)take(8 * (size_t)z.seg_cap * bins);
            zero(x.band[b], 0xff, 8 * (size_t)z.seg_cap * bins);
            x.bor[b] = (unsigned long long *)take(8 * (size_t)z.seg_cap * bins);
            zero(x.bor[b], 0, 8 * (size_t)z.seg_cap * bins);
        }
        x.pend[b] = (Seg *)take(sizeof(Seg) * (size_t)z.seg_cap);
        x.pend_tile_base[b] = (int32_t *)take(4 * (size_t)(z.seg_cap + 1));
        x.pand[b] = (unsigned long long *)take(8 * (size_t)z.seg_cap);
        zero(x.pand[b], 0xff, 8 * (size_t)z.seg_cap);
        x.por[b] = (unsigned long long *)take(8 * (size_t)z.seg_cap);
        zero(x.por[b], 0, 8 * (size_t)z.seg_cap);
    }
    x.ctot = (uint32_t *)take(4 * (size_t)x.scan_cap * bins);
    x.plan_cnt = (int4 *)take(sizeof(int4) * (size_t)z.seg_cap);
    x.plan_mid = (int32_t *)take(4 * (size_t)z.seg_cap);
    x.fin = (Fin *)take(sizeof(Fin) * (size_t)z.fin_cap);
    x.mid = (Fin *)take(sizeof(Fin) * (size_t)z.mid_cap);
    x.mid_defer = (int32_t *)take(4 * (size_t)z.mid_cap);
    x.rel_cursor = (int32_t *)take(4 * (size_t)relink_max_buckets());
    zero(x.rel_cursor, 0, 4 * (size_t)relink_max_buckets());
    if (c)
        *c = x;
    return off + 256;
}

size_t workspace_bytes(int64_t ncap, int32_t L, int kb, Tune t, int sms) {
    if (t.digit_bits > 0)
        return bind(compute_sizes(ncap, L, kb, t, sms), nullptr, nullptr, nullptr);
    size_t w = 0;  // digit width not known yet (it follows the call's K): room for every width
    for (int d = 1; d <= max_digit_bits(); ++d) {
        t.digit_bits = d;
        w = std::max(w, bind(compute_sizes(ncap, L, kb, t, sms), nullptr, nullptr, nullptr));
    }
    return w;
}

static int ceil_log2(int64_t x) {
    int r = 0;
    while ((1ll << r) < x)
        ++r;
    return r;
}

// Enqueue the whole sort on stream s.  Returns PBIT_ECUDA if a launch failed.
pbit_status enqueue_sort(const Ctx &c, const MemsetList &ms, int mode, const ListDesc *tmpl,
                         const int64_t *d_offsets, const int32_t *d_roots, int M, cudaStream_t s,
                         int sms, int64_t *launches, bool small_lists, int stop_after) {
    NvtxRange whole("pbit_sort");
    const int64_t n0 = g_enqueued_launches;  // kernel launches of this call = the difference
    prof_begin(s);
    if (ms.count < 0)
        return PBIT_ENOMEM;
    for (int i = 0; i < ms.count; ++i) {
        const Memset &m = ms.items[i];
        if (cudaMemsetAsync(m.p, m.v, m.bytes, s) != cudaSuccess)
            return PBIT_ECUDA;
    }
    prof_mark("memset", s);
    Ctx cc = c;
    cc.M = M;
    // One list that starts the 256-bucket passes: the emit counts the first
    // pass's digits per tile (the list's tiles are the emit's blocks), so the
    // first histogram kernel is left out.  The test mirrors plan_init's.
    cc.emit_hist = 0;
    if (mode == 2 && tmpl && cc.num_lists == 1 && cc.D > digit_bits() && !cc.force_pass) {
        const int64_t nl = tmpl->n;
        const bool mid = nl <= kMidCap && M <= kMidSpan;
        cc.emit_hist = (nl > cc.cutoff && !mid) ? 1 : 0;
    }
    launch_setup(cc, d_offsets, d_roots, mode, tmpl, s, sms);
    if (small_lists && mode != 0) {
        NvtxRange r("pbit_short_lists");
        launch_small(cc, s, sms);
        if (g_prof.on) {
            g_prof.kb = cc.key_bytes;
            g_prof.small = true;
        }
        if (launches)
            *launches = g_enqueued_launches - n0;
        return cudaGetLastError() == cudaSuccess ? PBIT_OK : PBIT_ECUDA;
    }
    if (g_prof.on)
        g_prof.small = false;
    const int rounds = ceil_log2(cc.Scap) + 1;  // pointer jumping over the ruler walks
    {
        NvtxRange r("pbit_rank");
        launch_pack(cc, s, sms);
        launch_walk(cc, s, sms);
        launch_wyllie(cc, s, sms, rounds);
        launch_validate_emit(cc, s, sms);
    }
    if (stop_after == 1)
        return cudaGetLastError() == cudaSuccess ? PBIT_OK : PBIT_ECUDA;
    const int iters = (M + cc.D - 1) / cc.D;
    {
        NvtxRange r("pbit_msd_passes");
        launch_plan_init(cc, s);
        for (int it = 0; it < iters; ++it) {
            launch_iteration(cc, it, s, sms);
            if (stop_after == 2)
                return cudaGetLastError() == cudaSuccess ? PBIT_OK : PBIT_ECUDA;
        }
    }
    {
        NvtxRange r("pbit_finish_relink");
        launch_check_done(cc, iters, s);
        launch_finish_relink(cc, s, sms);
    }
    if (g_prof.on) {
        g_prof.rcap = cc.Rcap;
        g_prof.scap = cc.Scap;
        g_prof.rounds = rounds;
        g_prof.kb = cc.key_bytes;
        g_prof.blocked_relink = relink_blocked(cc);
        g_prof.emit_hist = cc.emit_hist != 0;
        g_prof.pack = cc.pack != nullptr;
    }
    if (launches)
        *launches = g_enqueued_launches - n0;
    if (cudaGetLastError() != cudaSuccess)
        return PBIT_ECUDA;
    return PBIT_OK;
}

pbit_status map_status(int st) {
    if (st == 0)
        return PBIT_OK;
    if (st == kStOverflow)
        return PBIT_ENOMEM;
    if (st > 0 && st <= PBIT_EPENDING)
        return (pbit_status)st;
    return PBIT_ECUDA;
}

bool check_pool(const pbit_pool *p, int M, int K) {
    if (!p || (p->pool_size > 0 && (!p->next || !p->key)))  // an empty pool may have no storage
        return false;
    const int kb = p->key_type;
    if (kb != 1 && kb != 2 && kb != 4 && kb != 8)
        return false;
    if (K < 1 || K > 16 || M < 1 || M > 8 * kb || M % K != 0)
        return false;
    if (p->pool_size < 0 || p->pool_size >= (1ll << 31))
        return false;
    if (p->next_stride_bytes < 4 || p->next_stride_bytes % 4 != 0)
        return false;
    if (p->key_stride_bytes < kb || p->key_stride_bytes % kb != 0)
        return false;
    if ((p->flags & (PBIT_SIGNED | PBIT_FLOAT)) && M != 8 * kb)
        return false;
    if ((p->flags & PBIT_FLOAT) && kb < 4)
        return false;
    if ((p->flags & PBIT_DOUBLY) && ((p->pool_size > 0 && !p->prev) || p->prev_stride_bytes < 4 ||
                                     p->prev_stride_bytes % 4 != 0))
        return false;
    if (p->flags & ~(PBIT_SIGNED | PBIT_DESCENDING | PBIT_DOUBLY | PBIT_FLOAT))
        return false;
    if ((reinterpret_cast<uintptr_t>(p->next) & 3) || (reinterpret_cast<uintptr_t>(p->key) & (kb - 1)))
        return false;
    return true;
}

ListDesc pool_template(const pbit_pool *p) {
    ListDesc t{};
    t.next = p->next;
    t.key = (const unsigned char *)p->key;
    t.prev = p->prev;
    t.next_stride = p->next_stride_bytes;
    t.key_stride = p->key_stride_bytes;
    t.prev_stride = p->prev_stride_bytes;
    return t;
}

// Enqueue a sort of a pool with list ranges (d_offsets) or of one list.
pbit_status enqueue_pool(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                const int64_t *d_offsets, int single_root, int64_t single_n, int M, int K,
                                int32_t *d_new_roots, const pbit_tune *tune, void *ws, size_t ws_bytes,
                                cudaStream_t s, Ctx *out, int stop_after) {
    Tune t;
    if (!resolve_tune(tune, pool->pool_size, pool->key_type, K, &t))
        return PBIT_EINVAL;
    const int sms = device_sms();
    Sizes z = compute_sizes(pool->pool_size, num_lists, pool->key_type, t, sms);
    pbit_tune cached;
    if (!tune && tune_cache_lookup(pool->pool_size, num_lists, pool->key_type, &cached)) {
        // the autotuned choice for this size class, when it fits the workspace
        Tune tc;
        if (resolve_tune(&cached, pool->pool_size, pool->key_type, K, &tc)) {
            const Sizes zc = compute_sizes(pool->pool_size, num_lists, pool->key_type, tc, sms);
            if (bind(zc, nullptr, nullptr, nullptr) <= ws_bytes)
                z = zc;
        }
    }
    Ctx c;
    MemsetList ms;
    const size_t need = bind(z, (unsigned char *)ws, &c, &ms);
    if (!ws || ws_bytes < need || (reinterpret_cast<uintptr_t>(ws) & 255))
        return ws_bytes < need ? PBIT_ENOMEM : PBIT_EINVAL;
    c.flags = pool->flags;
    c.shared_pool = 1;
    c.desc_next_stride = pool->next_stride_bytes;
    c.force_pass = stop_after == 2;  // stage check: every list takes a global pass
    if (z.tune.pack == 0 && pool->key_type == 4 && pool->next_stride_bytes == 8 && pool->key_stride_bytes == 8 &&
        (const unsigned char *)pool->key == (const unsigned char *)pool->next + 4)
        c.pack = nullptr;  // {int32 next; uint32 key} nodes are packed already
    if (d_new_roots)
        c.new_roots = d_new_roots;
    ListDesc tmpl = pool_template(pool);
    pbit_status rc;
    if (d_offsets) {
        rc = enqueue_sort(c, ms, 0, &tmpl, d_offsets, d_roots, M, s, sms, &g_last_launches, false, stop_after);
    } else {
        // single list: its descriptor comes from the call arguments
        ListDesc d = tmpl;
        d.n = (int32_t)single_n;
        d.root = single_root;
        d.id_base = 0;
        d.out_base = 0;
        rc = enqueue_sort(c, ms, 2, &d, nullptr, nullptr, M, s, sms, &g_last_launches,
                          single_n <= kSmallList && stop_after == 0, stop_after);
    }
    *out = c;
    return rc;
}

// Read back the status (and the single root), synchronizing the stream.
static pbit_status finish_call(const Ctx &c, int32_t *host_root, cudaStream_t s) {
    static thread_local int32_t *hbuf = nullptr;
    if (!hbuf && cudaMallocHost((void **)&hbuf, 64) != cudaSuccess)
        return PBIT_ECUDA;
    if (cudaMemcpyAsync(hbuf, c.status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (host_root && cudaMemcpyAsync(hbuf + 1, c.new_roots, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (g_prof.on && cudaMemcpyAsync(&g_prof.ctr, c.ctr, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess)
        return PBIT_ECUDA;
    if (g_prof.on) {
        g_prof.have_ctr = true;
        g_prof.n = g_prof.ctr.n_virt;
    }
    const pbit_status st = map_status(hbuf[0]);
    if (st == PBIT_OK && host_root)
        *host_root = hbuf[1];
    return st;
}

static pbit_status sort_pool(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                             const int64_t *d_offsets, int single_root, int64_t single_n, int M, int K,
                             int32_t *d_new_roots, int32_t *host_root, const pbit_tune *tune, void *ws,
                             size_t ws_bytes, cudaStream_t s) {
    Ctx c;
    const pbit_status rc = enqueue_pool(pool, num_lists, d_roots, d_offsets, single_root, single_n, M, K,
                                        d_new_roots, tune, ws, ws_bytes, s, &c);
    if (rc != PBIT_OK)
        return rc;
    return finish_call(c, host_root, s);
}

// The host-buffer call's copy of next[] back to the host, one relink window
// at a time (RelinkWindowHook): stream cs waits for the window's kernel on
// the sort stream, then copies the window's bytes.
struct WindowCopy {
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
    const unsigned char *dnext = nullptr;
    unsigned char *hnext = nullptr;
    int64_t stride = 4, n = 0, copied = 0;  // copied: nodes whose window is on its way
    size_t bytes = 0;                       // next[] span in bytes
    bool ok = false;
};

static void copy_window(void *arg, int64_t lo, int64_t hi, cudaStream_t s) {
    WindowCopy &w = *static_cast<WindowCopy *>(arg);
    if (!w.ok || lo != w.copied || hi > w.n || hi <= lo) {
        w.ok = false;
        return;
    }
    const size_t b0 = (size_t)(lo * w.stride), b1 = hi == w.n ? w.bytes : (size_t)(hi * w.stride);
    if (cudaEventRecord(w.ev, s) != cudaSuccess || cudaStreamWaitEvent(w.cs, w.ev, 0) != cudaSuccess ||
        cudaMemcpyAsync(w.hnext + b0, w.dnext + b0, b1 - b0, cudaMemcpyDeviceToHost, w.cs) != cudaSuccess) {
        w.ok = false;
        return;
    }
    w.copied = hi;
}

PoolSpan pool_span(const pbit_pool *p) {
    PoolSpan r{};
    const int64_t n = p->pool_size;
    r.next_bytes = (size_t)(n > 0 ? (n - 1) * p->next_stride_bytes + 4 : 0);
    const unsigned char *nb = (const unsigned char *)p->next, *kb = (const unsigned char *)p->key;
    r.key_off = kb - nb;
    r.key_inside = r.key_off >= 0 && r.key_off + (n > 0 ? (n - 1) * p->key_stride_bytes + p->key_type : 0) <=
                                         (ptrdiff_t)r.next_bytes + p->next_stride_bytes;
    if (r.key_inside)
        r.next_bytes = (size_t)(n > 0 ? n * p->next_stride_bytes : 0);
    r.key_bytes = r.key_inside ? 0 : (size_t)(n > 0 ? (n - 1) * p->key_stride_bytes + p->key_type : 0);
    r.prev_bytes = (p->flags & PBIT_DOUBLY) ? (size_t)(n > 0 ? (n - 1) * p->prev_stride_bytes + 4 : 0) : 0;
    return r;
}

}  // namespace pbit

using namespace pbit;



extern "C" {

const char *pbit_status_string(int status) {
    switch (status) {
    case PBIT_OK: return "ok";
    case PBIT_EINVAL: return "invalid argument";
    case PBIT_ENOMEM: return "workspace too small or capacity exceeded";
    case PBIT_EBADLIST: return "malformed list (cycle, wrong length, index out of range or bad root)";
    case PBIT_ETIMEOUT: return "a bounded device wait gave up";
    case PBIT_ECUDA: return "CUDA runtime error";
    case PBIT_EAGAIN: return "request not admitted";
    case PBIT_EPENDING: return "request pending";
    default: return "unknown status";
    }
}

pbit_status pbit_workspace_size(int64_t pool_size, int32_t num_lists, int32_t key_type, const pbit_tune *tune,
                                size_t *bytes) {
    if (!bytes || pool_size < 0 || pool_size >= (1ll << 31) || num_lists < 1)
        return PBIT_EINVAL;
    if (key_type != 1 && key_type != 2 && key_type != 4 && key_type != 8)
        return PBIT_EINVAL;
    Tune t;
    if (!resolve_tune(tune, pool_size, key_type, 0, &t))
        return PBIT_EINVAL;
    const int sms = device_sms();
    size_t w = workspace_bytes(pool_size, num_lists, key_type, t, sms);
    pbit_tune cached;
    Tune tc;
    if (!tune && tune_cache_lookup(pool_size, num_lists, key_type, &cached) &&
        resolve_tune(&cached, pool_size, key_type, 0, &tc))  // room for either choice
        w = std::max(w, workspace_bytes(pool_size, num_lists, key_type, tc, sms));
    *bytes = w;
    return PBIT_OK;
}

pbit_status pbit_sort_list(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                           int32_t *new_root_host, const pbit_tune *tune, void *ws, size_t ws_bytes,
                           void *stream) {
    if (!check_pool(pool, M, K) || !new_root_host)
        return PBIT_EINVAL;
    if (n != pool->pool_size)
        return PBIT_EINVAL;
    if (n == 0) {
        if (root != -1)
            return PBIT_EBADLIST;
        *new_root_host = -1;
        return PBIT_OK;
    }
    if (root < 0 || root >= n)
        return PBIT_EBADLIST;
    return sort_pool(pool, 1, nullptr, nullptr, root, n, M, K, nullptr, new_root_host, tune, ws, ws_bytes,
                     (cudaStream_t)stream);
}

pbit_status pbit_debug_stage(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K, int32_t stage,
                             void *ws, size_t ws_bytes, int32_t *d_idx, void *d_key, void *stream) {
    if (!check_pool(pool, M, K) || n != pool->pool_size || n < 1 || (stage != 1 && stage != 2) || !d_idx || !d_key)
        return PBIT_EINVAL;
    if (stage == 2 && n < 2)
        return PBIT_EINVAL;  // nothing to split
    if (root < 0 || root >= n)
        return PBIT_EBADLIST;
    cudaStream_t s = (cudaStream_t)stream;
    Ctx c;
    const pbit_status rc = enqueue_pool(pool, 1, nullptr, nullptr, root, n, M, K, nullptr, nullptr, ws, ws_bytes, s, &c,
                                        stage);
    if (rc != PBIT_OK)
        return rc;
    const int b = stage == 1 ? 0 : 1;  // the ranking fills buffer 0, the first pass writes buffer 1
    if (cudaMemcpyAsync(d_idx, c.idxb[b], 4 * (size_t)n, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(d_key, c.keyb[b], (size_t)pool->key_type * (size_t)n, cudaMemcpyDeviceToDevice, s) !=
            cudaSuccess)
        return PBIT_ECUDA;
    return finish_call(c, nullptr, s);
}

pbit_status pbit_sort_lists_batched(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                    const int64_t *d_offsets, int32_t M, int32_t K, int32_t *d_new_roots,
                                    const pbit_tune *tune, void *ws, size_t ws_bytes, void *stream) {
    if (!check_pool(pool, M, K) || num_lists < 1 || !d_roots || !d_offsets || !d_new_roots)
        return PBIT_EINVAL;
    return sort_pool(pool, num_lists, d_roots, d_offsets, 0, 0, M, K, d_new_roots, nullptr, tune, ws, ws_bytes,
                     (cudaStream_t)stream);
}

int64_t pbit_last_launch_count(void) { return g_last_launches; }

void pbit_profile_enable(int32_t on) { g_prof.on = on != 0; }

int32_t pbit_profile_read(pbit_kernel_stat *out, int32_t max) {
    if (!g_prof.on || !g_prof.start || !out || max <= 0)
        return 0;
    int32_t cnt = 0;
    cudaEvent_t prev = g_prof.start;
    for (auto &m : g_prof.marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prev, m.second) != cudaSuccess)
            return -1;
        prev = m.second;
        int32_t i = 0;
        while (i < cnt && std::strncmp(out[i].name, m.first, sizeof(out[i].name)) != 0)
            ++i;
        if (i == cnt) {
            if (cnt == max)
                continue;
            std::memset(&out[i], 0, sizeof(out[i]));
            std::strncpy(out[i].name, m.first, sizeof(out[i].name) - 1);
            ++cnt;
        }
        out[i].launches += 1;
        out[i].ms += ms;
    }
    if (g_prof.have_ctr) {
        const Counters &k = g_prof.ctr;
        const double n = (double)g_prof.n, kb = (double)g_prof.kb;
        for (int32_t i = 0; i < cnt; ++i) {
            const char *nm = out[i].name;
            double b = 0;
            const double rec = kb == 8 ? 16.0 : 8.0;  // packed record
            if (!std::strcmp(nm, "small")) {  // next + key read, order written
                b = n * (8.0 + kb);
            } else if (!std::strcmp(nm, "pack")) {
                b = n * (4.0 + kb + rec);
            } else if (!std::strcmp(nm, "walk")) {
                b = n * ((g_prof.pack ? rec : 4.0 + kb) + 4.0 + kb);
            } else if (!std::strcmp(nm, "emit")) {
                b = n * 2.0 * (4.0 + kb);
            } else if (!std::strcmp(nm, "wyllie")) {
                // ruler walks: read len + succ, write (walk, prefix) per ruler;
                // pointer jumping over the walks; expand: read both, write one
                b = (double)g_prof.rcap * (16.0 + 24.0) + (double)g_prof.scap * 24.0 * (double)g_prof.rounds;
            } else if (!std::strcmp(nm, "seg_stats")) {
                for (int it = g_prof.emit_hist ? 1 : 0; it < kMaxIters; ++it)
                    b += (double)k.stat_elems[it] * kb;
            } else if (!std::strcmp(nm, "pass")) {
                for (int it = 0; it < kMaxIters; ++it)
                    b += (double)k.pass_elems[it] * 2.0 * (4.0 + kb) - (double)k.pass_final_elems[it] * kb;
            } else if (!std::strcmp(nm, "finish")) {
                b = (double)k.fin_sort_elems * (kb + 8.0) + (double)k.fin_copy_elems * 8.0;
            } else if (!std::strcmp(nm, "relink")) {
                b = n * (g_prof.blocked_relink ? 24.0 : 8.0);
            }
            out[i].bytes = b;
        }
    }
    return cnt;
}

pbit_status pbit_workspace_size_host(const pbit_pool *host_pool, const pbit_tune *tune, size_t *bytes) {
    if (!host_pool || !bytes)
        return PBIT_EINVAL;
    size_t w = 0;
    const pbit_status st = pbit_workspace_size(host_pool->pool_size, 1, host_pool->key_type, tune, &w);
    if (st != PBIT_OK)
        return st;
    const PoolSpan sp = pool_span(host_pool);
    *bytes = w + ((sp.next_bytes + 255) & ~(size_t)255) + ((sp.key_bytes + 255) & ~(size_t)255) +
             ((sp.prev_bytes + 255) & ~(size_t)255) + 256;
    return PBIT_OK;
}

pbit_status pbit_sort_list_host(const pbit_pool *host_pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                int32_t *new_root_host, const pbit_tune *tune, void *ws, size_t ws_bytes,
                                void *stream) {
    if (!check_pool(host_pool, M, K) || !new_root_host || n != host_pool->pool_size)
        return PBIT_EINVAL;
    if (n == 0) {
        if (root != -1)
            return PBIT_EBADLIST;
        *new_root_host = -1;
        return PBIT_OK;
    }
    if (root < 0 || root >= n)
        return PBIT_EBADLIST;
    size_t need = 0;
    if (pbit_workspace_size_host(host_pool, tune, &need) != PBIT_OK)
        return PBIT_EINVAL;
    if (!ws || ws_bytes < need)
        return PBIT_ENOMEM;
    const PoolSpan sp = pool_span(host_pool);
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *w = (unsigned char *)ws;
    unsigned char *dnext = w;
    w += (sp.next_bytes + 255) & ~(size_t)255;
    unsigned char *dkey = w;
    w += (sp.key_bytes + 255) & ~(size_t)255;
    unsigned char *dprev = w;
    w += (sp.prev_bytes + 255) & ~(size_t)255;
    pbit_pool dp = *host_pool;
    dp.next = (int32_t *)dnext;
    dp.key = sp.key_inside ? (const void *)(dnext + sp.key_off) : (const void *)dkey;
    if (host_pool->flags & PBIT_DOUBLY)
        dp.prev = (int32_t *)dprev;
    if (cudaMemcpyAsync(dnext, host_pool->next, sp.next_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (sp.key_bytes &&
        cudaMemcpyAsync(dkey, host_pool->key, sp.key_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (sp.prev_bytes &&
        cudaMemcpyAsync(dprev, host_pool->prev, sp.prev_bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return PBIT_ECUDA;
    Ctx c;
    const size_t rest = ws_bytes - (size_t)(w - (unsigned char *)ws);
    // next[] goes back window by window on a second stream, each window as
    // soon as the relink kernel that writes it has run (copied back
    // unconditionally: on an error the device copy was not written)
    WindowCopy wc{};
    wc.dnext = dnext;
    wc.hnext = (unsigned char *)host_pool->next;
    wc.stride = host_pool->next_stride_bytes;
    wc.n = n;
    wc.bytes = sp.next_bytes;
    wc.ok = cudaStreamCreateWithFlags(&wc.cs, cudaStreamNonBlocking) == cudaSuccess;
    wc.ok = wc.ok && cudaEventCreateWithFlags(&wc.ev, cudaEventDisableTiming) == cudaSuccess;
    if (wc.ok)
        g_relink_hook = RelinkWindowHook{copy_window, &wc};
    pbit_status rc = enqueue_pool(&dp, 1, nullptr, nullptr, root, n, M, K, nullptr, tune, w, rest, s, &c);
    g_relink_hook = RelinkWindowHook{};
    bool copied = false;
    if (wc.ok && wc.copied == n) {  // every window is on its way: s waits for the copies
        copied = cudaEventRecord(wc.ev, wc.cs) == cudaSuccess && cudaStreamWaitEvent(s, wc.ev, 0) == cudaSuccess;
    }
    if (!copied && wc.cs)  // (no windows, or a window's copy failed: everything again on s)
        cudaStreamSynchronize(wc.cs);
    if (wc.ev)
        cudaEventDestroy(wc.ev);
    if (wc.cs)
        cudaStreamDestroy(wc.cs);  // (released once its copies are done)
    if (rc != PBIT_OK)
        return rc;
    if (!copied && cudaMemcpyAsync(host_pool->next, dnext, sp.next_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PBIT_ECUDA;
    if (sp.prev_bytes &&
        cudaMemcpyAsync(host_pool->prev, dprev, sp.prev_bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PBIT_ECUDA;
    return finish_call(c, new_root_host, s);
}

}  // extern "C"
