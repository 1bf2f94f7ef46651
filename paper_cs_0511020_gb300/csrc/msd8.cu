// msd8.cu -- MSD digit passes with windows of up to 8 bits (256 buckets).
//
// The paper measures Pbit with K = 4, 8 and 16 bits per level (Sec. "The
// length of bit pattern"): a wider digit means fewer levels over the list.
// These kernels run one level per pass with a window of 5..8 bits (K = 16 is
// two passes of 8 bits per level).  They keep the structure of the 4-bit
// passes (msd.cu) -- the lists still to be split are segments of the order
// buffers, one pass splits all of them stably into buckets laid out in
// ascending digit order, small and mid-size buckets go to the finishes -- but
// count differently: with 256 buckets a table of next-pass counts per output
// tile no longer fits in shared memory, so every pass is preceded by a
// histogram kernel that counts each tile's digits (one extra read of the keys,
// w bytes per element, against the 2 (w + 4) bytes the pass moves).
//
// One iteration (= one level for every live segment):
//   hist8         pending segments: per-tile 256-bin counts of the window
//                 below their top bit, and the AND/OR of their keys
//   plan_pending  (shared with the 4-bit passes) pending -> active / small /
//                 mid / done / pending again at the top varying bit; tile and
//                 scan-chunk bases of the active segments
//   tile_scan8    per chunk of 256 tiles: exclusive prefixes of the counts
//   chunk_scan8   per segment: prefixes over its chunks, then the start of
//                 each of its 256 buckets
//   pass8         per tile: warp-ballot ranking with per-warp counters in
//                 shared memory, stable scatter through shared memory,
//                 coalesced write-out per digit run
//   plan_count8 / plan_scan / plan_write8
//                 output buckets -> small (warp finish) / mid-size (CTA
//                 finish) / pending for the next iteration
#include "pbit_internal.cuh"

namespace pbit {

constexpr int k8TPB = 256;
constexpr int k8Warps = k8TPB / 32;
constexpr int k8Items = 8;
constexpr int k8Tile = k8TPB * k8Items;
static_assert(k8Tile == kPassTile, "the plan kernels count tiles of kPassTile elements");
constexpr int k8Bits = 8;
constexpr int k8Bins = 1 << k8Bits;
static_assert(k8Bins == k8TPB, "one thread per bucket in the per-tile steps");

// ------------------------------------------------------------------ hist8
// For every tile of every pending segment: the counts of the 256 digits of
// the window [max(hi - D, 0), hi) (row g of tcnt: plain stores), and the
// AND/OR of the segment's keys.  Tiles are dealt round-robin to persistent
// CTAs; the keys of the next tile are copied into shared memory by the bulk
// copy engine while the current one is counted.
struct Hist8Smem {
    uint32_t h[2][k8Warps][k8Bins];  // per-warp digit counts, one set per stage
    unsigned long long s_and[2], s_or[2];
    int32_t seg[2], cnt[2], shk[2], lo[2], hi[2];
    int32_t cs, ctb_next;         // the issuing thread's segment cursor
    alignas(8) uint64_t bar[2];
};

template <typename KeyT>
struct Hist8Layout {
    static constexpr int kStage = ((k8Tile * (int)sizeof(KeyT) + 32 + 127) / 128) * 128;
    static constexpr int kHdr = ((int)sizeof(Hist8Smem) + 127) / 128 * 128;
    static constexpr int kTotal = kHdr + 2 * kStage;
};

template <typename KeyT>
__device__ __forceinline__ void hist8_issue(const Ctx &c, int cur, int P, int g, int st, Hist8Smem &S,
                                            unsigned char *stage) {
    while (g >= S.ctb_next) {  // follow the segments forward
        ++S.cs;
        S.ctb_next = S.cs + 1 < P ? c.pend_tile_base[cur][S.cs + 1] : INT32_MAX;
    }
    const Seg sg = c.pend[cur][S.cs];
    const int k = g - c.pend_tile_base[cur][S.cs];
    const int64_t start = (int64_t)sg.start + (int64_t)k * k8Tile;
    const int cnt = (int)min((int64_t)k8Tile, (int64_t)sg.start + sg.len - start);
    constexpr int W = (int)sizeof(KeyT);
    const int64_t k_lo = (start * W) & ~15ll, k_hi = ((start + cnt) * W + 15) & ~15ll;
    S.seg[st] = S.cs;
    S.cnt[st] = cnt;
    S.shk[st] = (int32_t)((start * W - k_lo) / W);
    S.lo[st] = max(sg.hi - c.D, 0);
    S.hi[st] = sg.hi;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&S.bar[st], (uint32_t)(k_hi - k_lo));
    bulk_g2s(stage, c.keyb[sg.buf & 1] + k_lo, (uint32_t)(k_hi - k_lo), &S.bar[st]);
}

template <typename KeyT>
__global__ void __launch_bounds__(k8TPB) k_hist8(Ctx c, int it) {
    griddep_wait();
    extern __shared__ __align__(128) unsigned char smem[];
    Hist8Smem &S = *reinterpret_cast<Hist8Smem *>(smem);
    unsigned char *stages = smem + Hist8Layout<KeyT>::kHdr;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int P = c.ctr->pend_count[cur];
    const int T = c.ctr->stat_tiles[cur];
    const int g0 = blockIdx.x, G = gridDim.x;
    if (g0 >= T)
        return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    using U = typename KeyWord<KeyT>::U;
    for (int w = 0; w < k8Warps; ++w) {
        S.h[0][w][tid] = 0;
        S.h[1][w][tid] = 0;
    }
    if (tid == 0) {
        S.s_and[0] = S.s_and[1] = ~0ull;
        S.s_or[0] = S.s_or[1] = 0ull;
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        S.cs = upper_index(c.pend_tile_base[cur], P, g0) - 1;  // the issue steps onto g0's segment
        S.ctb_next = c.pend_tile_base[cur][S.cs + 1];
        hist8_issue<KeyT>(c, cur, P, g0, 0, S, stages);
    }
    __syncthreads();
    long long my_elems = 0;
    uint32_t phases = 0;
    int st = 0;
    for (int g = g0; g < T; g += G) {
        const bool more = g + G < T;
        if (tid == 0 && more)
            hist8_issue<KeyT>(c, cur, P, g + G, st ^ 1, S, stages + (st ^ 1) * Hist8Layout<KeyT>::kStage);
        const bool landed = (tid != 0) || mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            if (tid == 0) {  // wait (bounded) for the copies still in flight before leaving
                mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
                if (more)
                    mbar_wait_bounded(&S.bar[st ^ 1], (phases >> (st ^ 1)) & 1u, 1ll << 26);
            }
            return;
        }
        phases ^= 1u << st;
        const int cnt = S.cnt[st], lo = S.lo[st];
        const unsigned dmask = (1u << (S.hi[st] - lo)) - 1u;
        const KeyT *sk = reinterpret_cast<const KeyT *>(stages + st * Hist8Layout<KeyT>::kStage) + S.shk[st];
        my_elems += cnt;
        U w_and = ~(U)0, w_or = 0;
#pragma unroll
        for (int u = 0; u < k8Items; ++u) {
            const int pos = u * k8TPB + tid;
            if (pos < cnt) {
                const U kv = (U)sk[pos];
                w_and &= kv;
                w_or |= kv;
                atomicAdd(&S.h[st][wid][(unsigned)(kv >> lo) & dmask], 1u);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w_and &= __shfl_xor_sync(kFull, w_and, o);
            w_or |= __shfl_xor_sync(kFull, w_or, o);
        }
        if (lane == 0) {  // keys are zero-extended to 64 bits
            atomicAnd(&S.s_and[st], (unsigned long long)w_and);
            atomicOr(&S.s_or[st], (unsigned long long)w_or);
        }
        __syncthreads();
        // (the next tile counts into the other set: the barrier at its copy
        // wait orders these reads and clears before that set's next use)
        uint32_t sum = 0;
#pragma unroll
        for (int w = 0; w < k8Warps; ++w) {
            sum += S.h[st][w][tid];
            S.h[st][w][tid] = 0;
        }
        if ((int64_t)g < c.row_cap)
            c.tcnt[cur][(int64_t)g * k8Bins + tid] = sum;
        else
            set_status(c.status, kStOverflow);
        if (tid == 0) {  // this tile's AND/OR into its segment's
            atomicAnd(&c.pand[cur][S.seg[st]], S.s_and[st]);
            atomicOr(&c.por[cur][S.seg[st]], S.s_or[st]);
            S.s_and[st] = ~0ull;
            S.s_or[st] = 0ull;
        }
        st ^= 1;
    }
    if (tid == 0 && my_elems)
        atomicAdd((unsigned long long *)&c.ctr->stat_elems[it], (unsigned long long)my_elems);
}

// ------------------------------------------------------------- tile_scan8
// Per chunk of kScanChunk tiles of an active segment: each tile's counts
// become the exclusive prefix within the chunk, and the chunk totals go to
// ctot.  Four groups of 256 threads (one thread per digit) take a quarter of
// the chunk's rows each: they sum their rows, add the sums of the groups
// before them, and write their rows' prefixes (the rows are read twice; the
// second time from L2).
constexpr int kScanGroups = 4;
constexpr int kScanRowsPerGroup = kScanChunk / kScanGroups;

__global__ void __launch_bounds__(k8TPB * kScanGroups) k_tile_scan8(Ctx c, int it) {
    griddep_wait();
    __shared__ uint32_t part[kScanGroups][k8Bins];
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int A = c.ctr->act_count[cur];
    const int nch = c.ctr->num_chunks[cur];
    const int d = threadIdx.x & (k8Bins - 1), q = threadIdx.x / k8Bins;
    for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int a = upper_index(c.act_chunk_base[cur], A, ch);
        const Seg sg = c.act[cur][a];
        const int lc = ch - c.act_chunk_base[cur][a];
        const int nt = c.act_tile_base[cur][a + 1] - c.act_tile_base[cur][a];
        const int t0 = lc * kScanChunk + q * kScanRowsPerGroup;
        const int t1 = min(nt, t0 + kScanRowsPerGroup);  // this group's rows [t0, t1)
        uint32_t *col = c.tcnt[cur] + ((int64_t)sg.row + t0) * k8Bins + d;
        const int nr = max(0, t1 - t0);
        uint32_t sum = 0;
        int t = 0;
        for (; t + 8 <= nr; t += 8) {  // eight loads in flight
            uint32_t x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = col[(int64_t)(t + u) * k8Bins];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                sum += x[u];
        }
        for (; t < nr; ++t)
            sum += col[(int64_t)t * k8Bins];
        part[q][d] = sum;
        __syncthreads();
        uint32_t run = 0, total = 0;
#pragma unroll
        for (int g = 0; g < kScanGroups; ++g) {
            const uint32_t v = part[g][d];
            run += g < q ? v : 0u;
            total += v;
        }
        t = 0;
        for (; t + 8 <= nr; t += 8) {
            uint32_t x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                x[u] = col[(int64_t)(t + u) * k8Bins];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                col[(int64_t)(t + u) * k8Bins] = run;
                run += x[u];
            }
        }
        for (; t < nr; ++t) {
            const uint32_t x = col[(int64_t)t * k8Bins];
            col[(int64_t)t * k8Bins] = run;
            run += x;
        }
        if (q == 0)
            c.ctot[(int64_t)ch * k8Bins + d] = total;
        __syncthreads();  // part[] is reused by the next chunk
    }
}

// ------------------------------------------------------------ chunk_scan8
// One CTA per active segment, one thread per digit: exclusive prefixes over
// the segment's chunks (in place), then the start of each bucket within the
// segment (exclusive prefix over the digits of its histogram) in act_hist.
__global__ void __launch_bounds__(k8TPB) k_chunk_scan8(Ctx c, int it) {
    griddep_wait();
    __shared__ int sh[40];
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int A = c.ctr->act_count[cur];
    const int d = threadIdx.x;
    for (int a = blockIdx.x; a < A; a += gridDim.x) {
        const int nt = c.act_tile_base[cur][a + 1] - c.act_tile_base[cur][a];
        uint32_t h = 0;
        if (nt == 1) {
            h = c.tcnt[cur][(int64_t)c.act[cur][a].row * k8Bins + d];
        } else {
            const int c0 = c.act_chunk_base[cur][a], c1 = c.act_chunk_base[cur][a + 1];
            uint32_t *col = c.ctot + (int64_t)c0 * k8Bins + d;
            int ch = 0;
            for (; ch + 8 <= c1 - c0; ch += 8) {  // eight loads in flight, then the running sum
                uint32_t x[8];
#pragma unroll
                for (int u = 0; u < 8; ++u)
                    x[u] = col[(int64_t)(ch + u) * k8Bins];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    col[(int64_t)(ch + u) * k8Bins] = h;
                    h += x[u];
                }
            }
            for (; ch < c1 - c0; ++ch) {
                const uint32_t x = col[(int64_t)ch * k8Bins];
                col[(int64_t)ch * k8Bins] = h;
                h += x;
            }
        }
        int tot;
        const int ex = block_excl_scan((int)h, &tot, sh);
        c.act_hist[cur][(int64_t)a * k8Bins + d] = (uint32_t)ex;
    }
}

// ------------------------------------------------------------------ pass8
// What a CTA needs to know about one tile (written by the thread that issues
// its copy, read by all after a barrier).
struct Tile8 {
    int32_t seg, k, cnt, shk, shi;
    int32_t start, len, lo, hi, buf, final, row, ch;
};

// The issuing thread's view of the segment its tiles belong to: tiles are
// taken in increasing order, so the segment is followed forward.
struct SegCursor {
    int s;
    int32_t tb, tb_next;  // tile bases of segment s and s + 1
    Seg sg;
    int32_t ch0;          // first scan chunk of segment s
};

struct Pass8Smem {
    int32_t nt[2];                   // the tiles in the two stages (>= num_tiles: none)
    uint32_t wcnt[k8Warps][k8Bins];  // per-warp digit counts -> each warp's first tile slot per digit
    int32_t gdelta[k8Bins];          // output position - tile slot, per digit
    int sh[40];                      // block scan scratch
    Tile8 tl[2];                     // the tiles in the two stages
    SegCursor q;                     // the issuing thread's segment cursor
    alignas(8) uint64_t bar[2];
};

template <typename KeyT>
struct Pass8Layout {
    static constexpr int kKeyBytes = k8Tile * (int)sizeof(KeyT) + 32;
    static constexpr int kIdxBytes = k8Tile * 4 + 32;
    static constexpr int kStage = ((kKeyBytes + kIdxBytes + 127) / 128) * 128;
    static constexpr int kHdr = ((int)sizeof(Pass8Smem) + 127) / 128 * 128;
    static constexpr int kIdx2 = kHdr + 2 * kStage;  // the tile's node ids in digit order
    static constexpr int kTotal = kIdx2 + k8Tile * 4;
    static constexpr int kMinBlocks = sizeof(KeyT) == 8 ? 3 : 4;
};

__device__ __forceinline__ void cursor_seek(const Ctx &c, int cur, int A, int g, SegCursor &q) {
    if (g < q.tb_next)
        return;
    do {
        ++q.s;
        q.tb = q.tb_next;
        q.tb_next = c.act_tile_base[cur][q.s + 1];
    } while (g >= q.tb_next && q.s + 1 < A);
    q.sg = c.act[cur][q.s];
    q.ch0 = c.act_chunk_base[cur][q.s];
}

// Issue the bulk copies of tile g into stage st and describe the tile (one thread).
template <typename KeyT>
__device__ __forceinline__ void pass8_issue(const Ctx &c, int cur, int A, int g, int st, SegCursor &q, Pass8Smem &S,
                                            unsigned char *stage) {
    cursor_seek(c, cur, A, g, q);
    const Seg &sg = q.sg;
    const int k = g - q.tb;
    const int64_t start = (int64_t)sg.start + (int64_t)k * k8Tile;
    const int cnt = (int)min((int64_t)k8Tile, (int64_t)sg.start + sg.len - start);
    constexpr int W = (int)sizeof(KeyT);
    const unsigned char *kb = c.keyb[sg.buf & 1];
    const unsigned char *ib = reinterpret_cast<const unsigned char *>(c.idxb[sg.buf & 1]);
    // 16-byte aligned copies covering [start, start + cnt); the order buffers
    // carry 64 bytes of slack behind their end for the rounding up
    const int64_t k_lo = (start * W) & ~15ll, k_hi = ((start + cnt) * W + 15) & ~15ll;
    const int64_t i_lo = (start * 4) & ~15ll, i_hi = ((start + cnt) * 4 + 15) & ~15ll;
    Tile8 &t = S.tl[st];
    t.seg = q.s;
    t.k = k;
    t.cnt = cnt;
    t.shk = (int32_t)((start * W - k_lo) / W);
    t.shi = (int32_t)((start * 4 - i_lo) / 4);
    t.start = sg.start;
    t.len = sg.len;
    t.lo = sg.lo;
    t.hi = sg.hi;
    t.buf = sg.buf;
    t.final = sg.final;
    t.row = sg.row;
    t.ch = q.ch0 + k / kScanChunk;
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&S.bar[st], (uint32_t)((k_hi - k_lo) + (i_hi - i_lo)));
    bulk_g2s(stage, kb + k_lo, (uint32_t)(k_hi - k_lo), &S.bar[st]);
    bulk_g2s(stage + Pass8Layout<KeyT>::kKeyBytes, ib + i_lo, (uint32_t)(i_hi - i_lo), &S.bar[st]);
}

// Output position of the tile's first element of digit d: bucket start +
// the digit's count in the segment's earlier tiles.
__device__ __forceinline__ int32_t tile_base8(const Ctx &c, int cur, const Tile8 &t, int d) {
    int32_t gb = t.start + (int32_t)c.act_hist[cur][(int64_t)t.seg * k8Bins + d];
    if (t.k > 0)
        gb += (int32_t)(c.ctot[(int64_t)t.ch * k8Bins + d] + c.tcnt[cur][((int64_t)t.row + t.k) * k8Bins + d]);
    return gb;
}

// One tile of the pass: ranking, tile offsets, local scatter and write-out
// (kWhole: the tile holds k8Tile elements, so no element needs an end check).
// Returns the output bases of the next tile's digits (loaded meanwhile).
template <typename KeyT, bool kWhole>
__device__ __forceinline__ int32_t pass8_tile(const Ctx &c, int cur, Pass8Smem &S, unsigned char *stage, int st,
                                              int T, int32_t gb, int tid, int lane, int wid, unsigned lt) {
    const Tile8 &t = S.tl[st];  // (fields read from shared memory where used)
    const int lo = t.lo, cnt = kWhole ? k8Tile : t.cnt;
    const unsigned dmask = (1u << (t.hi - t.lo)) - 1u;
    const KeyT *sk = reinterpret_cast<const KeyT *>(stage) + t.shk;
    const int32_t *si = reinterpret_cast<const int32_t *>(stage + Pass8Layout<KeyT>::kKeyBytes) + t.shi;
    bool bad = false;  // an inconsistent count or position (cannot happen): reported, not written

    // ---- ranking within the warp
    KeyT key[k8Items];
    uint32_t rnk[k8Items];
    uint32_t *wc = S.wcnt[wid];
#pragma unroll
    for (int i = 0; i < k8Items; ++i) {
        const int pos = wid * (32 * k8Items) + i * 32 + lane;
        const bool valid = kWhole || pos < cnt;
        key[i] = valid ? sk[pos] : (KeyT)0;
        const unsigned dig = digit_of<KeyT>(key[i], lo, dmask);
        // peers: the valid lanes that differ from this one in no digit bit
        // (bits above a narrower window are 0 everywhere)
        unsigned diff = 0;
#pragma unroll
        for (int b = 0; b < k8Bits; ++b) {
            const int m = (int)(dig << (31 - b)) >> 31;  // -1 if bit b is set, else 0
            diff |= __ballot_sync(kFull, m != 0) ^ (unsigned)m;
        }
        const unsigned peers = (kWhole ? kFull : __ballot_sync(kFull, valid)) & ~diff;
        // every lane reads its digit's count; the lowest peer writes it back
        // advanced (the lowest peers of one group hold distinct digits)
        const uint32_t before = wc[dig];
        const unsigned below = peers & lt;
        if (valid && below == 0)
            wc[dig] = before + (uint32_t)__popc(peers);
        __syncwarp();
        rnk[i] = before + (uint32_t)__popc(below);
    }
    __syncthreads();
    // the next tile's output bases: loads in flight during the rest of this tile
    const bool more = S.nt[st ^ 1] < T;
    const int32_t gb_next = more ? tile_base8(c, cur, S.tl[st ^ 1], tid) : 0;
    // ---- tile offsets per digit (thread tid = digit), each warp's first slot
    {
        uint32_t cw[k8Warps];
        uint32_t tot = 0;
#pragma unroll
        for (int w = 0; w < k8Warps; ++w) {
            cw[w] = S.wcnt[w][tid];
            tot += cw[w];
        }
        int ttot;
        uint32_t run = (uint32_t)block_excl_scan_1bar((int)tot, &ttot, S.sh);
        S.gdelta[tid] = gb - (int32_t)run;
#pragma unroll
        for (int w = 0; w < k8Warps; ++w) {
            S.wcnt[w][tid] = run;
            run += cw[w];
        }
    }
    __syncthreads();
    // ---- local scatter: keys into the stage buffer (all of them are in
    // registers), node ids from the stage into a buffer of their own
    KeyT *ok = reinterpret_cast<KeyT *>(stage);
    int32_t *oi = reinterpret_cast<int32_t *>(reinterpret_cast<unsigned char *>(&S) + Pass8Layout<KeyT>::kIdx2);
#pragma unroll
    for (int i = 0; i < k8Items; ++i) {
        const int pos = wid * (32 * k8Items) + i * 32 + lane;
        const uint32_t lp = wc[digit_of<KeyT>(key[i], lo, dmask)] + rnk[i];
        const bool in = lp < (uint32_t)cnt;
        bad |= (kWhole || pos < cnt) && !in;
        if ((kWhole || pos < cnt) && in) {
            ok[lp] = key[i];
            oi[lp] = si[pos];
        }
    }
    __syncthreads();
#pragma unroll
    for (int w = 0; w < k8Warps; ++w)  // counters of the next tile
        S.wcnt[w][tid] = 0;
    // ---- coalesced write-out: slot j goes to gdelta[its digit] + j
    const int32_t start = t.start, len = t.len;
    if (lo == 0 || t.final) {
#pragma unroll
        for (int u = 0; u < k8Items; ++u) {
            const int j = u * k8TPB + tid;
            if (kWhole || j < cnt) {
                const int dst = S.gdelta[digit_of<KeyT>(ok[j], lo, dmask)] + j;
                const bool in = (unsigned)(dst - start) < (unsigned)len;
                bad |= !in;
                if (in)
                    c.F[dst] = oi[j];
            }
        }
    } else {
        KeyT *okey = reinterpret_cast<KeyT *>(c.keyb[(t.buf & 1) ^ 1]);
        int32_t *oidx = c.idxb[(t.buf & 1) ^ 1];
#pragma unroll
        for (int u = 0; u < k8Items; ++u) {
            const int j = u * k8TPB + tid;
            if (kWhole || j < cnt) {
                const KeyT kk = ok[j];
                const int dst = S.gdelta[digit_of<KeyT>(kk, lo, dmask)] + j;
                const bool in = (unsigned)(dst - start) < (unsigned)len;
                bad |= !in;
                if (in) {
                    okey[dst] = kk;
                    oidx[dst] = oi[j];
                }
            }
        }
    }
    if (bad)
        set_status(c.status, kStOverflow);
    return gb_next;
}

// Persistent CTAs claim tiles from a counter; the bulk copy of the next tile
// is in flight, and the output bases of its digits are being loaded, while
// the current one is ranked and written.  Ranking: for each 32-element group
// a warp finds the lanes holding the same digit (peers); the lowest of them
// adds the group's count to the warp's shared counter of that digit and
// passes the old value to its peers, so
// every element learns how many elements with its digit came before it in
// the warp's part of the tile (memory order = warp, group, lane: the order
// is stable).  Peers come from eight ballots, one per digit bit: a lane keeps
// the lanes that differ from it in no bit.  (The match instruction finds the
// same lanes in one instruction, but measured on this GPU it saturated the
// ADU pipe at 81% and the pass ran slower than with ballots, also when only
// every second or every fourth group used it.)
template <typename KeyT>
__global__ void __launch_bounds__(k8TPB, Pass8Layout<KeyT>::kMinBlocks) k_pass8(Ctx c, int it) {
    griddep_wait();
    extern __shared__ __align__(128) unsigned char smem[];
    Pass8Smem &S = *reinterpret_cast<Pass8Smem *>(smem);
    unsigned char *stages = smem + Pass8Layout<KeyT>::kHdr;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int A = c.ctr->act_count[cur];
    const int T = c.ctr->num_tiles[cur];
    if (A == 0 || T == 0)
        return;
    // Tiles are claimed from a counter one step ahead (the claim's latency
    // hides behind a tile), so the tiles in flight at one time are
    // neighbours: the runs they write into each bucket are neighbours too and
    // fill whole lines while they are still in L2.  A CTA's claims increase,
    // so its thread 0 follows the segments forward.
    SegCursor &q = S.q;  // used by thread 0 only
    int claim = 0;       // thread 0: the tile claimed for the next issue
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        const int g0 = atomicAdd(&c.ctr->tile_ctr[it], 1);
        S.nt[0] = g0;
        if (g0 < T) {
            q.s = upper_index(c.act_tile_base[cur], A, g0) - 1;  // the seek below steps onto g0's segment
            q.tb_next = c.act_tile_base[cur][q.s + 1];
            q.tb = q.tb_next;
            pass8_issue<KeyT>(c, cur, A, g0, 0, q, S, stages);
            claim = atomicAdd(&c.ctr->tile_ctr[it], 1);
        }
    }
#pragma unroll
    for (int w = 0; w < k8Warps; ++w)
        S.wcnt[w][tid] = 0;
    __syncthreads();
    int g = S.nt[0];
    if (g >= T)
        return;
    int32_t gb = tile_base8(c, cur, S.tl[0], tid);
    uint32_t phases = 0;  // bit b: parity of stage b's barrier
    int st = 0;
    while (g < T) {
        unsigned char *stage = stages + st * Pass8Layout<KeyT>::kStage;
        // one thread waits for the copy (acquire), the barrier publishes it;
        // every thread is past the previous tile, so the other stage is free
        const bool landed = (tid != 0) || mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            if (tid == 0)  // wait (bounded) for the copy still in flight before leaving
                mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
            return;
        }
        phases ^= 1u << st;
        if (tid == 0) {  // the next tile into the other stage (the others read its
                         // description after the tile's first barrier), claim the one after
            S.nt[st ^ 1] = claim;
            if (claim < T) {
                pass8_issue<KeyT>(c, cur, A, claim, st ^ 1, q, S, stages + (st ^ 1) * Pass8Layout<KeyT>::kStage);
                claim = atomicAdd(&c.ctr->tile_ctr[it], 1);
            }
        }
        // (almost every tile is full: its copy of the code has no end checks)
        const int32_t gb_next = S.tl[st].cnt == k8Tile
                                    ? pass8_tile<KeyT, true>(c, cur, S, stage, st, T, gb, tid, lane, wid, lt)
                                    : pass8_tile<KeyT, false>(c, cur, S, stage, st, T, gb, tid, lane, wid, lt);
        gb = gb_next;
        g = S.nt[st ^ 1];  // (written before the tile's barriers)
        st ^= 1;
    }
}

// ------------------------------------------------------------------ plan8
// Where an output bucket of an 8-bit pass goes (its varying bits are not
// known: they are counted by the next histogram if it stays in the passes):
// 0 none, 1 one node (copied), 2 small (warp finish on its low `lo` bits),
// 4 pending for the next iteration, 6 mid-size (CTA finish; a bucket with at
// most kMidSpan bits left always qualifies).
__device__ __forceinline__ int classify8(const Ctx &c, uint32_t cnt, int lo) {
    if (cnt == 0)
        return 0;
    if (cnt == 1)
        return 1;
    if ((int)cnt <= c.cutoff)
        return 2;
    if ((int)cnt <= kMidCap && lo <= kMidSpan)
        return 6;
    return 4;
}

// Lane l of the warp of a segment looks at digits 8l .. 8l + 7.
__device__ __forceinline__ uint32_t bucket_len8(const Ctx &c, int cur, int64_t a, int d, int len) {
    const uint32_t *bs = c.act_hist[cur] + a * k8Bins;
    const uint32_t s0 = bs[d];
    const uint32_t s1 = d + 1 < k8Bins ? bs[d + 1] : (uint32_t)len;
    return s1 - s0;
}

// One warp per active segment: how many pending, small and mid-size buckets
// (and stats tiles) its 256 buckets produce.
__global__ void k_plan_count8(Ctx c, int it) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int A = c.ctr->act_count[cur];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < A; a += nw) {
        const Seg sg = c.act[cur][a];
        int np = 0, nf = 0, nt = 0, nm = 0;
        if (sg.lo > 0 && !sg.final) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint32_t cnt = bucket_len8(c, cur, a, lane * 8 + j, sg.len);
                const int kd = classify8(c, cnt, sg.lo);
                np += kd == 4;
                nf += kd == 1 || kd == 2;
                nt += kd == 4 ? tiles_of(cnt, kPassTile) : 0;
                nm += kd == 6;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            np += __shfl_xor_sync(kFull, np, o);
            nf += __shfl_xor_sync(kFull, nf, o);
            nt += __shfl_xor_sync(kFull, nt, o);
            nm += __shfl_xor_sync(kFull, nm, o);
        }
        if (lane == 0) {
            c.plan_cnt[a] = make_int4(0, np, nf, nt);
            c.plan_mid[a] = nm;
        }
    }
}

__device__ __forceinline__ int warp_excl_sum(int v, int lane) {
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o)
            x += y;
    }
    return x - v;
}

// One warp per active segment: write its buckets' records at the offsets
// plan_scan computed, in ascending digit order.
__global__ void k_plan_write8(Ctx c, int it) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int A = c.ctr->act_count[cur];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < A; a += nw) {
        const Seg sg = c.act[cur][a];
        if (sg.lo == 0 || sg.final)
            continue;  // the pass wrote it to its final place
        uint32_t cnt[8];
        int np = 0, nf = 0, nt = 0, nm = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            cnt[j] = bucket_len8(c, cur, a, lane * 8 + j, sg.len);
            const int kd = classify8(c, cnt[j], sg.lo);
            np += kd == 4;
            nf += kd == 1 || kd == 2;
            nt += kd == 4 ? tiles_of(cnt[j], kPassTile) : 0;
            nm += kd == 6;
        }
        const int4 o = c.plan_cnt[a];
        int64_t p = o.y + warp_excl_sum(np, lane);
        int64_t f = o.z + warp_excl_sum(nf, lane);
        int64_t tb = o.w + warp_excl_sum(nt, lane);
        int64_t m = c.plan_mid[a] + warp_excl_sum(nm, lane);
        const int nbuf = (sg.buf & 1) ^ 1;
        int32_t bstart = sg.start + (int32_t)c.act_hist[cur][a * k8Bins + lane * 8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int kd = classify8(c, cnt[j], sg.lo);
            if (kd == 6) {
                if (m < c.mid_cap)
                    c.mid[m] = Fin{bstart, (int32_t)cnt[j], sg.lo, (1 << 8) | nbuf};
                ++m;
            } else if (kd == 1 || kd == 2) {
                if (f < c.fin_cap)
                    c.fin[f] = Fin{bstart, (int32_t)cnt[j], kd == 2 ? sg.lo : 0, ((kd == 2 ? 1 : 0) << 8) | nbuf};
                ++f;
            } else if (kd == 4) {
                if (p < c.seg_cap) {
                    c.pend[nxt][p] = Seg{bstart, (int32_t)cnt[j], 0, sg.lo, nbuf, 0, 0};
                    c.pend_tile_base[nxt][p] = (int32_t)tb;
                }
                tb += tiles_of(cnt[j], kPassTile);
                ++p;
            }
            bstart += (int32_t)cnt[j];
        }
    }
}

// ------------------------------------------------------------- launchers
void launch_plan_pending(const Ctx &c, int it, cudaStream_t s);  // msd.cu
void launch_plan_scan(const Ctx &c, int it, cudaStream_t s);     // msd.cu

template <typename KeyT>
static void launch_iter8_t(const Ctx &c, int it, cudaStream_t s, int sms) {
    const int smem = Pass8Layout<KeyT>::kTotal;
    cudaFuncSetAttribute(k_pass8<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int per_sm = Pass8Layout<KeyT>::kMinBlocks;
    const unsigned wblocks = (unsigned)max(1, min(sms * 8, (int)((c.seg_cap + 7) / 8)));  // 8 warps per CTA
    const unsigned sblocks = (unsigned)max(1, min(sms * 8, (int)c.seg_cap));
    if (it > 0 || !c.emit_hist) {  // (emit_hist: the emit counted the first pass's tiles)
        const int hsmem = Hist8Layout<KeyT>::kTotal;
        cudaFuncSetAttribute(k_hist8<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, hsmem);
        const int per_sm = max(1, min(8, (200 * 1024) / (hsmem + 1024)));
        launch_pdl(k_hist8<KeyT>, dim3(sms * per_sm), dim3(k8TPB), hsmem, s, c, it);
    }
    prof_mark("seg_stats", s);
    launch_plan_pending(c, it, s);
    launch_pdl(k_tile_scan8, dim3(sms * 2), dim3(k8TPB * kScanGroups), 0, s, c, it);
    launch_pdl(k_chunk_scan8, dim3(sblocks), dim3(k8TPB), 0, s, c, it);
    prof_mark("scan", s);
    launch_pdl(k_pass8<KeyT>, dim3(sms * per_sm), dim3(k8TPB), smem, s, c, it);
    prof_mark("pass", s);
    launch_pdl(k_plan_count8, dim3(wblocks), dim3(256), 0, s, c, it);
    launch_plan_scan(c, it, s);
    launch_pdl(k_plan_write8, dim3(wblocks), dim3(256), 0, s, c, it);
    prof_mark("plan", s);
}

void launch_iteration8(const Ctx &c, int it, cudaStream_t s, int sms) {
    switch (c.key_bytes) {
    case 1: launch_iter8_t<uint8_t>(c, it, s, sms); break;
    case 2: launch_iter8_t<uint16_t>(c, it, s, sms); break;
    case 4: launch_iter8_t<uint32_t>(c, it, s, sms); break;
    default: launch_iter8_t<unsigned long long>(c, it, s, sms); break;
    }
}

int wide_digit_bits() { return k8Bits; }

}  // namespace pbit
