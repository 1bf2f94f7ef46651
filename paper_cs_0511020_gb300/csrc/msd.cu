// msd.cu -- stage (b): Pbit's MSD digit passes over the ranked list.
//
// The paper splits the list on the top K bits, then recurses into each of the
// Omega = 2^K buckets with the next K bits (Sec. "Implementation in C++"),
// visiting buckets from Omega-1 down to 0 so that the concatenation comes out
// ascending (Sec. "Differences between sorting in descending and ascending
// order").  Here every recursion level is one data-parallel pass over all
// live buckets ("segments") at once: a stable counting split of each segment
// into 2^D sub-segments laid out in ascending digit order, which is the same
// order the ascending concatenation produces.
//
//   seg_stats     per pending segment: 16-bin histograms of every D-bit
//                 window and the AND/OR of its keys (which bits still vary)
//   plan_pending  pending segment -> active (window holding its top varying
//                 bit), small (finished in shared memory) or done
//   pass          per active segment tile: warp-ballot ranking, decoupled
//                 look-back over the segment's tiles, stable scatter through
//                 shared memory; fused: next-window histogram and AND/OR of
//                 every output bucket
//   plan          output buckets -> next active / pending / small / done
#include "pbit_internal.cuh"

namespace pbit {

constexpr int kTPB = 256;       // threads per pass / stats CTA
constexpr int kItems = 16;      // items per thread in a pass tile
constexpr int kTile = kTPB * kItems;  // 4096 elements per pass tile
constexpr int kStatTile = 8192; // elements per seg_stats tile
constexpr int kD = 4;           // GPU digit width (16 buckets, as the paper's K = 4)
constexpr int kBins = 1 << kD;
constexpr int kMaxWin = 16;     // 64-bit keys / 4-bit windows
static_assert(kTPB == kBins * kBins, "the next-window histogram flush maps one thread per counter");

__host__ __device__ constexpr int tiles_of(int64_t len, int64_t tile) { return (int)((len + tile - 1) / tile); }

// ---------------------------------------------------------------- scans
// Block-wide exclusive scan of one int per thread (blockDim.x <= 1024).
__device__ int block_excl_scan(int v, int *total, int *sh /* >= 33 ints */) {
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

__device__ __forceinline__ int top_bit(unsigned long long v) { return 63 - __clzll((long long)v); }
__device__ __forceinline__ unsigned long long low_mask(int bits) {
    return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
}

// ------------------------------------------------------------- plan_init
// Lists become the first segments: empty lists vanish, lists up to the
// cutoff go straight to the shared-memory finish, the rest are pending.
__global__ void __launch_bounds__(1024) k_plan_init(Ctx c) {
    __shared__ int sh[40];
    __shared__ int s_fin_base, s_pend_base, s_tile_base;
    if (*(volatile int32_t *)c.status)
        return;
    if (threadIdx.x == 0) {
        s_fin_base = 0;
        s_pend_base = 0;
        s_tile_base = 0;
    }
    __syncthreads();
    const int L = c.num_lists;
    for (int r0 = 0; r0 < L; r0 += blockDim.x) {
        int i = r0 + threadIdx.x;
        int n = 0, start = 0;
        if (i < L) {
            n = c.desc[i].n;
            start = c.desc[i].out_base;
        }
        int is_fin = (i < L && n >= 1 && n <= c.cutoff) ? 1 : 0;
        int is_pend = (i < L && n > c.cutoff) ? 1 : 0;
        int tiles = is_pend ? tiles_of(n, kStatTile) : 0;
        int tf, tp, tt;
        int pf = block_excl_scan(is_fin, &tf, sh);
        int pp = block_excl_scan(is_pend, &tp, sh);
        int pt = block_excl_scan(tiles, &tt, sh);
        if (is_fin) {
            int k = s_fin_base + pf;
            if (k < c.fin_cap)
                c.fin[k] = Fin{start, n, c.M, ((n == 1 ? 0 : 1) << 8) | 0};
            else
                set_status(c.status, kStOverflow);
        }
        if (is_pend) {
            int k = s_pend_base + pp;
            if (k < c.seg_cap) {
                c.pend[0][k] = Seg{start, n, 0, c.M};
                c.pend_tile_base[0][k] = s_tile_base + pt;
            } else {
                set_status(c.status, kStOverflow);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_fin_base += tf;
            s_pend_base += tp;
            s_tile_base += tt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.ctr->fin_count = s_fin_base;
        c.ctr->pend_count[0] = min((int64_t)s_pend_base, c.seg_cap);
        if (s_pend_base < c.seg_cap)
            c.pend_tile_base[0][s_pend_base] = s_tile_base;
        c.ctr->stat_tiles[0] = s_tile_base;
        c.ctr->act_count[0] = 0;
    }
}

// ------------------------------------------------------------- seg_stats
template <typename KeyT>
__global__ void __launch_bounds__(kTPB) k_seg_stats(Ctx c, int it) {
    __shared__ uint32_t s_cnt[kMaxWin * kBins];
    __shared__ unsigned long long s_and, s_or;
    __shared__ int s_tile;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int P = c.ctr->pend_count[cur];
    const int ntiles = c.ctr->stat_tiles[cur];
    const KeyT *keys = reinterpret_cast<const KeyT *>(c.keyb[cur]);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    for (int i = threadIdx.x; i < kMaxWin * kBins; i += kTPB)
        s_cnt[i] = 0;
    if (threadIdx.x == 0) {
        s_and = ~0ull;
        s_or = 0ull;
    }
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0)
            s_tile = atomicAdd(&c.ctr->stat_ctr[it], 1);
        __syncthreads();
        const int g = s_tile;
        if (g >= ntiles)
            break;
        const int s = upper_index(c.pend_tile_base[cur], P, g);
        const Seg sg = c.pend[cur][s];
        const int k = g - c.pend_tile_base[cur][s];
        const int64_t b0 = (int64_t)sg.start + (int64_t)k * kStatTile;
        const int cnt = (int)min((int64_t)kStatTile, (int64_t)sg.start + sg.len - b0);
        const int hi = sg.hi;
        const int nwin = (hi + kD - 1) / kD;
        uint32_t wc[kMaxWin];
#pragma unroll
        for (int w = 0; w < kMaxWin; ++w)
            wc[w] = 0;
        unsigned long long a_and = ~0ull, a_or = 0ull;
        for (int base = wid * 32; base < cnt; base += kTPB) {
            const int pos = base + lane;
            const bool valid = pos < cnt;
            unsigned long long key = valid ? (unsigned long long)keys[b0 + pos] : 0ull;
            if (valid) {
                a_and &= key;
                a_or |= key;
            }
            const unsigned vm = __ballot_sync(kFull, valid);
#pragma unroll
            for (int w = 0; w < kMaxWin; ++w) {
                if (w < nwin) {
                    const int whi = hi - kD * w;
                    const int wlo = max(whi - kD, 0);
                    const unsigned dig = (unsigned)((key >> wlo) & ((1ull << (whi - wlo)) - 1));
                    unsigned m = vm;
#pragma unroll
                    for (int b = 0; b < kD; ++b) {
                        const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                        m &= ((lane >> b) & 1) ? bb : ~bb;
                    }
                    wc[w] += __popc(m);
                }
            }
        }
        (void)lt;
        // warp AND/OR
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a_and &= __shfl_xor_sync(kFull, a_and, o);
            a_or |= __shfl_xor_sync(kFull, a_or, o);
        }
        if (lane < kBins) {
#pragma unroll
            for (int w = 0; w < kMaxWin; ++w)
                if (w < nwin && wc[w])
                    atomicAdd(&s_cnt[w * kBins + lane], wc[w]);
        }
        if (lane == 0) {
            atomicAnd(&s_and, a_and);
            atomicOr(&s_or, a_or);
        }
        __syncthreads();
        uint32_t *gh = c.phist[cur] + (int64_t)s * (kMaxWin * kBins);
        for (int i = threadIdx.x; i < nwin * kBins; i += kTPB) {
            uint32_t v = s_cnt[i];
            if (v) {
                atomicAdd(&gh[i], v);
                s_cnt[i] = 0;
            }
        }
        if (threadIdx.x == 0) {
            atomicAnd(&c.pand[cur][s], s_and);
            atomicOr(&c.por[cur][s], s_or);
            s_and = ~0ull;
            s_or = 0ull;
        }
    }
}

// ---------------------------------------------------------- plan_pending
__global__ void __launch_bounds__(1024) k_plan_pending(Ctx c, int it) {
    __shared__ int sh[40];
    __shared__ int s_act_base, s_fin_base, s_tile_base;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int P = c.ctr->pend_count[cur];
    if (threadIdx.x == 0) {
        s_act_base = c.ctr->act_count[cur];
        s_fin_base = 0;
        s_tile_base = 0;
    }
    __syncthreads();
    int fin_total = 0;
    for (int r0 = 0; r0 < P; r0 += blockDim.x) {
        const int s = r0 + threadIdx.x;
        int kind = 0;  // 1 fin copy, 2 fin sort, 3 active
        Seg sg{0, 0, 0, 0};
        int t = 0, w = 0;
        if (s < P) {
            sg = c.pend[cur][s];
            unsigned long long v = (c.por[cur][s] ^ c.pand[cur][s]) & low_mask(sg.hi);
            if (sg.len <= 1 || v == 0) {
                kind = 1;
            } else {
                t = top_bit(v);
                if (sg.len <= c.cutoff)
                    kind = 2;
                else {
                    kind = 3;
                    w = (sg.hi - 1 - t) / kD;
                }
            }
        }
        int tf, ta;
        int pf = block_excl_scan(kind == 1 || kind == 2, &tf, sh);
        int pa = block_excl_scan(kind == 3, &ta, sh);
        if (kind == 1 || kind == 2) {
            int64_t k = (int64_t)c.ctr->fin_count + fin_total + pf;
            if (k < c.fin_cap)
                c.fin[k] = Fin{sg.start, sg.len, kind == 2 ? t + 1 : 0, ((kind == 2 ? 1 : 0) << 8) | cur};
            else
                set_status(c.status, kStOverflow);
        }
        if (kind == 3) {
            int64_t a = (int64_t)s_act_base + pa;
            if (a < c.seg_cap) {
                const int hi2 = sg.hi - kD * w;
                const int lo2 = max(hi2 - kD, 0);
                c.act[cur][a] = Seg{sg.start, sg.len, lo2, hi2};
                const uint32_t *src = c.phist[cur] + (int64_t)s * (kMaxWin * kBins) + w * kBins;
                uint32_t *dst = c.act_hist[cur] + a * kBins;
                for (int b = 0; b < kBins; ++b)
                    dst[b] = src[b];
            } else {
                set_status(c.status, kStOverflow);
            }
        }
        if (s < P) {  // leave the stats rows clean for their next use
            uint32_t *row = c.phist[cur] + (int64_t)s * (kMaxWin * kBins);
            for (int b = 0; b < kMaxWin * kBins; ++b)
                row[b] = 0;
            c.pand[cur][s] = ~0ull;
            c.por[cur][s] = 0ull;
        }
        fin_total += tf;
        __syncthreads();
        if (threadIdx.x == 0)
            s_act_base += ta;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.ctr->fin_count += fin_total;
        c.ctr->act_count[cur] = (int32_t)min((int64_t)s_act_base, c.seg_cap);
    }
    __syncthreads();
    // tile bases of all active segments of this pass
    const int A = min((int64_t)s_act_base, c.seg_cap);
    for (int r0 = 0; r0 < A; r0 += blockDim.x) {
        const int a = r0 + threadIdx.x;
        int tiles = (a < A) ? tiles_of(c.act[cur][a].len, kTile) : 0;
        int tt;
        int pt = block_excl_scan(tiles, &tt, sh);
        if (a < A)
            c.act_tile_base[cur][a] = s_tile_base + pt;
        __syncthreads();
        if (threadIdx.x == 0)
            s_tile_base += tt;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (A < c.seg_cap + 1)
            c.act_tile_base[cur][A] = s_tile_base;
        if (s_tile_base > c.tile_cap)
            set_status(c.status, kStOverflow);
        c.ctr->num_tiles[cur] = min((int64_t)s_tile_base, c.tile_cap);
    }
}

// ------------------------------------------------------------------ pass
struct PassSmem {
    uint32_t wcnt[kTPB / 32][kBins];  // per-warp digit counts -> exclusive prefixes
    uint32_t tile_off[kBins + 1];
    uint32_t tile_cnt[kBins];
    int32_t gbase[kBins];
    uint32_t nh[kBins * kBins];
    int32_t st_seg[2], st_start[2], st_cnt[2], st_k[2], st_tile[2];
    int32_t st_shk[2], st_shi[2];
    int32_t nt[2];   // next tile id, one slot per stage
    int32_t err;
    alignas(8) uint64_t bar[2];
};

template <typename KeyT>
struct PassLayout {
    static constexpr int kKeyBytes = kTile * (int)sizeof(KeyT) + 32;
    static constexpr int kIdxBytes = kTile * 4 + 32;
    static constexpr int kStage = ((kKeyBytes + kIdxBytes + 127) / 128) * 128;
    static constexpr int kHdr = ((int)sizeof(PassSmem) + 127) / 128 * 128;
    static constexpr int kTotal = kHdr + 2 * kStage;
};

// Issue the bulk copies of tile g into stage st (one thread).
template <typename KeyT>
__device__ __forceinline__ void pass_issue(const Ctx &c, int cur, int g, int st, PassSmem &S,
                                           unsigned char *stage, int A) {
    const int s = upper_index(c.act_tile_base[cur], A, g);
    const Seg sg = c.act[cur][s];
    const int k = g - c.act_tile_base[cur][s];
    const int64_t start = (int64_t)sg.start + (int64_t)k * kTile;
    const int cnt = (int)min((int64_t)kTile, (int64_t)sg.start + sg.len - start);
    constexpr int W = (int)sizeof(KeyT);
    const unsigned char *kb = c.keyb[cur];
    const unsigned char *ib = reinterpret_cast<const unsigned char *>(c.idxb[cur]);
    const int64_t k_lo = (start * W) & ~15ll, k_hi = ((start + cnt) * W + 15) & ~15ll;
    const int64_t i_lo = (start * 4) & ~15ll, i_hi = ((start + cnt) * 4 + 15) & ~15ll;
    S.st_seg[st] = s;
    S.st_start[st] = (int32_t)start;
    S.st_cnt[st] = cnt;
    S.st_k[st] = k;
    S.st_tile[st] = g;
    S.st_shk[st] = (int32_t)((start * W - k_lo) / W);
    S.st_shi[st] = (int32_t)((start * 4 - i_lo) / 4);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&S.bar[st], (uint32_t)((k_hi - k_lo) + (i_hi - i_lo)));
    bulk_g2s(stage, kb + k_lo, (uint32_t)(k_hi - k_lo), &S.bar[st]);
    bulk_g2s(stage + PassLayout<KeyT>::kKeyBytes, ib + i_lo, (uint32_t)(i_hi - i_lo), &S.bar[st]);
}

template <typename KeyT>
__global__ void __launch_bounds__(kTPB, 2) k_pass(Ctx c, int it) {
    extern __shared__ __align__(128) unsigned char smem[];
    PassSmem &S = *reinterpret_cast<PassSmem *>(smem);
    unsigned char *stages = smem + PassLayout<KeyT>::kHdr;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt();
    const uint32_t epoch = (uint32_t)it + 1;

    // clear the other parity's bucket accumulators (consumed by the last plan)
    {
        const int64_t rows = (int64_t)c.ctr->act_count[nxt] * kBins;
        for (int64_t r = (int64_t)blockIdx.x * kTPB + tid; r < rows; r += (int64_t)gridDim.x * kTPB) {
            c.band[nxt][r] = ~0ull;
            c.bor[nxt][r] = 0ull;
            uint4 *z = reinterpret_cast<uint4 *>(c.nh[nxt] + r * kBins);
            z[0] = make_uint4(0, 0, 0, 0);
            z[1] = make_uint4(0, 0, 0, 0);
            z[2] = make_uint4(0, 0, 0, 0);
            z[3] = make_uint4(0, 0, 0, 0);
        }
    }
    const int A = c.ctr->act_count[cur];
    const int ntiles = c.ctr->num_tiles[cur];
    if (A == 0 || ntiles == 0)
        return;

    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    for (int i = tid; i < kBins * kBins; i += kTPB)
        S.nh[i] = 0;
    __syncthreads();

    KeyT *okey = reinterpret_cast<KeyT *>(c.keyb[nxt]);
    int32_t *oidx = c.idxb[nxt];
    uint32_t phase[2] = {0, 0};
    int st = 0;
    if (tid == 0) {
        S.err = 0;
        int g = atomicAdd(&c.ctr->tile_ctr[it], 1);
        S.nt[0] = g;
        if (g < ntiles)
            pass_issue<KeyT>(c, cur, g, 0, S, stages, A);
    }
    __syncthreads();
    int g = S.nt[0];
    while (g < ntiles) {
        unsigned char *stage = stages + st * PassLayout<KeyT>::kStage;
        // prefetch the next tile into the other stage
        if (tid == 0) {
            int g2 = atomicAdd(&c.ctr->tile_ctr[it], 1);
            S.nt[st ^ 1] = g2;
            if (g2 < ntiles)
                pass_issue<KeyT>(c, cur, g2, st ^ 1, S, stages + (st ^ 1) * PassLayout<KeyT>::kStage, A);
        }
        const bool landed = mbar_wait_bounded(&S.bar[st], phase[st], 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            if (tid == 0) {
                mbar_wait_bounded(&S.bar[st], phase[st], 1ll << 26);
                if (S.nt[st ^ 1] < ntiles)
                    mbar_wait_bounded(&S.bar[st ^ 1], phase[st ^ 1], 1ll << 26);
            }
            return;
        }
        phase[st] ^= 1;
        const int s = S.st_seg[st];
        const int k = S.st_k[st];
        const int cnt = S.st_cnt[st];
        const Seg sg = c.act[cur][s];
        const int lo = sg.lo, hi = sg.hi;
        const unsigned dmask = (1u << (hi - lo)) - 1u;
        const KeyT *sk = reinterpret_cast<const KeyT *>(stage) + S.st_shk[st];
        const int32_t *si = reinterpret_cast<const int32_t *>(stage + PassLayout<KeyT>::kKeyBytes) + S.st_shi[st];

        // ---- load + warp-ballot ranking (order: warp, item, lane == memory order)
        KeyT key[kItems];
        int32_t idx[kItems];
        uint32_t rnk[kItems];
        uint32_t run = 0;  // lane d < 16: count of digit d in this warp so far
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int pos = wid * (32 * kItems) + i * 32 + lane;
            const bool valid = pos < cnt;
            key[i] = valid ? sk[pos] : (KeyT)0;
            idx[i] = valid ? si[pos] : 0;
            const unsigned dig = valid ? (unsigned)((unsigned long long)key[i] >> lo) & dmask : 0u;
            const unsigned vm = __ballot_sync(kFull, valid);
            unsigned peers = vm, mine = vm;
#pragma unroll
            for (int b = 0; b < kD; ++b) {
                const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                peers &= ((dig >> b) & 1u) ? bb : ~bb;
                mine &= ((lane >> b) & 1) ? bb : ~bb;
            }
            const uint32_t before = __shfl_sync(kFull, run, (int)dig);
            rnk[i] = before + __popc(peers & lt);
            run += __popc(mine);
        }
        if (lane < kBins)
            S.wcnt[wid][lane] = run;
        __syncthreads();
        // ---- tile histogram, warp prefixes, look-back (lanes 0..15 of warp 0)
        if (wid == 0 && lane < kBins) {
            const int d = lane;
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kTPB / 32; ++w) {
                uint32_t x = S.wcnt[w][d];
                S.wcnt[w][d] = tot;
                tot += x;
            }
            S.tile_cnt[d] = tot;
            // exclusive scan over the 16 digits
            uint32_t incl = tot;
#pragma unroll
            for (int o = 1; o < kBins; o <<= 1) {
                uint32_t y = __shfl_up_sync(0xffffu, incl, o);
                if (d >= o)
                    incl += y;
            }
            S.tile_off[d] = incl - tot;
            if (d == kBins - 1)
                S.tile_off[kBins] = incl;
            // decoupled look-back over earlier tiles of the same segment
            const int g0 = S.st_tile[st];
            unsigned long long *lbw = c.lb + (int64_t)g0 * kBins + d;
            uint32_t excl = 0;
            if (k == 0) {
                st_release_u64(lbw, lb_pack(epoch, kLbIncl, tot));
            } else {
                st_release_u64(lbw, lb_pack(epoch, kLbAgg, tot));
                int gp = g0 - 1;
                long long spins = 0;
                uint64_t t0 = 0;
                while (true) {
                    unsigned long long x = ld_acquire_u64(c.lb + (int64_t)gp * kBins + d);
                    const uint32_t ep = (uint32_t)(x >> 56);
                    const unsigned long long stt = (x >> 54) & 3ull;
                    if (ep != (epoch & 0xff) || stt == 0) {
                        ++spins;
                        if (spins == 1)
                            t0 = globaltimer_ns();
                        if (spins > (1ll << 26) || ((spins & 63) == 0 && globaltimer_ns() - t0 > kWaitLimitNs)) {
                            set_status(c.status, PBIT_ETIMEOUT);
                            S.err = 1;
                            break;
                        }
                        if (spins > 64)
                            __nanosleep(64);
                        continue;
                    }
                    excl += (uint32_t)(x & ((1ull << 54) - 1));
                    if (stt == kLbIncl)
                        break;
                    --gp;
                }
                st_release_u64(lbw, lb_pack(epoch, kLbIncl, (unsigned long long)excl + tot));
            }
            uint32_t bex = 0;
            const uint32_t *h = c.act_hist[cur] + (int64_t)s * kBins;
            for (int b = 0; b < d; ++b)
                bex += h[b];
            S.gbase[d] = sg.start + (int32_t)bex + (int32_t)excl;
        }
        __syncthreads();
        if (S.err) {  // a look-back gave up: write nothing, drain the prefetch
            if (tid == 0 && S.nt[st ^ 1] < ntiles)
                mbar_wait_bounded(&S.bar[st ^ 1], phase[st ^ 1], 1ll << 26);
            return;
        }
        // ---- local scatter into the stage buffer (now free: all items are in registers)
        KeyT *ok = reinterpret_cast<KeyT *>(stage);
        int32_t *oi = reinterpret_cast<int32_t *>(stage + PassLayout<KeyT>::kKeyBytes);
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int pos = wid * (32 * kItems) + i * 32 + lane;
            if (pos < cnt) {
                const unsigned dig = (unsigned)((unsigned long long)key[i] >> lo) & dmask;
                const uint32_t lp = S.tile_off[dig] + S.wcnt[wid][dig] + rnk[i];
                ok[lp] = key[i];
                oi[lp] = idx[i];
            }
        }
        __syncthreads();
        // ---- coalesced write-out (+ next-window histogram)
        const int nlo = max(lo - kD, 0);
        const unsigned nmask = (1u << (lo - nlo)) - 1u;
        if (lo == 0) {
            for (int j = tid; j < cnt; j += kTPB) {
                const KeyT kk = ok[j];
                const unsigned dig = (unsigned)((unsigned long long)kk >> lo) & dmask;
                const int dst = S.gbase[dig] + (j - (int)S.tile_off[dig]);
                if (dst < sg.start || dst >= sg.start + sg.len) {
                    set_status(c.status, kStOverflow);
                    continue;
                }
                c.F[dst] = oi[j];
            }
        } else {
            for (int j = tid; j < cnt; j += kTPB) {
                const KeyT kk = ok[j];
                const unsigned dig = (unsigned)((unsigned long long)kk >> lo) & dmask;
                const int dst = S.gbase[dig] + (j - (int)S.tile_off[dig]);
                if (dst < sg.start || dst >= sg.start + sg.len) {
                    set_status(c.status, kStOverflow);
                    continue;
                }
                okey[dst] = kk;
                oidx[dst] = oi[j];
                const unsigned nd = (unsigned)((unsigned long long)kk >> nlo) & nmask;
                atomicAdd(&S.nh[dig * kBins + nd], 1u);
            }
            // AND/OR of every output bucket: warp wid handles digits wid, wid+8
            for (int d = wid; d < kBins; d += kTPB / 32) {
                const int b0 = (int)S.tile_off[d], n0 = (int)S.tile_cnt[d];
                if (n0 == 0)
                    continue;
                unsigned long long aa = ~0ull, oo = 0ull;
                for (int j = lane; j < n0; j += 32) {
                    const unsigned long long kk = (unsigned long long)ok[b0 + j];
                    aa &= kk;
                    oo |= kk;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    aa &= __shfl_xor_sync(kFull, aa, o);
                    oo |= __shfl_xor_sync(kFull, oo, o);
                }
                if (lane == 0) {
                    const int64_t r = (int64_t)s * kBins + d;
                    atomicAnd(&c.band[cur][r], aa);
                    atomicOr(&c.bor[cur][r], oo);
                }
            }
            __syncthreads();
            {
                const uint32_t v = S.nh[tid];
                if (v) {
                    atomicAdd(&c.nh[cur][(int64_t)s * kBins * kBins + tid], v);
                    S.nh[tid] = 0;
                }
            }
        }
        __syncthreads();
        g = S.nt[st ^ 1];
        st ^= 1;
    }
}

// ------------------------------------------------------------------ plan
__device__ __forceinline__ int classify_bucket(const Ctx &c, int cur, int s, const Seg &sg, int d,
                                               uint32_t cnt, int *t_out) {
    // 0 none, 1 fin copy, 2 fin sort, 3 next active, 4 pending
    if (cnt == 0 || sg.lo == 0)
        return 0;
    const int64_t r = (int64_t)s * kBins + d;
    const unsigned long long v = (c.bor[cur][r] ^ c.band[cur][r]) & low_mask(sg.lo);
    if (cnt == 1 || v == 0)
        return 1;
    const int t = top_bit(v);
    *t_out = t;
    if ((int)cnt <= c.cutoff)
        return 2;
    return (t + kD >= sg.lo) ? 3 : 4;
}

__global__ void __launch_bounds__(1024) k_plan(Ctx c, int it) {
    __shared__ int sh[40];
    __shared__ int s_act, s_pend, s_fin, s_tiles;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int A = c.ctr->act_count[cur];
    if (threadIdx.x == 0) {
        s_act = 0;
        s_pend = 0;
        s_fin = c.ctr->fin_count;
        s_tiles = 0;
    }
    __syncthreads();
    for (int r0 = 0; r0 < A; r0 += blockDim.x) {
        const int s = r0 + threadIdx.x;
        Seg sg{0, 0, 0, 0};
        uint32_t h[kBins];
        int na = 0, np = 0, nf = 0, nt = 0;
        if (s < A) {
            sg = c.act[cur][s];
            for (int d = 0; d < kBins; ++d)
                h[d] = c.act_hist[cur][(int64_t)s * kBins + d];
            for (int d = 0; d < kBins; ++d) {
                int t = 0;
                int kd = classify_bucket(c, cur, s, sg, d, h[d], &t);
                na += kd == 3;
                np += kd == 4;
                nf += (kd == 1 || kd == 2);
                nt += (kd == 4) ? tiles_of(h[d], kStatTile) : 0;
            }
        } else {
            for (int d = 0; d < kBins; ++d)
                h[d] = 0;
        }
        int ta, tp, tf, tt;
        int pa = block_excl_scan(na, &ta, sh);
        int pp = block_excl_scan(np, &tp, sh);
        int pf = block_excl_scan(nf, &tf, sh);
        int pt = block_excl_scan(nt, &tt, sh);
        if (s < A) {
            int64_t a = (int64_t)s_act + pa, p = (int64_t)s_pend + pp, f = (int64_t)s_fin + pf;
            int64_t tb = (int64_t)s_tiles + pt;
            int32_t bstart = sg.start;
            for (int d = 0; d < kBins; ++d) {
                int t = 0;
                const uint32_t cnt = h[d];
                const int kd = classify_bucket(c, cur, s, sg, d, cnt, &t);
                if (kd == 1 || kd == 2) {
                    if (f < c.fin_cap)
                        c.fin[f] = Fin{bstart, (int32_t)cnt, kd == 2 ? t + 1 : 0, ((kd == 2 ? 1 : 0) << 8) | nxt};
                    else
                        set_status(c.status, kStOverflow);
                    ++f;
                } else if (kd == 3) {
                    if (a < c.seg_cap) {
                        const int nlo = max(sg.lo - kD, 0);
                        c.act[nxt][a] = Seg{bstart, (int32_t)cnt, nlo, sg.lo};
                        const uint32_t *src = c.nh[cur] + ((int64_t)s * kBins + d) * kBins;
                        uint32_t *dst = c.act_hist[nxt] + a * kBins;
                        for (int b = 0; b < kBins; ++b)
                            dst[b] = src[b];
                    } else {
                        set_status(c.status, kStOverflow);
                    }
                    ++a;
                } else if (kd == 4) {
                    if (p < c.seg_cap) {
                        c.pend[nxt][p] = Seg{bstart, (int32_t)cnt, 0, t + 1};
                        c.pend_tile_base[nxt][p] = (int32_t)tb;
                    } else {
                        set_status(c.status, kStOverflow);
                    }
                    tb += tiles_of(cnt, kStatTile);
                    ++p;
                }
                bstart += (int32_t)cnt;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_act += ta;
            s_pend += tp;
            s_fin += tf;
            s_tiles += tt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.ctr->act_count[nxt] = (int32_t)min((int64_t)s_act, c.seg_cap);
        c.ctr->pend_count[nxt] = (int32_t)min((int64_t)s_pend, c.seg_cap);
        if (s_pend < c.seg_cap)
            c.pend_tile_base[nxt][s_pend] = s_tiles;
        c.ctr->stat_tiles[nxt] = s_tiles;
        c.ctr->fin_count = (int32_t)min((int64_t)s_fin, c.fin_cap);
    }
}

// ------------------------------------------------------------- launchers
template <typename KeyT>
static void launch_pass_t(const Ctx &c, int it, cudaStream_t s, int sms) {
    const int smem = PassLayout<KeyT>::kTotal;
    cudaFuncSetAttribute(k_pass<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int per_sm = (2 * smem + 2048 <= 227 * 1024) ? 2 : 1;
    k_seg_stats<KeyT><<<sms * 4, kTPB, 0, s>>>(c, it);
    k_plan_pending<<<1, 1024, 0, s>>>(c, it);
    k_pass<KeyT><<<sms * per_sm, kTPB, smem, s>>>(c, it);
    k_plan<<<1, 1024, 0, s>>>(c, it);
}

void launch_plan_init(const Ctx &c, cudaStream_t s) { k_plan_init<<<1, 1024, 0, s>>>(c); }

void launch_iteration(const Ctx &c, int it, cudaStream_t s, int sms) {
    switch (c.key_bytes) {
    case 1: launch_pass_t<uint8_t>(c, it, s, sms); break;
    case 2: launch_pass_t<uint16_t>(c, it, s, sms); break;
    case 4: launch_pass_t<uint32_t>(c, it, s, sms); break;
    default: launch_pass_t<unsigned long long>(c, it, s, sms); break;
    }
}

int64_t launches_per_iteration() { return 4; }
int pass_tile() { return kTile; }
int stat_tile() { return kStatTile; }
int digit_bits() { return kD; }

}  // namespace pbit
