// msd.cu -- stage (b): Pbit's MSD digit passes over the ranked list.
//
// The paper splits the list on the top K bits, then recurses into each of the
// Omega = 2^K buckets with the next K bits (Sec. "Implementation in C++"),
// visiting buckets from Omega-1 down to 0 so that the concatenation comes out
// ascending (Sec. "Differences between sorting in descending and ascending
// order").  Here every recursion level is one data-parallel pass over all
// live buckets ("segments") at once: a stable counting split of each segment
// into 2^D sub-segments laid out in ascending digit order, which is the order
// the ascending concatenation produces.
//
// A pass needs, for every tile, where each of its digits starts in the
// output: the segment's bucket start plus the counts of that digit in the
// segment's earlier tiles.  Those per-tile counts are produced one step ahead
// -- by the previous pass while it writes each element (it knows the element's
// next tile and next digit), or by seg_stats for a segment's first pass -- and
// turned into prefixes by a two-level scan, so the pass itself has no
// dependence between tiles and can prefetch its next tile freely.
//
// One iteration (= one recursion level for every live segment):
//   seg_stats     pending segments: per-tile counts of the window under their
//                 top bit, and the AND/OR of their keys
//   plan_pending  pending -> active / small / mid / done / pending again (when the
//                 top window does not vary, the segment retries one window
//                 lower, at its highest varying bit); tile, chunk and
//                 next-row bases of all active segments
//   tile_scan     per chunk of 256 tiles: exclusive prefixes of the counts
//   chunk_scan    per segment: prefixes over its chunks; segment histogram
//   pass          per tile: warp-ballot ranking, stable scatter through
//                 shared memory; fused: counts per next-pass tile and AND/OR
//                 per output bucket
//   plan_count / plan_scan / plan_write
//                 output buckets -> next active / pending / small (warp
//                 finish) / mid-size (CTA finish) / done
#include "pbit_internal.cuh"

namespace pbit {

constexpr int kTPB = 256;             // threads per pass / stats CTA
constexpr int kItems = 8;             // items per thread in a pass tile
constexpr int kTileLog = 11;
constexpr int kTile = kTPB * kItems;  // 2048 elements per pass tile
static_assert(kTile == 1 << kTileLog, "tile is a power of two");
static_assert(kTile == kPassTile, "the plan kernels count tiles of kPassTile elements");
constexpr int kD = 4;                 // widest window of these kernels (16 buckets, the paper's K = 4)
constexpr int kBins = 1 << kD;
constexpr int kScanRows = kScanChunk; // tiles per scan chunk (one per thread)
constexpr int kRowPad = kBins;        // extra next-pass rows per segment (one per bucket)

// Block-wide exclusive scan of 16-vectors (one per thread, 256 threads):
// v[] becomes the exclusive prefix, tot[] the block totals (all threads).
__device__ void block_excl_scan16(uint32_t (&v)[kBins], uint32_t (&tot)[kBins], uint32_t *sh /* 8 x 16 + 16 */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc[kBins];
#pragma unroll
    for (int j = 0; j < kBins; ++j) {
        uint32_t x = v[j];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, x, o);
            if (lane >= o)
                x += y;
        }
        inc[j] = x;
    }
    if (lane == 31) {
#pragma unroll
        for (int j = 0; j < kBins; ++j)
            sh[wid * kBins + j] = inc[j];
    }
    __syncthreads();
    if (threadIdx.x < kBins) {
        const int j = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < kTPB / 32; ++w) {
            const uint32_t x = sh[w * kBins + j];
            sh[w * kBins + j] = run;
            run += x;
        }
        sh[(kTPB / 32) * kBins + j] = run;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kBins; ++j) {
        v[j] = inc[j] - v[j] + sh[wid * kBins + j];
        tot[j] = sh[(kTPB / 32) * kBins + j];
    }
    __syncthreads();
}

__device__ __forceinline__ int top_bit(unsigned long long v) { return 63 - __clzll((long long)v); }

// A bucket of more than the cutoff goes to the CTA finish when it fits its
// shared memory and at most kMidSpan of its key bits vary (v: varying bits).
__device__ __forceinline__ bool mid_bucket(int len, unsigned long long v) {
    return len <= kMidCap && (v == 0 || top_bit(v) - (__ffsll((long long)v) - 1) < kMidSpan);
}
__device__ __forceinline__ unsigned long long low_mask(int bits) {
    return bits >= 64 ? ~0ull : ((1ull << bits) - 1ull);
}

// ------------------------------------------------------------- plan_init
// Lists become the first segments: empty lists vanish, lists up to the
// cutoff go straight to the shared-memory finish, the rest are pending.
__global__ void __launch_bounds__(1024) k_plan_init(Ctx c) {
    griddep_wait();
    __shared__ int sh[40];
    __shared__ int s_fin_base, s_pend_base, s_tile_base, s_mid_base;
    if (*(volatile int32_t *)c.status)
        return;
    if (threadIdx.x == 0) {
        s_fin_base = 0;
        s_pend_base = 0;
        s_tile_base = 0;
        s_mid_base = 0;
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
        // (a stage check forces every list of two or more nodes into the passes)
        const int cut = c.force_pass ? 1 : c.cutoff;
        int is_fin = (i < L && n >= 1 && n <= cut) ? 1 : 0;
        // (a list's varying bits are not known yet: only M bits few enough
        // for the CTA finish qualify it directly; others go through seg_stats)
        int is_mid = (i < L && n > cut && n <= kMidCap && c.M <= kMidSpan && !c.force_pass) ? 1 : 0;
        int is_pend = (i < L && n > cut && !is_mid) ? 1 : 0;
        int tiles = is_pend ? tiles_of(n, kTile) : 0;
        int tf, tp, tt, tm;
        int pf = block_excl_scan(is_fin, &tf, sh);
        int pp = block_excl_scan(is_pend, &tp, sh);
        int pt = block_excl_scan(tiles, &tt, sh);
        int pm = block_excl_scan(is_mid, &tm, sh);
        if (is_mid) {
            int k = s_mid_base + pm;
            if (k < c.mid_cap)
                c.mid[k] = Fin{start, n, c.M, (1 << 8) | 0};
            else
                set_status(c.status, kStOverflow);
        }
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
                c.pend[0][k] = Seg{start, n, 0, (int16_t)c.M, 0, 0, 0};
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
            s_mid_base += tm;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.ctr->fin_count = s_fin_base;
        c.ctr->mid_count = (int32_t)min((int64_t)s_mid_base, c.mid_cap);
        c.ctr->pend_count[0] = (int32_t)min((int64_t)s_pend_base, c.seg_cap);
        if (s_pend_base < c.seg_cap)
            c.pend_tile_base[0][s_pend_base] = s_tile_base;
        c.ctr->stat_tiles[0] = s_tile_base;
        c.ctr->act_count[0] = 0;
        c.ctr->brows[0] = 0;
        if (s_tile_base > c.row_cap)
            set_status(c.status, kStOverflow);
    }
}

// ------------------------------------------------------------- seg_stats
// For every pass tile of every pending segment: the counts of the digits in
// the window [max(hi-D,0), hi) (plain stores into its tcnt row, placed after
// the rows the previous pass filled), and the AND/OR of the segment's keys.
template <typename KeyT>
__global__ void __launch_bounds__(kTPB) k_seg_stats(Ctx c, int it) {
    griddep_wait();
    __shared__ uint32_t s_cnt[kBins];
    __shared__ unsigned long long s_and, s_or;
    __shared__ int s_aseg;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int P = c.ctr->pend_count[cur];
    const int ntiles = c.ctr->stat_tiles[cur];
    const int rbase = c.ctr->brows[cur];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long my_elems = 0;
    if (threadIdx.x < kBins)
        s_cnt[threadIdx.x] = 0;
    if (threadIdx.x == 0) {
        s_and = ~0ull;
        s_or = 0ull;
        s_aseg = -1;
    }
    // tiles in a static grid-stride order (uniform work: no claiming counter)
    for (int g = blockIdx.x; g < ntiles; g += gridDim.x) {
        __syncthreads();  // the previous tile's counts are stored and cleared
        const int s = upper_index(c.pend_tile_base[cur], P, g);
        if (threadIdx.x == 0 && s != s_aseg) {  // AND/OR are merged per segment, not per tile
            if (s_aseg >= 0) {
                atomicAnd(&c.pand[cur][s_aseg], s_and);
                atomicOr(&c.por[cur][s_aseg], s_or);
            }
            s_and = ~0ull;
            s_or = 0ull;
            s_aseg = s;
        }
        __syncthreads();  // the reset above precedes this tile's merges into s_and / s_or
        const Seg sg = c.pend[cur][s];
        const int k = g - c.pend_tile_base[cur][s];
        const int64_t b0 = (int64_t)sg.start + (int64_t)k * kTile;
        const int cnt = (int)min((int64_t)kTile, (int64_t)sg.start + sg.len - b0);
        const KeyT *keys = reinterpret_cast<const KeyT *>(c.keyb[sg.buf & 1]);
        const int hi = sg.hi, lo = max(hi - c.D, 0);
        const unsigned dmask = (1u << (hi - lo)) - 1u;
        my_elems += cnt;
        using U = typename KeyWord<KeyT>::U;  // 32-bit words for keys up to 4 bytes
        U kv[kItems];
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
            const int pos = wid * 32 * kItems + u * 32 + lane;
            kv[u] = pos < cnt ? (U)keys[b0 + pos] : (U)0;
        }
        uint32_t wc = 0;
        U w_and = ~(U)0, w_or = 0;
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
            const int pos = wid * 32 * kItems + u * 32 + lane;
            const bool valid = pos < cnt;
            if (valid) {
                w_and &= kv[u];
                w_or |= kv[u];
            }
            const unsigned dig = (unsigned)(kv[u] >> lo) & dmask;
            unsigned m = __ballot_sync(kFull, valid);
#pragma unroll
            for (int b = 0; b < kD; ++b) {
                const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                m &= ((lane >> b) & 1) ? bb : ~bb;
            }
            wc += __popc(m);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            w_and &= __shfl_xor_sync(kFull, w_and, o);
            w_or |= __shfl_xor_sync(kFull, w_or, o);
        }
        const unsigned long long a_and = (unsigned long long)w_and, a_or = (unsigned long long)w_or;
        if (lane < kBins && wc)
            atomicAdd(&s_cnt[lane], wc);
        if (lane == 0) {
            atomicAnd(&s_and, a_and);
            atomicOr(&s_or, a_or);
        }
        __syncthreads();
        if (threadIdx.x < kBins) {
            const int64_t row = (int64_t)rbase + g;
            if (row < c.row_cap)
                c.tcnt[cur][row * kBins + threadIdx.x] = s_cnt[threadIdx.x];
            s_cnt[threadIdx.x] = 0;
        }
    }
    if (threadIdx.x == 0) {
        if (s_aseg >= 0) {
            atomicAnd(&c.pand[cur][s_aseg], s_and);
            atomicOr(&c.por[cur][s_aseg], s_or);
        }
        if (my_elems)
            atomicAdd((unsigned long long *)&c.ctr->stat_elems[it], (unsigned long long)my_elems);
    }
}

// ---------------------------------------------------------- plan_pending
__global__ void __launch_bounds__(1024) k_plan_pending(Ctx c, int it) {
    griddep_wait();
    __shared__ int sh[40];
    __shared__ int s_act_base, s_re_base, s_re_tiles, s_tile_base, s_chunk_base, s_nrow_base;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int P = c.ctr->pend_count[cur];
    const int rbase = c.ctr->brows[cur];
    if (threadIdx.x == 0) {
        s_act_base = c.ctr->act_count[cur];
        s_re_base = 0;
        s_re_tiles = 0;
        s_tile_base = 0;
        s_chunk_base = 0;
        s_nrow_base = 0;
    }
    __syncthreads();
    int fin_total = 0, mid_total = 0;
    for (int r0 = 0; r0 < P; r0 += blockDim.x) {
        const int s = r0 + threadIdx.x;
        int kind = 0;  // 1 small (no varying bit), 2 small, 3 active, 4 pending again, 5 active final
        Seg sg{0, 0, 0, 0, 0, 0, 0};
        int t = 0;
        if (s < P) {
            sg = c.pend[cur][s];
            const unsigned long long v = (c.por[cur][s] ^ c.pand[cur][s]) & low_mask(sg.hi);
            if (sg.len <= 1 || v == 0) {
                kind = sg.len <= c.cutoff ? 1 : 5;
            } else {
                t = top_bit(v);
                if (sg.len <= c.cutoff && !c.force_pass)
                    kind = 2;
                else
                    kind = (t >= sg.hi - c.D) ? 3 : 4;
            }
            if (kind >= 3 && mid_bucket(sg.len, v) && !c.force_pass)
                kind = 6;  // one CTA finishes it
        }
        const int tiles = kind == 4 ? tiles_of(sg.len, kTile) : 0;
        int tf, ta, tr, tt;
        const int pf = block_excl_scan(kind == 1 || kind == 2, &tf, sh);
        const int pa = block_excl_scan(kind == 3 || kind == 5, &ta, sh);
        const int pr = block_excl_scan(kind == 4, &tr, sh);
        const int pt = block_excl_scan(tiles, &tt, sh);
        int tm;
        const int pm = block_excl_scan(kind == 6, &tm, sh);
        if (kind == 6) {
            const int64_t k = (int64_t)c.ctr->mid_count + mid_total + pm;
            if (k < c.mid_cap)
                c.mid[k] = Fin{sg.start, sg.len, sg.hi, (1 << 8) | (sg.buf & 1)};
            else
                set_status(c.status, kStOverflow);
        } else if (kind == 1 || kind == 2) {
            const int64_t k = (int64_t)c.ctr->fin_count + fin_total + pf;
            if (k < c.fin_cap)
                c.fin[k] = Fin{sg.start, sg.len, kind == 2 ? t + 1 : 0, ((kind == 2 ? 1 : 0) << 8) | (sg.buf & 1)};
            else
                set_status(c.status, kStOverflow);
        } else if (kind == 3 || kind == 5) {
            const int64_t a = (int64_t)s_act_base + pa;
            if (a < c.seg_cap)
                c.act[cur][a] = Seg{sg.start, sg.len, (int16_t)max(sg.hi - c.D, 0), sg.hi, sg.buf,
                                    rbase + c.pend_tile_base[cur][s], kind == 5 ? 1 : 0};
            else
                set_status(c.status, kStOverflow);
        } else if (kind == 4) {
            const int64_t r = (int64_t)s_re_base + pr;
            if (r < c.seg_cap) {
                c.pend[nxt][r] = Seg{sg.start, sg.len, 0, (int16_t)(t + 1), sg.buf, 0, 0};
                c.pend_tile_base[nxt][r] = s_re_tiles + pt;
            } else {
                set_status(c.status, kStOverflow);
            }
        }
        if (s < P) {  // leave the AND/OR slots clean for their next use
            c.pand[cur][s] = ~0ull;
            c.por[cur][s] = 0ull;
        }
        fin_total += tf;
        mid_total += tm;
        __syncthreads();
        if (threadIdx.x == 0) {
            s_act_base += ta;
            s_re_base += tr;
            s_re_tiles += tt;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        c.ctr->fin_count += fin_total;
        c.ctr->mid_count = (int32_t)min((int64_t)c.ctr->mid_count + mid_total, c.mid_cap);
        c.ctr->act_count[cur] = (int32_t)min((int64_t)s_act_base, c.seg_cap);
        c.ctr->pend_count[nxt] = (int32_t)min((int64_t)s_re_base, c.seg_cap);
        c.ctr->stat_tiles[nxt] = s_re_tiles;
    }
    __syncthreads();
    // tile, scan-chunk and next-row bases of all active segments of this pass
    // (8 consecutive segments per thread per round); the 8-bit passes count
    // their tiles with a histogram kernel instead of next-pass rows
    constexpr int kPer = 8;
    const bool wide = c.D > kD;
    const int A = (int)min((int64_t)s_act_base, c.seg_cap);
    long long my_elems = 0, my_final = 0;
    for (int r0 = 0; r0 < A; r0 += blockDim.x * kPer) {
        const int a0 = r0 + threadIdx.x * kPer;
        int tiles = 0, chunks = 0, nrows = 0;
        for (int u = 0; u < kPer && a0 + u < A; ++u) {
            const Seg sa = c.act[cur][a0 + u];
            const int nt = tiles_of(sa.len, kTile);
            tiles += nt;
            chunks += nt > 1 ? tiles_of(nt, kScanRows) : 0;
            nrows += (!wide && sa.lo > 0 && !sa.final) ? nt + kRowPad : 0;
            my_elems += sa.len;
            if (sa.lo == 0 || sa.final)
                my_final += sa.len;
        }
        int tt, tc, tn;
        int pt = block_excl_scan(tiles, &tt, sh);
        int pc = block_excl_scan(chunks, &tc, sh);
        int pn = block_excl_scan(nrows, &tn, sh);
        for (int u = 0; u < kPer && a0 + u < A; ++u) {
            const Seg sa = c.act[cur][a0 + u];
            const int nt = tiles_of(sa.len, kTile);
            c.act_tile_base[cur][a0 + u] = s_tile_base + pt;
            c.act_chunk_base[cur][a0 + u] = s_chunk_base + pc;
            c.act_nrow_base[cur][a0 + u] = s_nrow_base + pn;
            pt += nt;
            pc += nt > 1 ? tiles_of(nt, kScanRows) : 0;
            pn += (!wide && sa.lo > 0 && !sa.final) ? nt + kRowPad : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_tile_base += tt;
            s_chunk_base += tc;
            s_nrow_base += tn;
        }
        __syncthreads();
    }
    if (my_elems) {
        atomicAdd((unsigned long long *)&c.ctr->pass_elems[it], (unsigned long long)my_elems);
        atomicAdd((unsigned long long *)&c.ctr->pass_final_elems[it], (unsigned long long)my_final);
    }
    if (threadIdx.x == 0) {
        c.act_tile_base[cur][A] = s_tile_base;
        c.act_chunk_base[cur][A] = s_chunk_base;
        c.act_nrow_base[cur][A] = s_nrow_base;
        if (s_tile_base > c.tile_cap || s_chunk_base > c.scan_cap || s_nrow_base + c.ctr->stat_tiles[nxt] > c.row_cap)
            set_status(c.status, kStOverflow);
        c.ctr->num_tiles[cur] = (int32_t)min((int64_t)s_tile_base, c.tile_cap);
        c.ctr->num_chunks[cur] = (int32_t)min((int64_t)s_chunk_base, c.scan_cap);
        c.ctr->brows[nxt] = s_nrow_base;
    }
}

// ------------------------------------------------------------- tile_scan
// Zero the next pass's count rows; then, per chunk of 256 tiles of an active
// segment, replace each tile's counts by the exclusive prefix within the
// chunk and record the chunk totals.
__global__ void __launch_bounds__(kTPB) k_tile_scan(Ctx c, int it) {
    griddep_wait();
    __shared__ uint32_t sh[(kTPB / 32 + 1) * kBins];
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    {
        const int64_t words = (int64_t)c.ctr->brows[nxt] * kBins / 4;
        uint4 *z = reinterpret_cast<uint4 *>(c.tcnt[nxt]);
        for (int64_t i = (int64_t)blockIdx.x * kTPB + threadIdx.x; i < words; i += (int64_t)gridDim.x * kTPB)
            z[i] = make_uint4(0, 0, 0, 0);
    }
    const int A = c.ctr->act_count[cur];
    const int nch = c.ctr->num_chunks[cur];
    for (int ch = blockIdx.x; ch < nch; ch += gridDim.x) {
        const int a = upper_index(c.act_chunk_base[cur], A, ch);
        const Seg sg = c.act[cur][a];
        const int lc = ch - c.act_chunk_base[cur][a];
        const int nt = c.act_tile_base[cur][a + 1] - c.act_tile_base[cur][a];
        const int t = lc * kScanRows + threadIdx.x;
        uint32_t v[kBins], tot[kBins];
        uint4 *row = reinterpret_cast<uint4 *>(c.tcnt[cur] + ((int64_t)sg.row + t) * kBins);
        if (t < nt) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint4 x = row[q];
                v[4 * q] = x.x;
                v[4 * q + 1] = x.y;
                v[4 * q + 2] = x.z;
                v[4 * q + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kBins; ++j)
                v[j] = 0;
        }
        block_excl_scan16(v, tot, sh);
        if (t < nt) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                row[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        if (threadIdx.x < kBins)
            c.ctot[(int64_t)ch * kBins + threadIdx.x] = tot[threadIdx.x];
    }
}

// ------------------------------------------------------------ chunk_scan
// One warp per active segment (lanes 0..15 = digits): exclusive prefixes over
// its chunks (in place) and the segment's digit histogram.  A segment of one
// tile has no chunk: its histogram is its tile's row.
__global__ void __launch_bounds__(kTPB) k_chunk_scan(Ctx c, int it) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int A = c.ctr->act_count[cur];
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t a = gw; a < A; a += nw) {
        if (lane >= kBins)
            continue;
        const int nt = c.act_tile_base[cur][a + 1] - c.act_tile_base[cur][a];
        uint32_t run = 0;
        if (nt == 1) {
            run = c.tcnt[cur][(int64_t)c.act[cur][a].row * kBins + lane];
        } else {
            const int c0 = c.act_chunk_base[cur][a], c1 = c.act_chunk_base[cur][a + 1];
            for (int ch = c0; ch < c1; ++ch) {
                uint32_t *p = c.ctot + (int64_t)ch * kBins + lane;
                const uint32_t t = *p;
                *p = run;
                run += t;
            }
        }
        c.act_hist[cur][a * kBins + lane] = run;
    }
}

// ------------------------------------------------------------------ pass
struct PassSmem {
    uint32_t wcnt[kTPB / 32][kBins];  // per-warp digit counts -> tile positions of each warp's digits
    uint32_t tile_off[kBins + 1];
    uint32_t tile_cnt[kBins];
    int32_t gbase[kBins];             // output position of this tile's first element of each digit
    int32_t gdelta[kBins];            // gbase - tile offset: output position = gdelta + tile position
    int32_t split[kBins];             // first output position in next-pass tile k0 + 1
    int32_t nrow[kBins];              // first next-pass row of each output bucket
    int32_t k0[kBins];                // next-pass tile of this tile's first element per bucket
    uint32_t nc[kBins * 2 * kBins];   // counts per (bucket, next tile k0/k0+1, next digit)
    unsigned long long aand[kBins], aor[kBins];  // AND/OR per bucket, merged over this CTA's tiles
    int32_t aseg;                     // segment those belong to (-1: none)
    int32_t st_seg[2], st_cnt[2], st_k[2], st_shk[2], st_shi[2];
    int32_t nt[2];
    alignas(8) uint64_t bar[2];
};

template <typename KeyT>
struct PassLayout {
    static constexpr int kKeyBytes = kTile * (int)sizeof(KeyT) + 32;
    static constexpr int kIdxBytes = kTile * 4 + 32;
    static constexpr int kStage = ((kKeyBytes + kIdxBytes + 127) / 128) * 128;
    static constexpr int kHdr = ((int)sizeof(PassSmem) + 127) / 128 * 128;
    static constexpr int kTotal = kHdr + 2 * kStage;
    static constexpr int kMinBlocks = sizeof(KeyT) == 8 ? 3 : 4;
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
    const unsigned char *kb = c.keyb[sg.buf & 1];
    const unsigned char *ib = reinterpret_cast<const unsigned char *>(c.idxb[sg.buf & 1]);
    const int64_t k_lo = (start * W) & ~15ll, k_hi = ((start + cnt) * W + 15) & ~15ll;
    const int64_t i_lo = (start * 4) & ~15ll, i_hi = ((start + cnt) * 4 + 15) & ~15ll;
    S.st_seg[st] = s;
    S.st_cnt[st] = cnt;
    S.st_k[st] = k;
    S.st_shk[st] = (int32_t)((start * W - k_lo) / W);
    S.st_shi[st] = (int32_t)((start * 4 - i_lo) / 4);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&S.bar[st], (uint32_t)((k_hi - k_lo) + (i_hi - i_lo)));
    bulk_g2s(stage, kb + k_lo, (uint32_t)(k_hi - k_lo), &S.bar[st]);
    bulk_g2s(stage + PassLayout<KeyT>::kKeyBytes, ib + i_lo, (uint32_t)(i_hi - i_lo), &S.bar[st]);
}

// Persistent CTAs take tiles from a counter and double-buffer them: the bulk
// copy of the next tile is in flight while the current one is ranked and
// written.  Tiles are independent: every tile reads its digits' output
// positions from the scanned counts.
template <typename KeyT>
__global__ void __launch_bounds__(kTPB, PassLayout<KeyT>::kMinBlocks) k_pass(Ctx c, int it) {
    griddep_wait();
    extern __shared__ __align__(128) unsigned char smem[];
    PassSmem &S = *reinterpret_cast<PassSmem *>(smem);
    unsigned char *stages = smem + PassLayout<KeyT>::kHdr;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt();

    // reset the other parity's bucket AND/OR (consumed by the last plan)
    {
        const int64_t rows = (int64_t)c.ctr->act_count[nxt] * kBins;
        for (int64_t r = (int64_t)blockIdx.x * kTPB + tid; r < rows; r += (int64_t)gridDim.x * kTPB) {
            c.band[nxt][r] = ~0ull;
            c.bor[nxt][r] = 0ull;
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
    for (int i = tid; i < kBins * 2 * kBins; i += kTPB)
        S.nc[i] = 0;
    if (tid < kBins) {
        S.aand[tid] = ~0ull;
        S.aor[tid] = 0ull;
    }
    if (tid == 0)
        S.aseg = -1;
    uint32_t phases = 0;  // bit b: parity of stage b's barrier
    int st = 0;
    if (tid == 0) {
        const int g = atomicAdd(&c.ctr->tile_ctr[it], 1);
        S.nt[0] = g;
        if (g < ntiles)
            pass_issue<KeyT>(c, cur, g, 0, S, stages, A);
    }
    __syncthreads();
    int g = S.nt[0];
    while (g < ntiles) {
        unsigned char *stage = stages + st * PassLayout<KeyT>::kStage;
        if (tid == 0) {  // prefetch the next tile into the other stage
            const int g2 = atomicAdd(&c.ctr->tile_ctr[it], 1);
            S.nt[st ^ 1] = g2;
            if (g2 < ntiles)
                pass_issue<KeyT>(c, cur, g2, st ^ 1, S, stages + (st ^ 1) * PassLayout<KeyT>::kStage, A);
        }
        // per-tile output bases (warp 1; overlaps the copy wait of the others)
        const int s = S.st_seg[st];
        const int k = S.st_k[st];
        const int cnt = S.st_cnt[st];
        const Seg sg = c.act[cur][s];
        const int lo = sg.lo, hi = sg.hi;
        if (wid == 1 && lane < kBins) {
            const int d = lane;
            const uint32_t h = c.act_hist[cur][(int64_t)s * kBins + d];
            uint32_t ex = h;  // exclusive prefix over digits of the segment histogram
            uint32_t nt_d = (uint32_t)tiles_of(h, kTile);
#pragma unroll
            for (int o = 1; o < kBins; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffu, ex, o);
                const uint32_t z = __shfl_up_sync(0xffffu, nt_d, o);
                if (d >= o) {
                    ex += y;
                    nt_d += z;
                }
            }
            ex -= h;
            nt_d -= (uint32_t)tiles_of(h, kTile);
            uint32_t before = 0;  // the first tile of a segment starts every bucket
            if (k > 0) {
                const int ch = c.act_chunk_base[cur][s] + k / kScanRows;
                before = c.ctot[(int64_t)ch * kBins + d] + c.tcnt[cur][((int64_t)sg.row + k) * kBins + d];
            }
            const int32_t bst = sg.start + (int32_t)ex;  // start of output bucket d
            const int32_t k0 = (int32_t)(before >> kTileLog);
            S.gbase[d] = bst + (int32_t)before;
            S.k0[d] = k0;
            S.split[d] = bst + ((k0 + 1) << kTileLog);  // first position of next-pass tile k0 + 1
            S.nrow[d] = c.act_nrow_base[cur][s] + (int32_t)nt_d;
            const int as = S.aseg;
            if (as != s) {  // new segment: flush the merged AND/OR of the previous one
                if (as >= 0 && (S.aand[d] != ~0ull || S.aor[d] != 0ull)) {
                    atomicAnd(&c.band[cur][(int64_t)as * kBins + d], S.aand[d]);
                    atomicOr(&c.bor[cur][(int64_t)as * kBins + d], S.aor[d]);
                }
                S.aand[d] = ~0ull;
                S.aor[d] = 0ull;
            }
            __syncwarp(0xffffu);
            if (d == 0)
                S.aseg = s;
        }
        uint32_t *wc = S.wcnt[wid];  // this warp's digit counts, then its digits' tile positions
        // one thread waits for the copy (acquire), the barrier then publishes
        // the tile to the whole CTA
        const bool landed = (tid != 0) || mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            if (tid == 0) {  // wait (bounded) for the copies still in flight before leaving
                mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
                if (S.nt[st ^ 1] < ntiles)
                    mbar_wait_bounded(&S.bar[st ^ 1], (phases >> (st ^ 1)) & 1u, 1ll << 26);
            }
            return;
        }
        phases ^= 1u << st;
        const unsigned dmask = (1u << (hi - lo)) - 1u;
        const KeyT *sk = reinterpret_cast<const KeyT *>(stage) + S.st_shk[st];
        const int32_t *si = reinterpret_cast<const int32_t *>(stage + PassLayout<KeyT>::kKeyBytes) + S.st_shi[st];

        // ---- load + warp-ballot ranking (order: warp, item, lane == memory order).
        // Four ballots give each lane the lanes holding its digit (peers) and
        // lane d < 16 the count of digit d in the item (mine); lane d keeps the
        // running count of digit d over the warp's earlier items.
        KeyT key[kItems];
        int32_t idx[kItems];
        uint32_t rnk[kItems];
        uint32_t run = 0;
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int pos = wid * (32 * kItems) + i * 32 + lane;
            const bool valid = pos < cnt;
            key[i] = valid ? sk[pos] : (KeyT)0;
            idx[i] = valid ? si[pos] : 0;
            const unsigned dig = valid ? digit_of<KeyT>(key[i], lo, dmask) : 0u;
            const unsigned vm = __ballot_sync(kFull, valid);
            unsigned peers = vm, mine = vm;
#pragma unroll
            for (int b = 0; b < kD; ++b) {
                const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                peers &= ((dig >> b) & 1u) ? bb : ~bb;
                mine &= ((lane >> b) & 1) ? bb : ~bb;
            }
            rnk[i] = __shfl_sync(kFull, run, (int)dig) + (uint32_t)__popc(peers & lt);
            run += (uint32_t)__popc(mine);
        }
        if (lane < kBins)
            wc[lane] = run;
        __syncthreads();
        if (wid == 0 && lane < kBins) {  // tile histogram, digit offsets, per-warp bases
            const int d = lane;
            uint32_t tot = 0;
#pragma unroll
            for (int w = 0; w < kTPB / 32; ++w)
                tot += S.wcnt[w][d];
            uint32_t incl = tot;
#pragma unroll
            for (int o = 1; o < kBins; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffu, incl, o);
                if (d >= o)
                    incl += y;
            }
            uint32_t run = incl - tot;  // tile offset of digit d
            S.tile_off[d] = run;
            S.tile_cnt[d] = tot;
            S.gdelta[d] = S.gbase[d] - (int32_t)run;
#pragma unroll
            for (int w = 0; w < kTPB / 32; ++w) {
                const uint32_t x = S.wcnt[w][d];
                S.wcnt[w][d] = run;
                run += x;
            }
        }
        __syncthreads();
        // ---- local scatter into the stage buffer (free now: all items are in registers)
        KeyT *ok = reinterpret_cast<KeyT *>(stage);
        int32_t *oi = reinterpret_cast<int32_t *>(stage + PassLayout<KeyT>::kKeyBytes);
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
            const int pos = wid * (32 * kItems) + i * 32 + lane;
            if (pos < cnt) {
                const uint32_t lp = wc[digit_of<KeyT>(key[i], lo, dmask)] + rnk[i];
                ok[lp] = key[i];
                oi[lp] = idx[i];
            }
        }
        __syncthreads();
        // ---- coalesced write-out (+ counts of the next pass's tiles)
        KeyT *okey = reinterpret_cast<KeyT *>(c.keyb[(sg.buf & 1) ^ 1]);
        int32_t *oidx = c.idxb[(sg.buf & 1) ^ 1];
        if (lo == 0 || sg.final) {
#pragma unroll
            for (int u = 0; u < kItems; ++u) {
                const int j = u * kTPB + tid;
                if (j < cnt) {
                    const int dst = S.gdelta[digit_of<KeyT>(ok[j], lo, dmask)] + j;
                    if ((unsigned)(dst - sg.start) >= (unsigned)sg.len)
                        set_status(c.status, kStOverflow);
                    else
                        c.F[dst] = oi[j];
                }
            }
        } else {
            const int nlo = max(lo - c.D, 0);
            const unsigned nmask = (1u << (lo - nlo)) - 1u;
#pragma unroll
            for (int u = 0; u < kItems; ++u) {
                const int j = u * kTPB + tid;
                if (j < cnt) {
                    const KeyT kk = ok[j];
                    const unsigned dig = digit_of<KeyT>(kk, lo, dmask);
                    const int dst = S.gdelta[dig] + j;
                    if ((unsigned)(dst - sg.start) >= (unsigned)sg.len) {
                        set_status(c.status, kStOverflow);
                    } else {
                        okey[dst] = kk;
                        oidx[dst] = oi[j];
                        const unsigned nd = digit_of<KeyT>(kk, nlo, nmask);
                        const unsigned kk1 = dst >= S.split[dig] ? 1u : 0u;  // next-pass tile k0 or k0 + 1
                        atomicAdd(&S.nc[(dig * 2 + kk1) * kBins + nd], 1u);
                    }
                }
            }
            // AND/OR of every output bucket: warp wid handles digits wid, wid+8
            using U = typename KeyWord<KeyT>::U;
            for (int d = wid; d < kBins; d += kTPB / 32) {
                const int b0 = (int)S.tile_off[d], n0 = (int)S.tile_cnt[d];
                if (n0 == 0)
                    continue;
                U aa = ~(U)0, oo = 0;
                for (int j = lane; j < n0; j += 32) {
                    const U kk = (U)ok[b0 + j];
                    aa &= kk;
                    oo |= kk;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    aa &= __shfl_xor_sync(kFull, aa, o);
                    oo |= __shfl_xor_sync(kFull, oo, o);
                }
                if (lane == 0) {  // keys are zero-extended to 64 bits, as in seg_stats
                    S.aand[d] &= (unsigned long long)aa;
                    S.aor[d] |= (unsigned long long)oo;
                }
            }
            __syncthreads();
            for (int i = tid; i < kBins * 2 * kBins; i += kTPB) {
                const uint32_t v = S.nc[i];
                if (v) {
                    const int d = i / (2 * kBins), kk1 = (i / kBins) & 1, nd = i % kBins;
                    const int64_t row = (int64_t)S.nrow[d] + S.k0[d] + kk1;
                    if (row < c.row_cap)
                        atomicAdd(&c.tcnt[nxt][row * kBins + nd], v);
                    else
                        set_status(c.status, kStOverflow);
                    S.nc[i] = 0;
                }
            }
        }
        __syncthreads();
        g = S.nt[st ^ 1];
        st ^= 1;
    }
    if (tid < kBins && S.aseg >= 0 && (S.aand[tid] != ~0ull || S.aor[tid] != 0ull)) {
        atomicAnd(&c.band[cur][(int64_t)S.aseg * kBins + tid], S.aand[tid]);
        atomicOr(&c.bor[cur][(int64_t)S.aseg * kBins + tid], S.aor[tid]);
    }
}

// ------------------------------------------------------------------ plan
// kinds: 0 none, 1 small (no varying bit), 2 small, 3 next active, 4 pending,
// 5 next active final (all keys equal; written straight to F by the pass),
// 6 mid-size (finished by one CTA in shared memory)
__device__ __forceinline__ int classify_bucket(const Ctx &c, int cur, int s, const Seg &sg, int d,
                                               uint32_t cnt, int *t_out) {
    if (cnt == 0 || sg.lo == 0 || sg.final)
        return 0;
    const int64_t r = (int64_t)s * kBins + d;
    const unsigned long long v = (c.bor[cur][r] ^ c.band[cur][r]) & low_mask(sg.lo);
    if ((int)cnt > c.cutoff && mid_bucket((int)cnt, v))
        return 6;  // one CTA finishes it
    if (cnt == 1 || v == 0)
        return (int)cnt <= c.cutoff ? 1 : 5;
    const int t = top_bit(v);
    *t_out = t;
    if ((int)cnt <= c.cutoff)
        return 2;
    return (t + c.D >= sg.lo) ? 3 : 4;
}

// per active segment: how many next-active, pending, small/done buckets and
// stats tiles its buckets produce
__global__ void k_plan_count(Ctx c, int it) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1;
    const int A = c.ctr->act_count[cur];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A; s += gridDim.x * blockDim.x) {
        const Seg sg = c.act[cur][s];
        int na = 0, np = 0, nf = 0, nt = 0, nm = 0;
        const uint32_t *h = c.act_hist[cur] + (int64_t)s * kBins;
        for (int d = 0; d < kBins; ++d) {
            int t = 0;
            const uint32_t cnt = h[d];
            const int kd = classify_bucket(c, cur, s, sg, d, cnt, &t);
            na += kd == 3 || kd == 5;
            np += kd == 4;
            nf += (kd == 1 || kd == 2);
            nt += (kd == 4) ? tiles_of(cnt, kTile) : 0;
            nm += kd == 6;
        }
        c.plan_cnt[s] = make_int4(na, np, nf, nt);
        c.plan_mid[s] = nm;
    }
}

// exclusive scan of the per-segment counts (one CTA), new counters
__global__ void __launch_bounds__(1024) k_plan_scan(Ctx c, int it) {
    griddep_wait();
    __shared__ int sh[40];
    __shared__ int s_a, s_p, s_f, s_t, s_m;
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int A = c.ctr->act_count[cur];
    if (threadIdx.x == 0) {
        s_a = 0;
        s_p = c.ctr->pend_count[nxt];  // after the segments plan_pending re-queued
        s_f = c.ctr->fin_count;
        s_t = c.ctr->stat_tiles[nxt];
        s_m = c.ctr->mid_count;
    }
    __syncthreads();
    constexpr int kPer = 8;
    for (int r0 = 0; r0 < A; r0 += blockDim.x * kPer) {
        const int s0 = r0 + threadIdx.x * kPer;
        int4 sum = make_int4(0, 0, 0, 0);
        int msum = 0;
        for (int u = 0; u < kPer && s0 + u < A; ++u) {
            const int4 v = c.plan_cnt[s0 + u];
            sum.x += v.x;
            sum.y += v.y;
            sum.z += v.z;
            sum.w += v.w;
            msum += c.plan_mid[s0 + u];
        }
        int ta, tp, tf, tt, tm;
        int pm = block_excl_scan(msum, &tm, sh);
        int pa = block_excl_scan(sum.x, &ta, sh);
        int pp = block_excl_scan(sum.y, &tp, sh);
        int pf = block_excl_scan(sum.z, &tf, sh);
        int pt = block_excl_scan(sum.w, &tt, sh);
        for (int u = 0; u < kPer && s0 + u < A; ++u) {
            const int4 v = c.plan_cnt[s0 + u];
            c.plan_cnt[s0 + u] = make_int4(s_a + pa, s_p + pp, s_f + pf, s_t + pt);
            const int vm = c.plan_mid[s0 + u];
            c.plan_mid[s0 + u] = s_m + pm;
            pm += vm;
            pa += v.x;
            pp += v.y;
            pf += v.z;
            pt += v.w;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            s_a += ta;
            s_p += tp;
            s_f += tf;
            s_t += tt;
            s_m += tm;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_a > c.seg_cap || s_p > c.seg_cap || s_f > c.fin_cap || c.ctr->brows[nxt] + s_t > c.row_cap ||
            s_m > c.mid_cap)
            set_status(c.status, kStOverflow);
        c.ctr->mid_count = (int32_t)min((int64_t)s_m, c.mid_cap);
        c.ctr->act_count[nxt] = (int32_t)min((int64_t)s_a, c.seg_cap);
        c.ctr->pend_count[nxt] = (int32_t)min((int64_t)s_p, c.seg_cap);
        if (s_p <= c.seg_cap)
            c.pend_tile_base[nxt][s_p] = s_t;
        c.ctr->stat_tiles[nxt] = s_t;
        c.ctr->fin_count = (int32_t)min((int64_t)s_f, c.fin_cap);
    }
}

__global__ void k_plan_write(Ctx c, int it) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int cur = it & 1, nxt = cur ^ 1;
    const int A = c.ctr->act_count[cur];
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < A; s += gridDim.x * blockDim.x) {
        const Seg sg = c.act[cur][s];
        const int4 o = c.plan_cnt[s];
        int64_t a = o.x, p = o.y, f = o.z, tb = o.w, m = c.plan_mid[s];
        const uint32_t *h = c.act_hist[cur] + (int64_t)s * kBins;
        int32_t bstart = sg.start;
        int32_t nrow = c.act_nrow_base[cur][s];
        for (int d = 0; d < kBins; ++d) {
            int t = 0;
            const uint32_t cnt = h[d];
            const int kd = classify_bucket(c, cur, s, sg, d, cnt, &t);
            if (kd == 6) {
                if (m < c.mid_cap)
                    c.mid[m] = Fin{bstart, (int32_t)cnt, sg.lo, (1 << 8) | ((sg.buf & 1) ^ 1)};
                ++m;
            } else if (kd == 1 || kd == 2) {
                if (f < c.fin_cap)
                    c.fin[f] = Fin{bstart, (int32_t)cnt, kd == 2 ? t + 1 : 0,
                                   ((kd == 2 ? 1 : 0) << 8) | ((sg.buf & 1) ^ 1)};
                ++f;
            } else if (kd == 3 || kd == 5) {
                if (a < c.seg_cap)
                    c.act[nxt][a] = Seg{bstart, (int32_t)cnt, (int16_t)max(sg.lo - c.D, 0), sg.lo,
                                        (sg.buf & 1) ^ 1, nrow, kd == 5 ? 1 : 0};
                ++a;
            } else if (kd == 4) {
                if (p < c.seg_cap) {
                    c.pend[nxt][p] = Seg{bstart, (int32_t)cnt, 0, (int16_t)(t + 1), (sg.buf & 1) ^ 1, 0, 0};
                    c.pend_tile_base[nxt][p] = (int32_t)tb;
                }
                tb += tiles_of(cnt, kTile);
                ++p;
            }
            bstart += (int32_t)cnt;
            nrow += tiles_of(cnt, kTile);
        }
    }
}

// ------------------------------------------------------------- launchers
template <typename KeyT>
static void launch_iter_t(const Ctx &c, int it, cudaStream_t s, int sms) {
    const int smem = PassLayout<KeyT>::kTotal;
    cudaFuncSetAttribute(k_pass<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int per_sm = PassLayout<KeyT>::kMinBlocks;
    const unsigned pblocks = (unsigned)max(1, min(sms * 4, (int)((c.seg_cap + 255) / 256)));
    launch_pdl(k_seg_stats<KeyT>, dim3(sms * 8), dim3(kTPB), 0, s, c, it);
    prof_mark("seg_stats", s);
    launch_pdl(k_plan_pending, dim3(1), dim3(1024), 0, s, c, it);
    prof_mark("plan", s);
    launch_pdl(k_tile_scan, dim3(sms * 4), dim3(kTPB), 0, s, c, it);
    launch_pdl(k_chunk_scan, dim3(sms * 4), dim3(kTPB), 0, s, c, it);
    prof_mark("scan", s);
    launch_pdl(k_pass<KeyT>, dim3(sms * per_sm), dim3(kTPB), smem, s, c, it);
    prof_mark("pass", s);
    launch_pdl(k_plan_count, dim3(pblocks), dim3(256), 0, s, c, it);
    launch_pdl(k_plan_scan, dim3(1), dim3(1024), 0, s, c, it);
    launch_pdl(k_plan_write, dim3(pblocks), dim3(256), 0, s, c, it);
    prof_mark("plan", s);
}

void launch_plan_pending(const Ctx &c, int it, cudaStream_t s) {
    launch_pdl(k_plan_pending, dim3(1), dim3(1024), 0, s, c, it);
    prof_mark("plan", s);
}

void launch_plan_scan(const Ctx &c, int it, cudaStream_t s) {
    launch_pdl(k_plan_scan, dim3(1), dim3(1024), 0, s, c, it);
}

void launch_plan_init(const Ctx &c, cudaStream_t s) {
    launch_pdl(k_plan_init, dim3(1), dim3(1024), 0, s, c);
    prof_mark("plan", s);
}

void launch_iteration(const Ctx &c, int it, cudaStream_t s, int sms) {
    if (c.D > kD) {  // windows of 5..8 bits: msd8.cu
        launch_iteration8(c, it, s, sms);
        return;
    }
    switch (c.key_bytes) {
    case 1: launch_iter_t<uint8_t>(c, it, s, sms); break;
    case 2: launch_iter_t<uint16_t>(c, it, s, sms); break;
    case 4: launch_iter_t<uint32_t>(c, it, s, sms); break;
    default: launch_iter_t<unsigned long long>(c, it, s, sms); break;
    }
}

int pass_tile() { return kTile; }
int stat_tile() { return kTile; }
int digit_bits() { return kD; }
int max_digit_bits() { return wide_digit_bits(); }
int scan_rows() { return kScanRows; }
int row_pad() { return kRowPad; }

}  // namespace pbit
