// finish.cu -- stages (c) and (d).
//
// (c) Small buckets are finished in registers or shared memory.  In the paper the recursion
//     runs every bucket down to M == 0 and merge() then appends the leaf
//     buckets (Sec. "Implementation in C++", Sec. 5.1); the paper itself notes
//     that MSD sorting spends too long on small chunks (Sec. "Differences
//     between Pbit and other algorithms sorting with bit key").  Here one warp
//     takes a bucket of at most kFinCap nodes, sorts it stably on its
//     remaining low bits by counting passes in registers (least significant
//     4-bit window first, skipping windows in which no key differs), and
//     writes its node ids to the final order buffer F.  Warps never wait for
//     each other, so a whole SM's worth of buckets is in flight at once.
// (d) The relink concatenates the sorted fragments: next[s[i]] = s[i+1],
//     next[s[n-1]] = -1, root = s[0] -- the effect of the merge() chain
//     (Sec. 5.1) done for all nodes at once.  For doubly-linked pools the
//     predecessor pointers are rebuilt in the same step (Sec. "Double-linked
//     lists sorting").
#include "pbit_internal.cuh"

namespace pbit {

constexpr int kFinCap = 512;             // largest bucket a warp finishes
constexpr int kFD = 4;
constexpr int kFBins = 1 << kFD;
constexpr int kFWarps = 4;               // warps per finish CTA

constexpr int kNetMax = 512;  // buckets up to this size are sorted by a register network

// Warp-wide bitonic sorting network over N values held in registers (lane l
// holds the values at positions l, 32 + l, ...): stage (k, s) compares the
// values at positions e and e ^ s and leaves the smaller at the lower
// position when e & k == 0 (the larger otherwise).  Exchanges across lanes
// go through shuffles, exchanges within a lane are register swaps.
template <typename C, int N>
__device__ __forceinline__ void warp_bitonic(C (&c)[N / 32], int lane) {
    constexpr int J = N / 32;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int s = k >> 1; s > 0; s >>= 1) {
            if (s >= 32) {
                const int js = s >> 5;
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    if ((j & js) == 0) {
                        const bool asc = ((j * 32) & k) == 0;  // k > 32 here: lane bits do not matter
                        const C x = c[j], y = c[j | js];
                        const C lo = x < y ? x : y, hi = x < y ? y : x;
                        c[j] = asc ? lo : hi;
                        c[j | js] = asc ? hi : lo;
                    }
                }
            } else {
#pragma unroll
                for (int j = 0; j < J; ++j) {
                    const C o = __shfl_xor_sync(kFull, c[j], s);
                    const bool keep_lo = ((lane & s) == 0) == (((j * 32 + lane) & k) == 0);
                    const C lo = c[j] < o ? c[j] : o, hi = c[j] < o ? o : c[j];
                    c[j] = keep_lo ? lo : hi;
                }
            }
        }
    }
}

// Sort a bucket of len <= N nodes with the network: the sort key of a node is
// (its varying key bits, its position in the bucket) -- unique, so the
// network's order is the stable order -- and after the sort each slot's
// position field names the node whose id goes there.  Returns false (nothing
// written) when the varying bits and the position do not fit in 64 bits.
template <typename KeyT, int N, typename C>
__device__ __forceinline__ void net_sort(const KeyT (&k)[N / 32], const int32_t *is, int32_t *dst, int len,
                                         int lv, int sbits, int lane) {
    constexpr int J = N / 32;
    constexpr int PB = N == 32 ? 5 : (N == 64 ? 6 : (N == 128 ? 7 : (N == 256 ? 8 : 9)));
    const unsigned long long smask = sbits >= 64 ? ~0ull : ((1ull << sbits) - 1ull);
    C c[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = j * 32 + lane;
        c[j] = e < len ? (C)(((((unsigned long long)k[j] >> lv) & smask) << PB) | (unsigned long long)e) : ~(C)0;
    }
    warp_bitonic<C, N>(c, lane);
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = j * 32 + lane;
        if (e < len)
            dst[e] = is[(int)(c[j] & (C)(N - 1))];
    }
}

template <typename KeyT, int N>
__device__ __forceinline__ bool net_bucket(const KeyT *ks, const int32_t *is, int32_t *dst, int len, int hi,
                                           int lane) {
    constexpr int J = N / 32;
    constexpr int PB = N == 32 ? 5 : (N == 64 ? 6 : (N == 128 ? 7 : (N == 256 ? 8 : 9)));
    using U = typename KeyWord<KeyT>::U;
    KeyT k[J];
    U a_and = ~(U)0, a_or = 0;
#pragma unroll
    for (int j = 0; j < J; ++j) {
        const int e = j * 32 + lane;
        k[j] = 0;
        if (e < len) {
            k[j] = ks[e];
            a_and &= (U)k[j];
            a_or |= (U)k[j];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a_and &= __shfl_xor_sync(kFull, a_and, o);
        a_or |= __shfl_xor_sync(kFull, a_or, o);
    }
    const unsigned long long vary =
        (unsigned long long)(a_and ^ a_or) & (hi >= 64 ? ~0ull : ((1ull << hi) - 1ull));
    if (!vary) {  // every key agrees on the remaining bits: list order stands
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int e = j * 32 + lane;
            if (e < len)
                dst[e] = is[e];
        }
        return true;
    }
    const int lv = __ffsll((long long)vary) - 1, hv = 63 - __clzll((long long)vary);
    const int sbits = hv - lv + 1;
    if (sbits + PB <= 32)
        net_sort<KeyT, N, uint32_t>(k, is, dst, len, lv, sbits, lane);
    else if (N <= 256 && sbits + PB <= 64)  // (measured: at 512 nodes the counting passes win)
        net_sort<KeyT, N, unsigned long long>(k, is, dst, len, lv, sbits, lane);
    else
        return false;
    return true;
}

template <typename KeyT>
__device__ __forceinline__ bool net_finish(const KeyT *ks, const int32_t *is, int32_t *dst, int len, int hi,
                                           int lane) {
    if (len <= 32)
        return net_bucket<KeyT, 32>(ks, is, dst, len, hi, lane);
    if (len <= 64)
        return net_bucket<KeyT, 64>(ks, is, dst, len, hi, lane);
    if (len <= 128)
        return net_bucket<KeyT, 128>(ks, is, dst, len, hi, lane);
    if (len <= 256)
        return net_bucket<KeyT, 256>(ks, is, dst, len, hi, lane);
    return net_bucket<KeyT, 512>(ks, is, dst, len, hi, lane);
}

// Keys whose varying bits are too wide for the network's sort key are sorted in the warp's two shared-memory buffers by counting
// passes: every window is two sweeps over its 32-element groups, count the
// digits (4 ballots per group), then rank each group again and scatter it to
// the other buffer at its digit's offset.
template <typename KeyT>
__device__ __forceinline__ void lsd_bucket(const KeyT *src_key, const int32_t *src_idx, int32_t *dst, int len,
                                           int hi, KeyT *sk0, int32_t *si0, int lane, unsigned lt) {
    const int ng = (len + 31) >> 5;  // 32-element groups (warp-uniform)
    int a = 0;                        // buffer holding the current order
    unsigned long long a_and = ~0ull, a_or = 0ull;
    for (int g = 0; g < ng; ++g) {
        const int pos = g * 32 + lane;
        if (pos < len) {
            const KeyT k = src_key[pos];
            sk0[pos] = k;
            si0[pos] = src_idx[pos];
            a_and &= (unsigned long long)k;
            a_or |= (unsigned long long)k;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a_and &= __shfl_xor_sync(kFull, a_and, o);
        a_or |= __shfl_xor_sync(kFull, a_or, o);
    }
    __syncwarp();
    const unsigned long long vary = (a_and ^ a_or) & (hi >= 64 ? ~0ull : ((1ull << hi) - 1ull));
    for (int wl = 0; wl < hi; wl += kFD) {
        const int width = min(kFD, hi - wl);
        const unsigned dmask = (1u << width) - 1u;
        if (((vary >> wl) & dmask) == 0)
            continue;  // every key agrees on this window
        const KeyT *ka = sk0 + a * kFinCap;
        const int32_t *ia = si0 + a * kFinCap;
        KeyT *kb = sk0 + (a ^ 1) * kFinCap;
        int32_t *ib = si0 + (a ^ 1) * kFinCap;
        // sweep 1: digit totals (lane d < 16 holds digit d)
        uint32_t tot = 0;
        for (int g = 0; g < ng; ++g) {
            const int pos = g * 32 + lane;
            const bool valid = pos < len;
            const unsigned dig = valid ? digit_of<KeyT>(ka[pos], wl, dmask) : 0u;
            unsigned mine = __ballot_sync(kFull, valid);
#pragma unroll
            for (int b = 0; b < kFD; ++b) {
                const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                mine &= ((lane >> b) & 1) ? bb : ~bb;
            }
            tot += __popc(mine);
        }
        uint32_t incl = lane < kFBins ? tot : 0u;
#pragma unroll
        for (int o = 1; o < kFBins; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o)
                incl += y;
        }
        uint32_t run = incl - (lane < kFBins ? tot : 0u);  // next free slot of digit lane
        // sweep 2: stable scatter, group by group
        for (int g = 0; g < ng; ++g) {
            const int pos = g * 32 + lane;
            const bool valid = pos < len;
            KeyT k = 0;
            int32_t x = 0;
            if (valid) {
                k = ka[pos];
                x = ia[pos];
            }
            const unsigned dig = valid ? digit_of<KeyT>(k, wl, dmask) : 0u;
            const unsigned vm = __ballot_sync(kFull, valid);
            unsigned peers = vm, mine = vm;
#pragma unroll
            for (int b = 0; b < kFD; ++b) {
                const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                peers &= ((dig >> b) & 1u) ? bb : ~bb;
                mine &= ((lane >> b) & 1) ? bb : ~bb;
            }
            const uint32_t p = __shfl_sync(kFull, run, (int)dig) + __popc(peers & lt);
            if (valid) {
                kb[p] = k;
                ib[p] = x;
            }
            run += __popc(mine);
        }
        __syncwarp();
        a ^= 1;
    }
    const int32_t *ia = si0 + a * kFinCap;
    for (int g = 0; g < ng; ++g) {
        const int pos = g * 32 + lane;
        if (pos < len)
            dst[pos] = ia[pos];
    }
    __syncwarp();
}

// Start copying a small bucket's keys and ids into staging buffers
// (asynchronous: they land while the previous bucket is being sorted).
template <typename KeyT>
__device__ __forceinline__ bool stage_bucket(const Ctx &c, const Fin &f, KeyT *pk, int32_t *pi, int lane) {
    if (sizeof(KeyT) < 4 || f.len <= 0 || f.len > kNetMax)
        return false;
    const int buf = f.mode_buf & 1;
    const KeyT *sk = reinterpret_cast<const KeyT *>(c.keyb[buf]) + f.start;
    const int32_t *si = c.idxb[buf] + f.start;
    for (int pos = lane; pos < f.len; pos += 32) {
        cp_async<(int)sizeof(KeyT) < 4 ? 4 : (int)sizeof(KeyT)>(pk + pos, sk + pos);
        cp_async<4>(pi + pos, si + pos);
    }
    cp_async_commit();
    return true;
}

// One warp per bucket, buckets taken in a software pipeline: while one small
// bucket is sorted, the next one's record is loaded and its data copied into
// the other staging buffer.
template <typename KeyT>
__global__ void __launch_bounds__(32 * kFWarps) k_finish(Ctx c) {
    griddep_wait();
    __shared__ __align__(16) KeyT s_key[kFWarps][2][kFinCap];
    __shared__ int32_t s_idx[kFWarps][2][kFinCap];
    if (*(volatile int32_t *)c.status)
        return;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const int nfin = c.ctr->fin_count;
    const int64_t gw = (int64_t)blockIdx.x * kFWarps + wid, nw = (int64_t)gridDim.x * kFWarps;
    KeyT *sk0 = &s_key[wid][0][0];
    int32_t *si0 = &s_idx[wid][0][0];
    long long my_elems = 0;
    Fin f = gw < nfin ? c.fin[gw] : Fin{0, 0, 0, 0};
    int sb = 0;  // staging buffer of f
    bool staged = stage_bucket<KeyT>(c, f, sk0, si0, lane);
    for (int64_t e = gw; e < nfin; e += nw) {
        const Fin fn = e + nw < nfin ? c.fin[e + nw] : Fin{0, 0, 0, 0};
        const int buf = f.mode_buf & 1;
        const int start = f.start, len = f.len;
        const int32_t *src_idx = c.idxb[buf] + start;
        const KeyT *src_key = reinterpret_cast<const KeyT *>(c.keyb[buf]) + start;
        int32_t *dst = c.F + start;
        bool done = false;
        if (len > kFinCap) {
            set_status(c.status, kStOverflow);
            done = true;
        } else if (len <= kNetMax) {
            my_elems += len;
            const bool nst = stage_bucket<KeyT>(c, fn, sk0 + (sb ^ 1) * kFinCap, si0 + (sb ^ 1) * kFinCap, lane);
            if (staged) {
                if (nst)
                    cp_async_wait_group1();
                else
                    cp_async_wait_all();
                __syncwarp();
            }
            done = net_finish<KeyT>(staged ? sk0 + sb * kFinCap : src_key, staged ? si0 + sb * kFinCap : src_idx,
                                    dst, len, f.hi, lane);
            __syncwarp();
            if (done) {
                staged = nst;
                sb ^= 1;
            } else {
                my_elems -= len;  // counted again below
            }
        }
        if (!done) {  // the counting path needs both buffers: nothing may be in flight into them
            my_elems += len;
            cp_async_wait_all();
            __syncwarp();
            lsd_bucket<KeyT>(src_key, src_idx, dst, len, f.hi, sk0, si0, lane, lt);
            staged = stage_bucket<KeyT>(c, fn, sk0, si0, lane);
            sb = 0;
        }
        f = fn;
    }
    cp_async_wait_all();  // no copy may be in flight when the warp exits
    // element count for the byte accounting (warp-uniform): one atomic per warp
    if (lane == 0 && my_elems)
        atomicAdd((unsigned long long *)&c.ctr->fin_sort_elems, (unsigned long long)my_elems);
}

// Mid-size buckets (more than the warp finish takes, at most kMidCap nodes,
// with at most kMidSpan varying key bits): one CTA per bucket.  The bulk copy
// engine loads the bucket into shared memory; the CTA sorts it there, least
// significant window first, on windows of up to 8 bits spread evenly over the
// bits that vary in it (one window for spans up to 8 bits, two up to 16),
// and writes the node ids to F.  A window is a stable counting split: each
// warp ranks its contiguous slice of the bucket group by group (32 elements:
// the lanes holding the same digit find each other through a per-warp table
// of peer masks and counts in shared memory, warp_rank_by_or), one thread per
// digit then turns the (warp, digit) counts into each warp's first slot
// (digit-major, warps in slice order: stable), and every element moves to its
// slot in the other buffer.  This replaces the further global passes, their planning and the
// small-bucket finish that such a bucket would otherwise go through.
constexpr int kMidTPB = 256;
constexpr int kMidWarps = kMidTPB / 32;
constexpr int kMidBits = 8;
constexpr int kMidBins = 1 << kMidBits;
static_assert(kMidBins == kMidTPB, "one thread per digit");

// Buffers for buckets of up to kCap nodes.  Keys of 4 and 8 bytes have two
// copies of the kernel: one sized for kMidSmallCap nodes (nearly every
// bucket the passes leave; its smaller buffers let more CTAs share an SM),
// which defers larger buckets to the one sized for kMidCap.
template <typename KeyT, int kCap>
struct MidLayout {
    static constexpr int kKeyBuf = kCap * (int)sizeof(KeyT) + 32;  // + room for the copy's 16-byte rounding
    static constexpr int kIdxBuf = kCap * 4 + 32;
    static constexpr int kBuf = ((kKeyBuf + kIdxBuf + 127) / 128) * 128;
    static constexpr int kTotal = 2 * kBuf;
    static constexpr int kItems = kCap / kMidTPB;  // groups of 32 per warp slice, at most
    static constexpr int kMinBlocks = kCap < kMidCap ? (sizeof(KeyT) == 8 ? 3 : 4) : (sizeof(KeyT) == 8 ? 2 : 3);
};

static_assert(kMidWarps * kMidBins * (int)sizeof(uint2) <= MidLayout<uint8_t, kMidCap>::kBuf &&
                  kMidWarps * kMidBins * (int)sizeof(uint2) <= MidLayout<uint32_t, kMidSmallCap>::kBuf,
              "the ranking table fits in a bucket buffer");

struct MidSmem {
    uint32_t wcnt[kMidWarps][kMidBins];  // per warp and digit: the warp's first slot
    int sh[40];
    unsigned long long s_and, s_or;
    int32_t next;  // bucket claimed next
    alignas(8) uint64_t bar;
};

// kDeferred: the buckets the smaller copy left (their indices in mid_defer).
template <typename KeyT, int kCap, bool kDeferred>
__global__ void __launch_bounds__(kMidTPB, (MidLayout<KeyT, kCap>::kMinBlocks)) k_finish_mid(Ctx c) {
    griddep_wait();
    extern __shared__ __align__(128) unsigned char msm[];
    __shared__ MidSmem S;
    using U = typename KeyWord<KeyT>::U;
    using L = MidLayout<KeyT, kCap>;
    constexpr int kMidItems = L::kItems;
    constexpr bool kDefers = kCap < kMidCap;  // larger buckets go to the kDeferred copy
    if (*(volatile int32_t *)c.status)
        return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt(), lane_bit = 1u << lane;
    const int nmid = kDeferred ? c.ctr->defer_count : c.ctr->mid_count;
    int32_t *claim_ctr = kDeferred ? &c.ctr->fin_ctr2.v : &c.ctr->fin_ctr.v;
    unsigned char *bufA = msm, *bufB = msm + L::kBuf;
    if (tid == 0) {
        mbar_init(&S.bar, 1);
        fence_mbar_init();
        S.next = atomicAdd(claim_ctr, 1);
    }
    __syncthreads();
    uint32_t phase = 0;
    long long my_elems = 0;
    for (int m = S.next; m < nmid; m = S.next) {
        const Fin f = c.mid[kDeferred ? c.mid_defer[m] : m];
        const int len = f.len, hi = f.hi;
        if (kDefers && len > kCap) {  // (CTA-uniform) for the larger copy
            __syncthreads();  // every thread has read m
            if (tid == 0) {
                c.mid_defer[atomicAdd(&c.ctr->defer_count, 1)] = m;
                S.next = atomicAdd(claim_ctr, 1);
            }
            __syncthreads();
            continue;
        }
        const bool ok_len = len > 0 && len <= kCap;
        constexpr int W = (int)sizeof(KeyT);
        int shk = 0, shi = 0;
        {
            const int64_t start = f.start;
            const int64_t k_lo = (start * W) & ~15ll, k_hi = ((start + len) * W + 15) & ~15ll;
            const int64_t i_lo = (start * 4) & ~15ll, i_hi = ((start + len) * 4 + 15) & ~15ll;
            shk = (int)((start * W - k_lo) / W);
            shi = (int)((start * 4 - i_lo) / 4);
            if (tid == 0 && ok_len) {
                const int buf = f.mode_buf & 1;
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&S.bar, (uint32_t)((k_hi - k_lo) + (i_hi - i_lo)));
                bulk_g2s(bufA, c.keyb[buf] + k_lo, (uint32_t)(k_hi - k_lo), &S.bar);
                bulk_g2s(bufA + L::kKeyBuf, reinterpret_cast<const unsigned char *>(c.idxb[buf]) + i_lo,
                         (uint32_t)(i_hi - i_lo), &S.bar);
            }
        }
        if (tid == 0) {
            S.s_and = ~0ull;
            S.s_or = 0ull;
        }
        const bool landed = (tid != 0) || !ok_len || mbar_wait_bounded(&S.bar, phase, 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            if (tid == 0)  // wait (bounded) for the copy in flight before leaving
                mbar_wait_bounded(&S.bar, phase, 1ll << 26);
            return;
        }
        if (tid == 0)  // every thread has read m: claim the next bucket
            S.next = atomicAdd(claim_ctr, 1);
        if (!ok_len) {  // (a planning error: cannot happen)
            set_status(c.status, kStOverflow);
            __syncthreads();
            continue;
        }
        phase ^= 1u;
        my_elems += len;
        // the bits that vary in the bucket
        KeyT *ka = reinterpret_cast<KeyT *>(bufA) + shk;
        int32_t *ia = reinterpret_cast<int32_t *>(bufA + L::kKeyBuf) + shi;
        KeyT *kb = reinterpret_cast<KeyT *>(bufB);
        int32_t *ib = reinterpret_cast<int32_t *>(bufB + L::kKeyBuf);
        {
            U a_and = ~(U)0, a_or = 0;
            for (int e = tid; e < len; e += kMidTPB) {
                const U k = (U)ka[e];
                a_and &= k;
                a_or |= k;
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a_and &= __shfl_xor_sync(kFull, a_and, o);
                a_or |= __shfl_xor_sync(kFull, a_or, o);
            }
            if (lane == 0) {
                atomicAnd(&S.s_and, (unsigned long long)a_and);
                atomicOr(&S.s_or, (unsigned long long)a_or);
            }
        }
        __syncthreads();
        const unsigned long long vary = (S.s_and ^ S.s_or) & (hi >= 64 ? ~0ull : ((1ull << hi) - 1ull));
        const int32_t *res = ia;  // node ids in final order
        if (vary) {
            const int lv = __ffsll((long long)vary) - 1, hv = 63 - __clzll((long long)vary);
            const int span = hv - lv + 1;
            const int nwin = (span + kMidBits - 1) / kMidBits;
            const int width = (span + nwin - 1) / nwin;
            const int nitems = (len + kMidTPB - 1) / kMidTPB;  // groups per warp slice
            const int s0 = wid * 32 * nitems;
            unsigned char *dst_buf = bufB, *src_buf = bufA;
            for (int w = 0; w < nwin; ++w) {
                const int wl = lv + w * width;
                const unsigned dmask = (1u << min(width, hv + 1 - wl)) - 1u;
                const bool last = w == nwin - 1;
                // the ranking's {peer mask, count} table lives in the window's
                // destination buffer, which is written only after the ranking
                uint2 *tab = reinterpret_cast<uint2 *>(dst_buf);
#pragma unroll
                for (int e = tid; e < kMidWarps * kMidBins / 2; e += kMidTPB)
                    reinterpret_cast<uint4 *>(tab)[e] = make_uint4(0u, 0u, 0u, 0u);
                __syncthreads();
                uint32_t rnk[kMidItems];
#pragma unroll
                for (int i = 0; i < kMidItems; ++i) {
                    rnk[i] = 0;
                    if (i < nitems) {  // warp-uniform
                        const int pos = s0 + i * 32 + lane;
                        const bool valid = pos < len;
                        const unsigned dig = valid ? digit_of<KeyT>(ka[pos], wl, dmask) : 0u;
                        rnk[i] = warp_rank_by_or(tab + wid * kMidBins, dig, valid, lane_bit, lt);
                    }
                }
                __syncthreads();
                {  // each warp's first slot per digit (thread tid = digit)
                    uint32_t cw[kMidWarps];
                    uint32_t tot = 0;
#pragma unroll
                    for (int x = 0; x < kMidWarps; ++x) {
                        cw[x] = tab[x * kMidBins + tid].y;
                        tot += cw[x];
                    }
                    int ttot;
                    uint32_t run = (uint32_t)block_excl_scan_1bar((int)tot, &ttot, S.sh);
#pragma unroll
                    for (int x = 0; x < kMidWarps; ++x) {
                        S.wcnt[x][tid] = run;
                        run += cw[x];
                    }
                }
                __syncthreads();  // (the table is read: the scatter may overwrite it)
#pragma unroll
                for (int i = 0; i < kMidItems; ++i) {
                    if (i < nitems) {
                        const int pos = s0 + i * 32 + lane;
                        if (pos < len) {
                            const KeyT k = ka[pos];
                            const uint32_t p = S.wcnt[wid][digit_of<KeyT>(k, wl, dmask)] + rnk[i];
                            if (p < (uint32_t)len) {
                                if (!last)
                                    kb[p] = k;
                                ib[p] = ia[pos];
                            } else {
                                set_status(c.status, kStOverflow);  // (inconsistent counts: cannot happen)
                            }
                        }
                    }
                }
                __syncthreads();  // the scatter is complete before the next window ranks
                res = ib;
                KeyT *tk = ka;  // the other buffer is the next window's source
                ka = kb;
                kb = tk;
                int32_t *ti = ia;
                ia = ib;
                ib = ti;
                unsigned char *tb = src_buf;
                src_buf = dst_buf;
                dst_buf = tb;
            }
        }
        int32_t *dst = c.F + f.start;
        for (int e = tid; e < len; e += kMidTPB)
            dst[e] = res[e];
        __syncthreads();  // the buffers and counters are reused by the next bucket
    }
    if (tid == 0 && my_elems)  // every thread counted the same buckets
        atomicAdd((unsigned long long *)&c.ctr->fin_sort_elems, (unsigned long long)my_elems);
}

// Stage (d): relink, direct form: one thread per sorted position writes
// next[s[q]] = s[q+1] straight into the pool (scattered 4-byte stores).  Used
// when the lists live in different pools (the request server).
__global__ void k_relink(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int32_t nv = c.ctr->n_virt;
    const int L = c.num_lists;
    const bool doubly = (c.flags & PBIT_DOUBLY) != 0;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nv; q += (int64_t)gridDim.x * blockDim.x) {
        const int lst = upper_index(c.out_base, L, (int32_t)q);
        const ListDesc &d = c.desc[lst];
        const int32_t p = c.F[q];
        const int32_t loc = p - d.out_base;
        const int64_t end = (int64_t)d.out_base + d.n;
        if (loc < 0 || loc >= d.n || q >= end) {
            set_status(c.status, kStOverflow);
            continue;
        }
        int32_t succ = -1;
        if (q + 1 < end) {
            const int32_t ls = c.F[q + 1] - d.out_base;
            if (ls < 0 || ls >= d.n) {
                set_status(c.status, kStOverflow);
                continue;
            }
            succ = d.id_base + ls;
            if (doubly)
                *(int32_t *)((unsigned char *)d.prev + (int64_t)(d.id_base + ls) * d.prev_stride) = d.id_base + loc;
        }
        *(int32_t *)((unsigned char *)d.next + (int64_t)(d.id_base + loc) * d.next_stride) = succ;
        if (q == d.out_base) {
            c.new_roots[lst] = d.id_base + loc;
            if (doubly)
                *(int32_t *)((unsigned char *)d.prev + (int64_t)(d.id_base + loc) * d.prev_stride) = -1;
        }
    }
}

// Stage (d), blocked form for lists sharing one pool.  Scattered 4-byte
// stores into a pool much larger than L2 each cost a read-modify-write of a
// DRAM granule; instead the (node, successor) pairs are first bucketed by
// the node's pool block (2^rb nodes, a window of a few MB), then applied
// block after block, so the stores of one window merge in L2 and leave as
// full lines.  The two order buffers idxb[0], idxb[1] (free by now) hold the
// pairs; bucket b owns slots [b << rb, (b << rb) + count).  Each tile first
// groups its pairs by bucket in shared memory so that its writes to a
// bucket are one contiguous run.
constexpr int kRelTPB = 256;
constexpr int kRelItems = 8;  // (16 took 108 registers: 2 CTAs per SM, latency-bound)
constexpr int kRelTile = kRelTPB * kRelItems;
constexpr int kMaxRelBuckets = 512;
constexpr int kCursorStride = 32;  // one 128-byte line per bucket cursor

struct RelSmem {
    int32_t cnt[kMaxRelBuckets];
    int32_t loc[kMaxRelBuckets + 1];
    int32_t base[kMaxRelBuckets];
    int32_t sv[kRelTile];
    int32_t ss[kRelTile];
    uint16_t sb[kRelTile];
    int32_t nt[2];                       // the tiles in the two stages (>= tiles: none)
    alignas(16) int32_t fstage[2][kRelTile + 8];  // F[q0 .. q0 + kRelTile] of each stage (+ the next)
    alignas(8) uint64_t bar[2];
};

// Issue the bulk copy of the order entries F[q0, q0 + kRelTile] that tile g
// uses (its own and the successor of its last one; fewer at the end of the
// order) into stage st (one thread).  q0 is a multiple of 4, so the copy
// starts 16-byte aligned; rounding its length up to 16 bytes stays inside
// F's 64 bytes of slack.
__device__ __forceinline__ void relink_issue(const Ctx &c, int g, int st, int32_t nv, RelSmem &S) {
    const int64_t q0 = (int64_t)g * kRelTile;
    const int64_t cnt = min((int64_t)kRelTile + 1, (int64_t)nv - q0);
    const uint32_t bytes = (uint32_t)(((cnt + 3) & ~3ll) * 4);
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&S.bar[st], bytes);
    bulk_g2s(S.fstage[st], c.F + q0, bytes, &S.bar[st]);
}

// Tiles of kRelTile sorted positions are claimed from a counter one step
// ahead; the bulk copy engine brings each tile's order entries (and the one
// after it) into shared memory while the previous tile is bucketed.
// kOne: a single list (its descriptor is read once); kDoubly: prev[] too.
template <bool kOne, bool kDoubly>
__global__ void __launch_bounds__(kRelTPB, 4) k_relink_part(Ctx c, int rb) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char rel_smem[];
    RelSmem &S = *reinterpret_cast<RelSmem *>(rel_smem);
    __shared__ int sh[40];
    if (*(volatile int32_t *)c.status)
        return;
    const int32_t nv = c.ctr->n_virt;
    const int L = c.num_lists;
    const int nb = (int)((c.ncap + (1ll << rb) - 1) >> rb);
    const int T = (int)((nv + kRelTile - 1) / kRelTile);
    ListDesc d1{};
    if constexpr (kOne)
        d1 = c.desc[0];
    int32_t *tv = c.idxb[0], *ts = c.idxb[1];
    int claim = 0;  // thread 0: the tile claimed for the next issue
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
        const int g0 = atomicAdd(&c.ctr->rel_ctr.v, 1);
        S.nt[0] = g0;
        if (g0 < T) {
            relink_issue(c, g0, 0, nv, S);
            claim = atomicAdd(&c.ctr->rel_ctr.v, 1);
        }
    }
    __syncthreads();
    uint32_t phases = 0;
    int st = 0;
    for (int g = S.nt[0]; g < T;) {
        if (threadIdx.x == 0) {  // the next tile into the other stage, claim the one after
            S.nt[st ^ 1] = claim;
            if (claim < T) {
                relink_issue(c, claim, st ^ 1, nv, S);
                claim = atomicAdd(&c.ctr->rel_ctr.v, 1);
            }
        }
        for (int b = threadIdx.x; b < nb; b += kRelTPB)
            S.cnt[b] = 0;
        const bool landed = threadIdx.x != 0 || mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
        if (!__syncthreads_and(landed)) {
            set_status(c.status, PBIT_ETIMEOUT);
            if (threadIdx.x == 0) {  // wait (bounded) for the copies still in flight before leaving
                mbar_wait_bounded(&S.bar[st], (phases >> st) & 1u, 1ll << 26);
                if (S.nt[st ^ 1] < T)
                    mbar_wait_bounded(&S.bar[st ^ 1], (phases >> (st ^ 1)) & 1u, 1ll << 26);
            }
            return;
        }
        phases ^= 1u << st;
        const int64_t q0 = (int64_t)g * kRelTile;
        const int32_t *fs = S.fstage[st];
        int32_t vv[kRelItems], ss[kRelItems], rk[kRelItems];
#pragma unroll
        for (int i = 0; i < kRelItems; ++i) {
            const int e = i * kRelTPB + threadIdx.x;
            const int64_t q = q0 + e;
            vv[i] = -1;
            ss[i] = -1;
            if (q < nv) {
                const int lst = kOne ? 0 : upper_index(c.out_base, L, (int32_t)q);
                const ListDesc &d = kOne ? d1 : c.desc[lst];
                const int32_t loc = fs[e] - d.out_base;
                const int64_t end = (int64_t)d.out_base + d.n;
                int32_t succ = -1;
                bool bad = (uint32_t)loc >= (uint32_t)d.n;
                if (q + 1 < end) {
                    const int32_t ls = fs[e + 1] - d.out_base;
                    bad |= (uint32_t)ls >= (uint32_t)d.n;
                    succ = d.id_base + ls;
                    if (kDoubly && !bad)
                        *(int32_t *)((unsigned char *)d.prev + (int64_t)succ * d.prev_stride) = d.id_base + loc;
                }
                if (bad) {
                    set_status(c.status, kStOverflow);
                } else {
                    vv[i] = d.id_base + loc;
                    ss[i] = succ;
                    if (q == d.out_base) {
                        c.new_roots[lst] = vv[i];
                        if (kDoubly)
                            *(int32_t *)((unsigned char *)d.prev + (int64_t)vv[i] * d.prev_stride) = -1;
                    }
                }
            }
        }
#pragma unroll
        for (int i = 0; i < kRelItems; ++i)
            rk[i] = vv[i] >= 0 ? atomicAdd(&S.cnt[vv[i] >> rb], 1) : 0;
        __syncthreads();
        // local bucket offsets (exclusive scan of the counts) and the global
        // reservation of each bucket's run
        {
            const int per = (nb + kRelTPB - 1) / kRelTPB;  // buckets per thread (<= 2)
            int sum = 0;
            for (int j = 0; j < per; ++j) {
                const int b = threadIdx.x * per + j;
                sum += b < nb ? S.cnt[b] : 0;
            }
            int tot;
            int ex = block_excl_scan(sum, &tot, sh);
            for (int j = 0; j < per; ++j) {
                const int b = threadIdx.x * per + j;
                if (b < nb) {
                    S.loc[b] = ex;
                    ex += S.cnt[b];
                    S.base[b] = S.cnt[b] ? atomicAdd(&c.rel_cursor[b * kCursorStride], S.cnt[b]) : 0;
                }
            }
            if (threadIdx.x == 0)
                S.loc[nb] = tot;
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kRelItems; ++i) {
            if (vv[i] >= 0) {
                const int b = vv[i] >> rb;
                const int p = S.loc[b] + rk[i];
                S.sv[p] = vv[i];
                S.ss[p] = ss[i];
                S.sb[p] = (uint16_t)b;
            }
        }
        __syncthreads();
        const int total = S.loc[nb];
        for (int j = threadIdx.x; j < total; j += kRelTPB) {
            const int b = S.sb[j];
            const int64_t slot = ((int64_t)b << rb) + S.base[b] + (j - S.loc[b]);
            tv[slot] = S.sv[j];
            ts[slot] = S.ss[j];
        }
        __syncthreads();  // staging and counts are reused by the next tile
        g = S.nt[st ^ 1];
        st ^= 1;
    }
}

// Apply the pairs of node block b0: one launch per window so the stores in
// flight stay inside a few MB of next[].
__global__ void k_relink_apply(Ctx c, int rb, int b0) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int32_t *tv = c.idxb[0], *ts = c.idxb[1];
    unsigned char *next = reinterpret_cast<unsigned char *>(c.desc[0].next);
    const int64_t stride = c.desc[0].next_stride;
    const int32_t cnt = c.rel_cursor[b0 * kCursorStride];
    const int64_t base = (int64_t)b0 << rb;  // a multiple of 2^20: 16-byte aligned runs
    // 16 pairs per thread (four 16-byte loads per array), all loads issued
    // before the stores: the kernel waits on its loads, so keep many in flight
    const int64_t n16 = cnt >> 4;
    const int4 *tv4 = reinterpret_cast<const int4 *>(tv + base), *ts4 = reinterpret_cast<const int4 *>(ts + base);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x) {
        int4 v[4], s[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            v[u] = tv4[4 * i + u];
            s[u] = ts4[4 * i + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            *(int32_t *)(next + (int64_t)v[u].x * stride) = s[u].x;
            *(int32_t *)(next + (int64_t)v[u].y * stride) = s[u].y;
            *(int32_t *)(next + (int64_t)v[u].z * stride) = s[u].z;
            *(int32_t *)(next + (int64_t)v[u].w * stride) = s[u].w;
        }
    }
    for (int64_t i = 16 * n16 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt;
         i += (int64_t)gridDim.x * blockDim.x)
        *(int32_t *)(next + (int64_t)tv[base + i] * stride) = ts[base + i];
}

__global__ void k_empty_roots(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.num_lists; i += gridDim.x * blockDim.x)
        if (c.desc[i].n == 0)
            c.new_roots[i] = -1;
}

// Every node must have been placed by a pass or by the finish: any segment
// still live after the last pass means the pass budget was too small.
__global__ void k_check_done(Ctx c, int iters) {
    griddep_wait();
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int p = iters & 1;
        if (c.ctr->act_count[p] != 0 || c.ctr->pend_count[p] != 0)
            set_status(c.status, kStOverflow);
    }
}

template <typename KeyT>
static void launch_finish_t(const Ctx &c, cudaStream_t s, int sms) {
    {
        using LB = MidLayout<KeyT, kMidCap>;
        using LS = MidLayout<KeyT, kMidSmallCap>;
        static_assert(3 * (MidLayout<uint32_t, kMidCap>::kTotal + (int)sizeof(MidSmem) + 1024) <= 228 * 1024 &&
                          4 * (MidLayout<uint32_t, kMidSmallCap>::kTotal + (int)sizeof(MidSmem) + 1024) <= 228 * 1024,
                      "3 (4) CTAs per SM");
        static_assert(2 * (MidLayout<unsigned long long, kMidCap>::kTotal + (int)sizeof(MidSmem) + 1024) <= 228 * 1024 &&
                          3 * (MidLayout<unsigned long long, kMidSmallCap>::kTotal + (int)sizeof(MidSmem) + 1024) <=
                              228 * 1024,
                      "2 (3) CTAs per SM");
        // (registers and shared memory allow kMinBlocks CTAs per SM)
        if constexpr (sizeof(KeyT) >= 4) {
            cudaFuncSetAttribute(k_finish_mid<KeyT, kMidSmallCap, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, LS::kTotal);
            launch_pdl(k_finish_mid<KeyT, kMidSmallCap, false>, dim3((unsigned)(sms * LS::kMinBlocks)), dim3(kMidTPB),
                       LS::kTotal, s, c);
            cudaFuncSetAttribute(k_finish_mid<KeyT, kMidCap, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 LB::kTotal);
            launch_pdl(k_finish_mid<KeyT, kMidCap, true>, dim3((unsigned)(sms * LB::kMinBlocks)), dim3(kMidTPB),
                       LB::kTotal, s, c);
        } else {
            cudaFuncSetAttribute(k_finish_mid<KeyT, kMidCap, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 LB::kTotal);
            launch_pdl(k_finish_mid<KeyT, kMidCap, false>, dim3((unsigned)(sms * LB::kMinBlocks)), dim3(kMidTPB),
                       LB::kTotal, s, c);
        }
    }
    const int smem = (int)(kFWarps * 2 * kFinCap * (sizeof(KeyT) + 4));
    const int per_sm = max(1, min(16, (200 * 1024) / smem));
    launch_pdl(k_finish<KeyT>, dim3((unsigned)(sms * per_sm)), dim3(32 * kFWarps), 0, s, c);
    prof_mark("finish", s);
}

void launch_finish_relink(const Ctx &c, cudaStream_t s, int sms) {
    switch (c.key_bytes) {
    case 1: launch_finish_t<uint8_t>(c, s, sms); break;
    case 2: launch_finish_t<uint16_t>(c, s, sms); break;
    case 4: launch_finish_t<uint32_t>(c, s, sms); break;
    default: launch_finish_t<unsigned long long>(c, s, sms); break;
    }
    if (relink_blocked(c)) {
        const int rb = relink_bucket_bits(c);
        const int64_t pblocks = min((int64_t)sms * 4, max((int64_t)1, (c.ncap + kRelTile - 1) / kRelTile));
        const int smem = (int)sizeof(RelSmem);
        const bool one = c.num_lists == 1, doubly = (c.flags & PBIT_DOUBLY) != 0;
        auto part = one ? (doubly ? k_relink_part<true, true> : k_relink_part<true, false>)
                        : (doubly ? k_relink_part<false, true> : k_relink_part<false, false>);
        cudaFuncSetAttribute(part, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        launch_pdl(part, dim3((unsigned)pblocks), dim3(kRelTPB), smem, s, c, rb);
        const int64_t ablocks = min((int64_t)sms * 8, (int64_t)(((1ll << rb) / 16 + 255) / 256));
        const int nb = (int)((c.ncap + (1ll << rb) - 1) >> rb);
        for (int b = 0; b < nb; ++b) {
            launch_pdl(k_relink_apply, dim3((unsigned)ablocks), dim3(256), 0, s, c, rb, b);
            if (g_relink_hook.fn)
                g_relink_hook.fn(g_relink_hook.arg, (int64_t)b << rb, min(((int64_t)b + 1) << rb, c.ncap), s);
        }
    } else {
        const int64_t blocks = min((int64_t)sms * 16, max((int64_t)1, (c.ncap + 255) / 256));
        launch_pdl(k_relink, dim3((unsigned)blocks), dim3(256), 0, s, c);
    }
    prof_mark("relink", s);
    launch_pdl(k_empty_roots, dim3(max(1, min(sms, (c.num_lists + 255) / 256))), dim3(256), 0, s, c);
    prof_mark("relink", s);
}

void launch_relink_direct(const Ctx &c, cudaStream_t s, int sms) {
    const int64_t blocks = min((int64_t)sms * 16, max((int64_t)1, (c.ncap + 255) / 256));
    launch_pdl(k_relink, dim3((unsigned)blocks), dim3(256), 0, s, c);
    prof_mark("relink", s);
    launch_pdl(k_empty_roots, dim3(max(1, min(sms, (c.num_lists + 255) / 256))), dim3(256), 0, s, c);
    prof_mark("relink", s);
}

void launch_check_done(const Ctx &c, int iters, cudaStream_t s) {
    launch_pdl(k_check_done, dim3(1), dim3(32), 0, s, c, iters);
    prof_mark("plan", s);
}

int finish_capacity() { return kFinCap; }

// Blocked relink when every list shares one pool (not the request server's
// per-request pools): window of 2^rb nodes = at most 16 MB of next[].
bool relink_blocked(const Ctx &c) { return c.shared_pool != 0; }
int relink_bucket_bits(const Ctx &c) {
    int rb = c.desc_next_stride <= 4 ? 22 : (c.desc_next_stride <= 8 ? 21 : 20);
    while (rb < 31 && ((c.ncap + (1ll << rb) - 1) >> rb) > kMaxRelBuckets)
        ++rb;
    return rb;
}
int relink_max_buckets() { return kMaxRelBuckets * kCursorStride; }

}  // namespace pbit
