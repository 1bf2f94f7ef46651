// small.cu -- short lists in one kernel: one CTA sorts a whole list of at most
// kSmallList nodes in shared memory.
//
// The general path spends about a hundred launches on a list whatever its
// length; for a list of a few thousand nodes that fixed cost is the whole
// latency.  Here one CTA per list does all four steps of the method:
//   1. load next[] and the sort keys of the list's pool range into shared
//      memory, checking every successor index;
//   2. rank by pointer jumping (Wyllie) in shared memory: dist(v) = nodes
//      from v to the end; the root must reach NULL after exactly n nodes
//      (otherwise: a cycle, a short list or a node not on the list);
//   3. place every node at rank n - dist(v) (list order) and sort stably by
//      least significant windows of up to 4 bits over the bits that vary
//      (block-wide ballot ranking, as in the finish kernels);
//   4. write the sorted order to F; the direct relink kernel then applies
//      next[s[i]] = s[i+1] (and prev[] for doubly-linked pools) and the new
//      heads -- only if every list of the call was valid, so a call that
//      fails leaves every pool untouched.
#include "pbit_internal.cuh"

namespace pbit {

constexpr int kSmallTPB = 512;
constexpr int kSmallWarps = kSmallTPB / 32;
constexpr int kSmallPer = kSmallList / kSmallTPB;  // nodes per thread
static_assert(kSmallPer * kSmallTPB == kSmallList, "threads cover the list");
constexpr int kSmallD = 4;                          // LSD window width

template <typename KeyT>
struct SmallLayout {
    static constexpr int kKeys = 2 * kSmallList * (int)sizeof(KeyT);  // two key buffers
    static constexpr int kIds = 2 * kSmallList * 4;                   // two id buffers
    static constexpr int kRank = 2 * kSmallList * 4;                  // succ + dist
    static constexpr int kTotal = kKeys + kIds + kRank;
};

template <typename KeyT>
__global__ void __launch_bounds__(kSmallTPB) k_small_sort(Ctx c) {
    griddep_wait();
    extern __shared__ __align__(16) unsigned char ssm[];
    using U = typename KeyWord<KeyT>::U;
    using L = SmallLayout<KeyT>;
    __shared__ uint32_t s_cnt[kSmallWarps][32];
    __shared__ U s_and[kSmallWarps], s_or[kSmallWarps];
    KeyT *skey = reinterpret_cast<KeyT *>(ssm);                                 // [2][kSmallList]
    int32_t *sidx = reinterpret_cast<int32_t *>(ssm + L::kKeys);                // [2][kSmallList]
    int32_t *succ = reinterpret_cast<int32_t *>(ssm + L::kKeys + L::kIds);      // [kSmallList]
    int32_t *dist = succ + kSmallList;                                          // [kSmallList]
    if (*(volatile int32_t *)c.status)
        return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt();
    for (int li = blockIdx.x; li < c.num_lists; li += gridDim.x) {
        const ListDesc d = c.desc[li];
        const int n = d.n;
        if (n <= 0)
            continue;
        if (n > kSmallList || d.root < 0 || d.root >= n) {
            if (tid == 0)
                set_status(c.status, n > kSmallList ? kStOverflow : PBIT_EBADLIST);
            continue;
        }
        // 1. load
        const unsigned char *nb = reinterpret_cast<const unsigned char *>(d.next);
        bool bad = false;
        for (int v = tid; v < n; v += kSmallTPB) {
            const int64_t node = (int64_t)d.id_base + v;
            const int32_t raw = *reinterpret_cast<const int32_t *>(nb + node * d.next_stride);
            int32_t s = -1;
            if (raw != -1) {
                s = raw - d.id_base;
                if (raw < d.id_base || s >= n) {
                    bad = true;
                    s = -1;
                }
            }
            succ[v] = s;
            dist[v] = 1;
            skey[v] = sort_key<KeyT>(load_key_raw<KeyT>(d.key + node * d.key_stride), c.flags, c.M);
        }
        if (__syncthreads_or(bad)) {
            if (tid == 0)
                set_status(c.status, PBIT_EBADLIST);
            continue;
        }
        // 2. rank: pointer jumping, reads of a round before its writes
        for (int span = 1; span < n; span <<= 1) {
            int32_t ns[kSmallPer], nd[kSmallPer];
#pragma unroll
            for (int q = 0; q < kSmallPer; ++q) {
                const int v = q * kSmallTPB + tid;
                ns[q] = -1;
                nd[q] = 0;
                if (v < n) {
                    const int32_t s = succ[v];
                    ns[q] = s;
                    nd[q] = dist[v];
                    if (s >= 0) {
                        nd[q] += dist[s];
                        ns[q] = succ[s];
                    }
                }
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < kSmallPer; ++q) {
                const int v = q * kSmallTPB + tid;
                if (v < n) {
                    succ[v] = ns[q];
                    dist[v] = nd[q];
                }
            }
            __syncthreads();
        }
        // the root must reach NULL after exactly n nodes: otherwise a cycle,
        // or nodes that are not on the list
        if (__syncthreads_or(tid == 0 && (succ[d.root] != -1 || dist[d.root] != n))) {
            if (tid == 0)
                set_status(c.status, PBIT_EBADLIST);
            continue;
        }
        // 3. list order into buffer 1, then the sort
        U a_and = ~(U)0, a_or = 0;
        for (int v = tid; v < n; v += kSmallTPB) {
            const int r = n - dist[v];
            const KeyT k = skey[v];
            skey[kSmallList + r] = k;
            sidx[kSmallList + r] = v;
            a_and &= (U)k;
            a_or |= (U)k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a_and &= __shfl_xor_sync(kFull, a_and, o);
            a_or |= __shfl_xor_sync(kFull, a_or, o);
        }
        if (lane == 0) {
            s_and[wid] = a_and;
            s_or[wid] = a_or;
        }
        __syncthreads();
        a_and = ~(U)0;
        a_or = 0;
#pragma unroll
        for (int w = 0; w < kSmallWarps; ++w) {
            a_and &= s_and[w];
            a_or |= s_or[w];
        }
        const unsigned long long vary = (unsigned long long)(a_and ^ a_or);
        // each warp owns a contiguous slice of whole 32-element groups
        const int ngr = (n + 31) >> 5;
        const int gpw = (ngr + kSmallWarps - 1) / kSmallWarps;
        const int s0 = min(n, wid * gpw * 32), s1 = min(n, (wid + 1) * gpw * 32);
        int a = 1;
        if (vary) {
            const int lv = __ffsll((long long)vary) - 1, hv = 63 - __clzll((long long)vary);
            const int spanb = hv - lv + 1;
            const int nwin = (spanb + kSmallD - 1) / kSmallD;
            const int width0 = (spanb + nwin - 1) / nwin;
            int wl = lv;
            while (wl <= hv && (vary >> wl) != 0) {  // block-uniform
                wl += __ffsll((long long)(vary >> wl)) - 1;
                const int width = min(width0, hv + 1 - wl);
                const unsigned dmask = (1u << width) - 1u;
                const KeyT *ka = skey + a * kSmallList;
                const int32_t *ia = sidx + a * kSmallList;
                KeyT *kb = skey + (a ^ 1) * kSmallList;
                int32_t *ib = sidx + (a ^ 1) * kSmallList;
                // counts: lane d of each warp counts digit d in the warp's slice
                uint32_t tot = 0;
                for (int p0 = s0; p0 < s1; p0 += 32) {
                    const int pos = p0 + lane;
                    const bool valid = pos < s1;
                    const unsigned dig = valid ? digit_of<KeyT>(ka[pos], wl, dmask) : 0u;
                    unsigned mine = __ballot_sync(kFull, valid);
#pragma unroll
                    for (int bit = 0; bit < kSmallD; ++bit) {
                        if (bit < width) {
                            const unsigned bb = __ballot_sync(kFull, (dig >> bit) & 1u);
                            mine &= ((lane >> bit) & 1) ? bb : ~bb;
                        }
                    }
                    tot += (uint32_t)__popc(mine);
                }
                s_cnt[wid][lane] = (unsigned)lane <= dmask ? tot : 0u;  // lanes past the digits alias
                __syncthreads();
                if (wid == 0) {  // slots: digit-major, warps in slice order
                    uint32_t dtot = 0;
#pragma unroll
                    for (int w = 0; w < kSmallWarps; ++w)
                        dtot += s_cnt[w][lane];
                    uint32_t incl = dtot;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(kFull, incl, o);
                        if (lane >= o)
                            incl += y;
                    }
                    uint32_t run = incl - dtot;
#pragma unroll
                    for (int w = 0; w < kSmallWarps; ++w) {
                        const uint32_t x = s_cnt[w][lane];
                        s_cnt[w][lane] = run;
                        run += x;
                    }
                }
                __syncthreads();
                // stable scatter of the warp's slice
                uint32_t run = s_cnt[wid][lane];
                for (int p0 = s0; p0 < s1; p0 += 32) {
                    const int pos = p0 + lane;
                    const bool valid = pos < s1;
                    KeyT k = 0;
                    int32_t x = 0;
                    if (valid) {
                        k = ka[pos];
                        x = ia[pos];
                    }
                    const unsigned dig = valid ? digit_of<KeyT>(k, wl, dmask) : 0u;
                    unsigned peers = __ballot_sync(kFull, valid), mine = peers;
#pragma unroll
                    for (int bit = 0; bit < kSmallD; ++bit) {
                        if (bit < width) {
                            const unsigned bb = __ballot_sync(kFull, (dig >> bit) & 1u);
                            peers &= ((dig >> bit) & 1u) ? bb : ~bb;
                            mine &= ((lane >> bit) & 1) ? bb : ~bb;
                        }
                    }
                    const uint32_t p = __shfl_sync(kFull, run, (int)dig) + (uint32_t)__popc(peers & lt);
                    if (valid) {
                        kb[p] = k;
                        ib[p] = x;
                    }
                    run += (uint32_t)__popc(mine);
                }
                __syncthreads();
                a ^= 1;
                wl += width;
            }
        }
        // 4. the sorted order (virtual positions), for the relink
        const int32_t *s = sidx + a * kSmallList;
        for (int i = tid; i < n; i += kSmallTPB)
            c.F[(int64_t)d.out_base + i] = d.out_base + s[i];
        __syncthreads();  // shared memory is reused by the next list
    }
}

template <typename KeyT>
static void launch_small_t(const Ctx &c, cudaStream_t s, int sms) {
    const int smem = SmallLayout<KeyT>::kTotal;
    cudaFuncSetAttribute(k_small_sort<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    const int blocks = max(1, min(c.num_lists, sms * 2));
    launch_pdl(k_small_sort<KeyT>, dim3((unsigned)blocks), dim3(kSmallTPB), smem, s, c);
}

void launch_small(const Ctx &c, cudaStream_t s, int sms) {
    switch (c.key_bytes) {
    case 1: launch_small_t<uint8_t>(c, s, sms); break;
    case 2: launch_small_t<uint16_t>(c, s, sms); break;
    case 4: launch_small_t<uint32_t>(c, s, sms); break;
    default: launch_small_t<unsigned long long>(c, s, sms); break;
    }
    prof_mark("small", s);
    launch_relink_direct(c, s, sms);
}

}  // namespace pbit
