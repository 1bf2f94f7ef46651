// finish.cu -- stages (c) and (d).
//
// (c) Small buckets are finished in shared memory.  In the paper the
//     recursion runs every bucket down to M == 0 and merge() then appends the
//     leaf buckets (Sec. "Implementation in C++", Sec. 5.1); the paper itself
//     notes that MSD sorting spends too long on small chunks (Sec.
//     "Differences between Pbit and other algorithms sorting with bit key").
//     Here a bucket of at most `cutoff` nodes is loaded once, sorted stably
//     on its remaining low bits by shared-memory counting passes (least
//     significant window first, skipping windows in which no key differs),
//     and its node ids are written to the final order buffer F.
// (d) The relink concatenates the sorted fragments: next[s[i]] = s[i+1],
//     next[s[n-1]] = -1, root = s[0] -- the effect of the merge() chain
//     (Sec. 5.1) done for all nodes at once.  For doubly-linked pools the
//     predecessor pointers are rebuilt in the same pass (Sec. "Double-linked
//     lists sorting").
#include "pbit_internal.cuh"

namespace pbit {

constexpr int kFTPB = 512;
constexpr int kFItems = 8;
constexpr int kFCap = kFTPB * kFItems;  // largest bucket the finish kernel sorts
constexpr int kFD = 4;
constexpr int kFBins = 1 << kFD;

template <typename KeyT>
constexpr int finish_smem() {
    return kFCap * (int)sizeof(KeyT) + kFCap * 4;
}

template <typename KeyT>
__global__ void __launch_bounds__(kFTPB, 2) k_finish(Ctx c) {
    extern __shared__ __align__(16) unsigned char f_smem[];
    KeyT *s_key = reinterpret_cast<KeyT *>(f_smem);
    int32_t *s_idx = reinterpret_cast<int32_t *>(f_smem + kFCap * sizeof(KeyT));
    __shared__ uint32_t s_w[kFTPB / 32][kFBins];
    __shared__ uint32_t s_off[kFBins];
    __shared__ unsigned long long s_and, s_or;
    __shared__ int s_e;
    if (*(volatile int32_t *)c.status)
        return;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const unsigned lt = lanemask_lt();
    const int nfin = c.ctr->fin_count;
    while (true) {
        __syncthreads();
        if (tid == 0) {
            s_e = atomicAdd(&c.ctr->fin_ctr, 1);
            s_and = ~0ull;
            s_or = 0ull;
        }
        __syncthreads();
        const int e = s_e;
        if (e >= nfin)
            break;
        const Fin f = c.fin[e];
        const int mode = f.mode_buf >> 8, buf = f.mode_buf & 1;
        const int start = f.start, len = f.len;
        const int32_t *src_idx = c.idxb[buf] + start;
        int32_t *dst = c.F + start;
        if (mode == 0 || len <= 1) {
            if (tid == 0)
                atomicAdd((unsigned long long *)&c.ctr->fin_copy_elems, (unsigned long long)len);
            for (int j = tid; j < len; j += kFTPB)
                dst[j] = src_idx[j];
            continue;
        }
        if (tid == 0)
            atomicAdd((unsigned long long *)&c.ctr->fin_sort_elems, (unsigned long long)len);
        if (len > kFCap) {
            set_status(c.status, kStOverflow);
            continue;
        }
        const KeyT *src_key = reinterpret_cast<const KeyT *>(c.keyb[buf]) + start;
        KeyT key[kFItems];
        int32_t idx[kFItems];
        unsigned long long a_and = ~0ull, a_or = 0ull;
        // item rounds of this warp that hold data (warp-uniform)
        const int wbase = wid * (32 * kFItems);
        const int nit = len <= wbase ? 0 : min(kFItems, (len - wbase + 31) / 32);
#pragma unroll
        for (int i = 0; i < kFItems; ++i) {
            const int pos = wid * (32 * kFItems) + i * 32 + lane;
            if (pos < len) {
                key[i] = src_key[pos];
                idx[i] = src_idx[pos];
                a_and &= (unsigned long long)key[i];
                a_or |= (unsigned long long)key[i];
            } else {
                key[i] = 0;
                idx[i] = 0;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a_and &= __shfl_xor_sync(kFull, a_and, o);
            a_or |= __shfl_xor_sync(kFull, a_or, o);
        }
        if (lane == 0) {
            atomicAnd(&s_and, a_and);
            atomicOr(&s_or, a_or);
        }
        __syncthreads();
        const int hi = f.hi;
        const unsigned long long vary = (s_and ^ s_or) & (hi >= 64 ? ~0ull : ((1ull << hi) - 1ull));
        for (int wl = 0; wl < hi; wl += kFD) {
            const int width = min(kFD, hi - wl);
            const unsigned dmask = (1u << width) - 1u;
            if (((vary >> wl) & dmask) == 0)
                continue;  // every key agrees on this window
            uint32_t rnk[kFItems];
            uint32_t run = 0;
#pragma unroll
            for (int i = 0; i < kFItems; ++i) {
                if (i >= nit)
                    break;
                const int pos = wid * (32 * kFItems) + i * 32 + lane;
                const bool valid = pos < len;
                const unsigned dig = valid ? (unsigned)((unsigned long long)key[i] >> wl) & dmask : 0u;
                const unsigned vm = __ballot_sync(kFull, valid);
                unsigned peers = vm, mine = vm;
#pragma unroll
                for (int b = 0; b < kFD; ++b) {
                    const unsigned bb = __ballot_sync(kFull, (dig >> b) & 1u);
                    peers &= ((dig >> b) & 1u) ? bb : ~bb;
                    mine &= ((lane >> b) & 1) ? bb : ~bb;
                }
                rnk[i] = __shfl_sync(kFull, run, (int)dig) + __popc(peers & lt);
                run += __popc(mine);
            }
            if (lane < kFBins)
                s_w[wid][lane] = run;
            __syncthreads();
            if (wid == 0 && lane < kFBins) {
                uint32_t tot = 0;
#pragma unroll
                for (int w = 0; w < kFTPB / 32; ++w) {
                    const uint32_t x = s_w[w][lane];
                    s_w[w][lane] = tot;
                    tot += x;
                }
                uint32_t incl = tot;
#pragma unroll
                for (int o = 1; o < kFBins; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffu, incl, o);
                    if (lane >= o)
                        incl += y;
                }
                s_off[lane] = incl - tot;
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kFItems; ++i) {
                if (i >= nit)
                    break;
                const int pos = wid * (32 * kFItems) + i * 32 + lane;
                if (pos < len) {
                    const unsigned dig = (unsigned)((unsigned long long)key[i] >> wl) & dmask;
                    const uint32_t lp = s_off[dig] + s_w[wid][dig] + rnk[i];
                    s_key[lp] = key[i];
                    s_idx[lp] = idx[i];
                }
            }
            __syncthreads();
#pragma unroll
            for (int i = 0; i < kFItems; ++i) {
                if (i >= nit)
                    break;
                const int pos = wid * (32 * kFItems) + i * 32 + lane;
                if (pos < len) {
                    key[i] = s_key[pos];
                    idx[i] = s_idx[pos];
                }
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < kFItems; ++i) {
            const int pos = wid * (32 * kFItems) + i * 32 + lane;
            if (pos < len)
                dst[pos] = idx[i];
        }
    }
}

// Stage (d): relink, direct form: one thread per sorted position writes
// next[s[q]] = s[q+1] straight into the pool (scattered 4-byte stores).  Used
// when the lists live in different pools (the request server).
__global__ void k_relink(Ctx c) {
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
// pairs; bucket b owns slots [b << rb, (b << rb) + count).
constexpr int kRelTPB = 256;
constexpr int kRelItems = 16;
constexpr int kRelTile = kRelTPB * kRelItems;
constexpr int kMaxRelBuckets = 512;

__global__ void __launch_bounds__(kRelTPB) k_relink_part(Ctx c, int rb) {
    __shared__ int32_t s_cnt[kMaxRelBuckets];
    __shared__ int32_t s_base[kMaxRelBuckets];
    if (*(volatile int32_t *)c.status)
        return;
    const int32_t nv = c.ctr->n_virt;
    const int L = c.num_lists;
    const int nb = (int)((c.ncap + (1ll << rb) - 1) >> rb);
    const bool doubly = (c.flags & PBIT_DOUBLY) != 0;
    int32_t *tv = c.idxb[0], *ts = c.idxb[1];
    for (int64_t q0 = (int64_t)blockIdx.x * kRelTile; q0 < nv; q0 += (int64_t)gridDim.x * kRelTile) {
        for (int b = threadIdx.x; b < nb; b += kRelTPB)
            s_cnt[b] = 0;
        __syncthreads();
        int32_t vv[kRelItems], ss[kRelItems], rk[kRelItems];
#pragma unroll
        for (int i = 0; i < kRelItems; ++i) {
            const int64_t q = q0 + i * kRelTPB + threadIdx.x;
            vv[i] = -1;
            if (q < nv) {
                const int lst = upper_index(c.out_base, L, (int32_t)q);
                const ListDesc &d = c.desc[lst];
                const int32_t loc = c.F[q] - d.out_base;
                const int64_t end = (int64_t)d.out_base + d.n;
                int32_t succ = -1;
                bool bad = loc < 0 || loc >= d.n;
                if (q + 1 < end) {
                    const int32_t ls = c.F[q + 1] - d.out_base;
                    bad |= ls < 0 || ls >= d.n;
                    succ = d.id_base + ls;
                    if (doubly && !bad)
                        *(int32_t *)((unsigned char *)d.prev + (int64_t)succ * d.prev_stride) = d.id_base + loc;
                }
                if (bad) {
                    set_status(c.status, kStOverflow);
                } else {
                    vv[i] = d.id_base + loc;
                    ss[i] = succ;
                    if (q == d.out_base) {
                        c.new_roots[lst] = vv[i];
                        if (doubly)
                            *(int32_t *)((unsigned char *)d.prev + (int64_t)vv[i] * d.prev_stride) = -1;
                    }
                    rk[i] = atomicAdd(&s_cnt[vv[i] >> rb], 1);
                }
            }
        }
        __syncthreads();
        for (int b = threadIdx.x; b < nb; b += kRelTPB)
            s_base[b] = s_cnt[b] ? atomicAdd(&c.rel_cursor[b], s_cnt[b]) : 0;
        __syncthreads();
#pragma unroll
        for (int i = 0; i < kRelItems; ++i) {
            if (vv[i] >= 0) {
                const int b = vv[i] >> rb;
                const int64_t slot = ((int64_t)b << rb) + s_base[b] + rk[i];
                tv[slot] = vv[i];
                ts[slot] = ss[i];
            }
        }
        __syncthreads();
    }
}

// Apply the pairs of node blocks [b0, b0 + nbk): one launch per window so
// the stores in flight stay inside a few MB of next[].
__global__ void k_relink_apply(Ctx c, int rb, int b0) {
    if (*(volatile int32_t *)c.status)
        return;
    const int32_t *tv = c.idxb[0], *ts = c.idxb[1];
    unsigned char *next = reinterpret_cast<unsigned char *>(c.desc[0].next);
    const int64_t stride = c.desc[0].next_stride;
    const int32_t cnt = c.rel_cursor[b0];
    const int64_t base = (int64_t)b0 << rb;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += (int64_t)gridDim.x * blockDim.x)
        *(int32_t *)(next + (int64_t)tv[base + i] * stride) = ts[base + i];
}

__global__ void k_empty_roots(Ctx c) {
    if (*(volatile int32_t *)c.status)
        return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.num_lists; i += gridDim.x * blockDim.x)
        if (c.desc[i].n == 0)
            c.new_roots[i] = -1;
}

// Every node must have been placed by a pass or by the finish: any segment
// still live after the last pass means the pass budget was too small.
__global__ void k_check_done(Ctx c, int iters) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const int p = iters & 1;
        if (c.ctr->act_count[p] != 0 || c.ctr->pend_count[p] != 0)
            set_status(c.status, kStOverflow);
    }
}

template <typename KeyT>
static void launch_finish_t(const Ctx &c, cudaStream_t s, int sms) {
    constexpr int smem = finish_smem<KeyT>();
    cudaFuncSetAttribute(k_finish<KeyT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_finish<KeyT><<<(unsigned)(sms * 2), kFTPB, smem, s>>>(c);
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
        const int64_t pblocks = min((int64_t)sms * 8, max((int64_t)1, (c.ncap + kRelTile - 1) / kRelTile));
        k_relink_part<<<(unsigned)pblocks, kRelTPB, 0, s>>>(c, rb);
        const int64_t ablocks = min((int64_t)sms * 8, (int64_t)(((1ll << rb) + 255) / 256));
        const int nb = (int)((c.ncap + (1ll << rb) - 1) >> rb);
        for (int b = 0; b < nb; ++b)
            k_relink_apply<<<(unsigned)ablocks, 256, 0, s>>>(c, rb, b);
    } else {
        const int64_t blocks = min((int64_t)sms * 16, max((int64_t)1, (c.ncap + 255) / 256));
        k_relink<<<(unsigned)blocks, 256, 0, s>>>(c);
    }
    prof_mark("relink", s);
    k_empty_roots<<<max(1, min(sms, (c.num_lists + 255) / 256)), 256, 0, s>>>(c);
    prof_mark("relink", s);
}

void launch_check_done(const Ctx &c, int iters, cudaStream_t s) {
    k_check_done<<<1, 32, 0, s>>>(c, iters);
    prof_mark("plan", s);
}

int finish_capacity() { return kFCap; }

// Blocked relink when every list shares one pool (not the request server's
// per-request pools): window of 2^rb nodes = at most 16 MB of next[].
bool relink_blocked(const Ctx &c) { return c.shared_pool != 0; }
int relink_bucket_bits(const Ctx &c) {
    int rb = c.desc_next_stride <= 4 ? 22 : (c.desc_next_stride <= 8 ? 21 : 20);
    while (rb < 31 && ((c.ncap + (1ll << rb) - 1) >> rb) > kMaxRelBuckets)
        ++rb;
    return rb;
}
int relink_max_buckets() { return kMaxRelBuckets; }

}  // namespace pbit
