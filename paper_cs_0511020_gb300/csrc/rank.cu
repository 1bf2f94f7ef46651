// rank.cu -- stage (a): list ranking.  Turns list order into array order:
// ord_idx[r] / ord_key[r] = node and sort key at list rank r.  In the paper
// this is what the split loop gets by walking L = L->next (Sec.
// "Implementation in C++"); on the GPU the walk is cut into many short
// sub-walks by a sparse ruling set so that thousands of them run at once.
//
//   setup     list descriptors, hash rulers, the root task of every list
//   walk      every ruler walks next[] to the next ruler, writing the nodes it
//             visits and their sort keys into chunks (one dependent gather of
//             next[] and one independent gather of key[] per hop)
//   wyllie    walks over the ruler chain from every 32nd ruler, pointer
//             jumping over those walks -> offset of each sublist
//   validate  the root's ruler chain must end at NULL after exactly n nodes
//   emit      chunks -> (ord_idx, ord_key) at their ranks
#include "pbit_internal.cuh"

namespace pbit {

// ------------------------------------------------------------------ setup
// mode 0: lists from device offsets/roots over one pool (pool fields in t)
// mode 1: desc[] already filled by the host (serving)
// mode 2: a single list described by t
__global__ void __launch_bounds__(1024) k_setup(Ctx c, ListDesc t, const int64_t *offsets,
                                                const int32_t *roots, int mode) {
    griddep_wait();
    __shared__ int32_t s_nvirt;
    __shared__ int32_t s_bad;
    const int L = c.num_lists;
    if (threadIdx.x == 0) {
        s_bad = 0;
        s_nvirt = 0;
    }
    __syncthreads();
    if (mode == 0) {
        const int64_t off0 = offsets[0];
        for (int i = threadIdx.x; i < L; i += blockDim.x) {
            int64_t a = offsets[i], b = offsets[i + 1];
            ListDesc d = t;
            bool bad = (a < off0) || (b < a) || (b > c.ncap);
            d.n = bad ? 0 : (int32_t)(b - a);
            d.id_base = (int32_t)a;
            d.out_base = (int32_t)(a - off0);
            int32_t r = roots[i];
            if (!bad) {
                if (d.n == 0) {
                    if (r != -1)
                        atomicExch(&s_bad, PBIT_EBADLIST);
                    d.root = -1;
                } else if (r < a || r >= b) {
                    atomicExch(&s_bad, PBIT_EBADLIST);
                    d.root = -1;
                } else {
                    d.root = (int32_t)(r - a);
                }
            } else {
                atomicExch(&s_bad, PBIT_EINVAL);
                d.root = -1;
            }
            c.desc[i] = d;
            c.out_base[i] = d.out_base;
        }
        if (threadIdx.x == 0) {
            int64_t tot = offsets[L] - off0;
            if (tot < 0 || tot > c.ncap)
                atomicExch(&s_bad, PBIT_EINVAL);
            s_nvirt = (int32_t)(tot < 0 ? 0 : tot);
            c.out_base[L] = s_nvirt;
        }
    } else if (mode == 2) {
        // one list whose descriptor came in as the kernel argument
        if (threadIdx.x == 0) {
            c.desc[0] = t;
            c.out_base[0] = 0;
            c.out_base[1] = t.n;
            s_nvirt = t.n;
            if (t.n < 0 || t.n > c.ncap)
                s_bad = PBIT_EINVAL;
        }
    } else {
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int i = 0; i < L; ++i) {
                c.out_base[i] = c.desc[i].out_base;
                tot = c.desc[i].out_base + c.desc[i].n;
            }
            s_nvirt = tot;
            c.out_base[L] = tot;
        }
    }
    __syncthreads();
    const int32_t nv = s_nvirt;
    for (int i = threadIdx.x; i < L; i += blockDim.x) {
        ListDesc d = c.desc[i];
        int32_t rt = -1;
        if (d.n > 0 && d.root >= 0) {
            int32_t p = d.out_base + d.root;
            rt = is_ruler(p, c.log2S, nv) ? (p >> c.log2S) : (c.R0 + i);
        }
        c.root_task[i] = rt;
    }
    if (threadIdx.x == 0) {
        c.ctr->n_virt = nv;
        if (s_bad)
            set_status(c.status, s_bad);
    }
}

// ------------------------------------------------------------------- pack
// One streaming pass over the pool: pack[p] = {next, sort key} of the node at
// list position p's pool slot (p = out_base + local index), so the walk's
// hop reads one 8-byte (or 16-byte) record instead of gathering next[] and
// key[] from two arrays.  Shared pools map positions to nodes by one
// constant shift; per-list pools (serving) look the list up.
template <typename KeyT>
__global__ void __launch_bounds__(256) k_pack(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t nv = c.ctr->n_virt;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    int64_t lo = 0, hi = -1, shift = 0, ns = 4, ks = sizeof(KeyT);
    const unsigned char *nb = nullptr, *kb = nullptr;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nv; p += stride) {
        if (p >= hi || p < lo) {
            const int32_t lst = c.shared_pool ? 0 : upper_index(c.out_base, c.num_lists, (int32_t)p);
            const ListDesc &d = c.desc[lst];
            lo = c.shared_pool ? 0 : d.out_base;
            hi = c.shared_pool ? nv : (int64_t)d.out_base + d.n;
            shift = (int64_t)d.id_base - d.out_base;
            nb = reinterpret_cast<const unsigned char *>(d.next);
            kb = d.key;
            ns = d.next_stride;
            ks = d.key_stride;
        }
        const int64_t node = p + shift;
        const int32_t raw = *reinterpret_cast<const int32_t *>(nb + node * ns);
        const KeyT k = sort_key<KeyT>(load_key_raw<KeyT>(kb + node * ks), c.flags, c.M);
        if constexpr (sizeof(KeyT) == 8) {
            reinterpret_cast<uint4 *>(c.pack)[p] =
                make_uint4((uint32_t)raw, 0u, (uint32_t)(unsigned long long)k, (uint32_t)((unsigned long long)k >> 32));
        } else {
            reinterpret_cast<uint2 *>(c.pack)[p] = make_uint2((uint32_t)raw, (uint32_t)k);
        }
    }
}

// ------------------------------------------------------------------- walk
// Every task (a ruler) walks next[] until the next ruler or NULL, one hop per
// loop trip per lane; the key of each visited node is gathered in the same
// trip (an independent load beside the dependent next[] load) and stored,
// already mapped to its sort key, next to the node id.  Warps take 64 tasks
// at a time from a global counter and hand them to idle lanes, so a long
// sub-walk occupies one lane, not a warp or a block.  Chunks of CH entries
// come from a per-warp super-chunk of kSuper chunks.
constexpr int kSuper = 64;
constexpr int kTaskBatch = 64;

// Chunk entries are staged per lane in shared memory and written 8 at a time
// (a full 32-byte sector of node ids), so no partially written sector is
// left in L2 to be read back from DRAM when it is evicted.
constexpr int kStageN = 8;
constexpr int kStagePad = kStageN + 1;  // odd row stride: conflict-free

template <typename KeyT>
__device__ __forceinline__ void flush_group(const Ctx &c, KeyT *ckey, int64_t base, const int32_t *si,
                                            const KeyT *sk, int cnt) {
    int32_t *di = c.chunk_data + base;
    KeyT *dk = ckey + base;
    if (cnt == kStageN) {
        reinterpret_cast<int4 *>(di)[0] = make_int4(si[0], si[1], si[2], si[3]);
        reinterpret_cast<int4 *>(di)[1] = make_int4(si[4], si[5], si[6], si[7]);
        if constexpr (sizeof(KeyT) == 4) {
            reinterpret_cast<uint4 *>(dk)[0] = make_uint4(sk[0], sk[1], sk[2], sk[3]);
            reinterpret_cast<uint4 *>(dk)[1] = make_uint4(sk[4], sk[5], sk[6], sk[7]);
        } else {
#pragma unroll
            for (int i = 0; i < kStageN; ++i)
                dk[i] = sk[i];
        }
    } else {
        for (int i = 0; i < cnt; ++i) {
            di[i] = si[i];
            dk[i] = sk[i];
        }
    }
}

template <typename KeyT>
__global__ void __launch_bounds__(256, 6) k_walk(Ctx c) {
    griddep_wait();
    __shared__ int32_t s_i[256 * kStagePad];
    __shared__ KeyT s_k[256 * kStagePad];
    if (*(volatile int32_t *)c.status)
        return;
    const int lane = threadIdx.x & 31;
    int32_t *my_i = s_i + threadIdx.x * kStagePad;
    KeyT *my_k = s_k + threadIdx.x * kStagePad;
    const int32_t ntask = c.Rcap;
    const int32_t nv = c.ctr->n_virt;
    const int32_t log2S = c.log2S;
    const int32_t CH = c.CH;
    const unsigned lt = lanemask_lt();
    KeyT *ckey = reinterpret_cast<KeyT *>(c.chunk_key);

    int32_t q_next = 0, q_end = 0;  // warp-uniform task queue
    bool exhausted = false;         // warp-uniform
    int32_t pool_next = 0, pool_end = 0;  // warp-uniform super-chunk

    int32_t t = -1, v = 0, j = 0, chunk = 0;
    int32_t saved = -1;  // Brent-style cycle check: the node seen at hop 2^k
    const unsigned char *nxt = nullptr, *kp = nullptr;
    int32_t nstride = 4, kstride = 4;
    int32_t dn = 0, did = 0, dob = 0;
    bool aos = false;

    while (true) {
        const bool idle = (t < 0);
        const unsigned im = __ballot_sync(kFull, idle);
        if (im != 0 && q_next >= q_end && !exhausted) {
            int32_t base = 0;
            if (lane == 0)
                base = atomicAdd(&c.ctr->task_next.v, kTaskBatch);
            base = __shfl_sync(kFull, base, 0);
            if (base >= ntask) {
                exhausted = true;
            } else {
                q_next = base;
                q_end = min(base + kTaskBatch, ntask);
            }
        }
        if (im != 0 && q_next < q_end) {
            const int32_t cand = q_next + __popc(im & lt);
            q_next = min(q_end, q_next + __popc(im));
            if (idle && cand < q_end) {
                int32_t p = -1, lst = -1;
                if (cand < c.R0) {
                    if (((int64_t)cand << log2S) < nv) {
                        p = ruler_of_block(cand, log2S, nv);
                        lst = upper_index(c.out_base, c.num_lists, p);
                    }
                } else {
                    const int32_t i = cand - c.R0;
                    if (c.root_task[i] == cand) {
                        lst = i;
                        p = c.desc[i].out_base + c.desc[i].root;
                    }
                }
                if (p >= 0) {
                    const ListDesc &d = c.desc[lst];
                    t = cand;
                    nxt = reinterpret_cast<const unsigned char *>(d.next);
                    kp = d.key;
                    nstride = (int32_t)d.next_stride;
                    kstride = (int32_t)d.key_stride;
                    dn = d.n;
                    did = d.id_base;
                    dob = d.out_base;
                    aos = sizeof(KeyT) == 4 && nstride == 8 && kstride == 8 && kp == nxt + 4 &&
                          (reinterpret_cast<uintptr_t>(nxt) & 7) == 0;
                    v = p - dob;
                    j = 0;
                    saved = -1;
                    c.task_list[cand] = lst;
                }
            }
        }
        bool active = (t >= 0);
        if (!__any_sync(kFull, active)) {
            if (exhausted && q_next >= q_end)
                break;
            continue;
        }
        // ---- chunk allocation for lanes starting a new chunk
        const bool need = active && (j % CH == 0);
        const unsigned nm = __ballot_sync(kFull, need);
        if (nm) {
            const int32_t cnt = __popc(nm);
            const int32_t avail = pool_end - pool_next;
            const int32_t r = __popc(nm & lt);
            if (need)
                chunk = pool_next + r;  // lanes ranked below `avail` use the current super-chunk
            if (avail < cnt) {
                int32_t base = 0;
                if (lane == 0)
                    base = atomicAdd(&c.ctr->chunk_next.v, kSuper);
                base = __shfl_sync(kFull, base, 0);
                if (need && r >= avail)
                    chunk = base + (r - avail);
                pool_next = base + (cnt - avail);
                pool_end = base + kSuper;
            } else {
                pool_next += cnt;
            }
            if (need) {
                if ((int64_t)chunk >= c.chunk_cap) {
                    set_status(c.status, kStOverflow);
                    t = -1;
                    active = false;
                } else {
                    c.chunk_task[chunk] = t;
                    c.chunk_j0[chunk] = j;
                }
            }
        }
        if (active) {
            int32_t raw;
            KeyT skey;
            if (c.pack) {  // one record per hop, the key already mapped
                if constexpr (sizeof(KeyT) == 8) {
                    const uint4 r = reinterpret_cast<const uint4 *>(c.pack)[dob + v];
                    raw = (int32_t)r.x;
                    skey = (KeyT)(((unsigned long long)r.w << 32) | r.z);
                } else {
                    const uint2 r = reinterpret_cast<const uint2 *>(c.pack)[dob + v];
                    raw = (int32_t)r.x;
                    skey = (KeyT)r.y;
                }
            } else {
                const int64_t node = (int64_t)(did + v);
                KeyT key;
                if (aos) {
                    const uint2 nk = *reinterpret_cast<const uint2 *>(nxt + node * 8);
                    raw = (int32_t)nk.x;
                    key = (KeyT)nk.y;
                } else {
                    raw = *reinterpret_cast<const int32_t *>(nxt + node * nstride);
                    key = load_key_raw<KeyT>(kp + node * kstride);
                }
                skey = sort_key<KeyT>(key, c.flags, c.M);
            }
            const int e = j % CH;
            const int slot = e & (kStageN - 1);
            my_i[slot] = dob + v;
            my_k[slot] = skey;
            ++j;
            bool done = false;
            int32_t succ = -1;
            if (raw == -1) {
                done = true;
            } else {
                const int32_t w = raw - did;
                if (raw < did || w >= dn) {
                    set_status(c.status, PBIT_EBADLIST);
                    done = true;
                } else {
                    const int32_t p = dob + w;
                    if (is_ruler(p, log2S, nv)) {
                        succ = p >> log2S;
                        done = true;
                    } else if (w == saved || j >= dn) {
                        set_status(c.status, PBIT_EBADLIST);  // cycle or longer than the list
                        done = true;
                    } else {
                        if ((j & (j - 1)) == 0)
                            saved = w;  // a cycle of length l is met again before j doubles past l
                        v = w;
                    }
                }
            }
            if (slot == kStageN - 1 || done)
                flush_group<KeyT>(c, ckey, (int64_t)chunk * CH + (e - slot), my_i, my_k, slot + 1);
            if (done) {
                c.task_len[t] = j;
                c.task_succ[t] = succ;
                t = -1;
            }
        }
    }
}

// ----------------------------------------------------------------- wyllie
// Ranking the rulers in two levels.  Every 32nd ruler task (and the task of
// every list's root) walks the ruler chain (task_succ) to the next such
// task, recording for each task it passes its walk and the number of nodes
// before it in the walk; a valid list never leads back into a root's task,
// so walks need not recognise roots.  Pointer jumping (Wyllie) then runs
// over the walks only, ~32 times fewer than the rulers, and every task's
// suffix length = its walk's suffix length - the nodes before it.
__device__ __forceinline__ int64_t wy_pack(int32_t succ, uint32_t v) {
    return (int64_t)(((uint64_t)(uint32_t)succ << 32) | v);
}

__global__ void k_ruler_walk(Ctx c) {
    griddep_wait();
    const int32_t nreg = (c.Rcap + 31) / 32;  // walks started at tasks 0, 32, 64, ...
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < c.Scap;
         w += (int64_t)gridDim.x * blockDim.x) {
        int32_t t = -1;
        if (w < nreg) {
            t = (int32_t)w * 32;
        } else if (w > nreg && w - nreg - 1 < c.num_lists) {
            const int32_t rt = c.root_task[w - nreg - 1];
            if (rt >= 0 && (rt & 31) != 0)
                t = rt;  // a root task off the 32-grid starts its own walk
        }
        if (t < 0 || t >= c.Rcap || c.task_len[t] <= 0) {
            c.sw[0][w] = wy_pack(-1, 0);  // no walk here
            continue;
        }
        uint32_t before = 0;
        int32_t u = t, succ = -1;
        for (int32_t hops = 0; hops <= c.Rcap; ++hops) {
            c.wy[1][u] = wy_pack((int32_t)w, before);
            before += (uint32_t)c.task_len[u];
            const int32_t v = c.task_succ[u];
            if (v < 0)
                break;
            if (v >= c.Rcap) {
                set_status(c.status, PBIT_EBADLIST);
                break;
            }
            if ((v & 31) == 0) {
                succ = v >> 5;
                break;
            }
            u = v;
            if (hops == c.Rcap)
                set_status(c.status, PBIT_EBADLIST);  // a cycle off the grid
        }
        c.sw[0][w] = wy_pack(succ, before);
    }
}

// One pointer-jumping round over the walks: (s, v) <- (succ(s), v + v(s)).
__global__ void k_wy_round(const int64_t *a, int64_t *b, int32_t n) {
    griddep_wait();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = (uint64_t)a[t];
        const int32_t s = (int32_t)(x >> 32);
        if (s >= 0) {
            const uint64_t y = (uint64_t)a[s];
            const uint32_t val = (uint32_t)x + (uint32_t)y;
            x = (y & 0xffffffff00000000ull) | val;
        }
        b[t] = (int64_t)x;
    }
}

// Every task: (end of its chain, suffix length) from its walk's.  A task no
// walk reached (only in a malformed list) gets succ -2.
__global__ void k_ruler_expand(Ctx c, int fin) {
    griddep_wait();
    const int64_t *sw = c.sw[fin];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < c.Rcap;
         t += (int64_t)gridDim.x * blockDim.x) {
        if (c.task_len[t] <= 0)
            continue;
        const uint64_t m = (uint64_t)c.wy[1][t];
        const int32_t w = (int32_t)(m >> 32);
        if (w < 0 || w >= c.Scap) {
            c.wy[0][t] = wy_pack(-2, 0);
            continue;
        }
        const uint64_t s = (uint64_t)sw[w];
        c.wy[0][t] = wy_pack((int32_t)(s >> 32), (uint32_t)s - (uint32_t)m);
    }
}

// --------------------------------------------------------- validate + emit
__global__ void k_validate(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t *w = c.wy[0];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.num_lists; i += gridDim.x * blockDim.x) {
        const ListDesc &d = c.desc[i];
        int32_t rt = c.root_task[i];
        if (d.n == 0)
            continue;
        if (rt < 0) {
            set_status(c.status, PBIT_EBADLIST);
            continue;
        }
        uint64_t x = (uint64_t)w[rt];
        if ((int32_t)(x >> 32) != -1 || (uint32_t)x != (uint32_t)d.n)
            set_status(c.status, PBIT_EBADLIST);
    }
}

// The emit writes the list-order arrays block by block: each block of
// kEmitBlock list positions is gathered from the chunks that fill it into
// shared memory and written out as whole lines (chunks land at random
// places, so writing each chunk where it belongs would leave partly written
// sectors that L2 must fill from DRAM).  First every chunk gets its place
// and the chunks are grouped by block (count, scan, fill).

// Step 1: each used chunk's first list position and entry count (its task's
// rank + its offset in the task), and the chunks per block; a chunk that
// runs past the end of its block is counted for the next block too.
__global__ void __launch_bounds__(256) k_chunk_place(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t nchunks = min((int64_t)c.ctr->chunk_next.v, c.chunk_cap);
    const int64_t *w = c.wy[0];
    const int32_t CH = c.CH;
    for (int64_t mc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; mc < nchunks;
         mc += (int64_t)gridDim.x * blockDim.x) {
        int2 pc = make_int2(-1, 0);
        const int32_t t = c.chunk_task[mc];
        if (t >= 0) {
            const int32_t j0 = c.chunk_j0[mc];
            const int32_t len = c.task_len[t];
            const int32_t lst = c.task_list[t];
            const uint32_t suffix = (uint32_t)((uint64_t)w[t]);
            const int32_t n = c.desc[lst].n, ob = c.desc[lst].out_base;
            const int32_t cnt = min(CH, len - j0);
            const int64_t pos0 = (int64_t)ob + ((int64_t)n - (int64_t)suffix) + j0;
            if (cnt > 0) {
                if (pos0 < ob || pos0 + cnt > (int64_t)ob + n) {
                    set_status(c.status, PBIT_EBADLIST);
                } else {
                    pc = make_int2((int32_t)pos0, cnt);
                    const int64_t bk = pos0 >> kEmitLog2;
                    atomicAdd(&c.blk_cnt[bk], 1);
                    if (((pos0 + cnt - 1) >> kEmitLog2) != bk)
                        atomicAdd(&c.blk_cnt[bk + 1], 1);
                }
            }
        }
        c.chunk_pc[mc] = pc;
    }
}

// Step 2 (one CTA): blk_start = exclusive prefix of the counts; the counts
// are reset to serve as the fill cursors.  Each thread takes 32 consecutive
// counts per round (eight 16-byte loads, all in flight).
__global__ void __launch_bounds__(1024) k_blk_scan(Ctx c) {
    griddep_wait();
    __shared__ int sh[40];
    __shared__ int s_base;
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t nblk = ((int64_t)c.ctr->n_virt + kEmitBlock - 1) >> kEmitLog2;
    if (threadIdx.x == 0)
        s_base = 0;
    __syncthreads();
    constexpr int kPer = 32;
    for (int64_t r0 = 0; r0 < nblk; r0 += (int64_t)blockDim.x * kPer) {
        const int64_t b0 = r0 + (int64_t)threadIdx.x * kPer;
        int v[kPer];
        int sum = 0;
        if (b0 + kPer <= nblk) {  // (blk_cnt is 256-byte aligned: b0 is a multiple of 32)
            const int4 *q = reinterpret_cast<const int4 *>(c.blk_cnt + b0);
#pragma unroll
            for (int u = 0; u < kPer / 4; ++u) {
                const int4 x = q[u];
                v[4 * u] = x.x;
                v[4 * u + 1] = x.y;
                v[4 * u + 2] = x.z;
                v[4 * u + 3] = x.w;
            }
        } else {
#pragma unroll
            for (int u = 0; u < kPer; ++u)
                v[u] = b0 + u < nblk ? c.blk_cnt[b0 + u] : 0;
        }
#pragma unroll
        for (int u = 0; u < kPer; ++u)
            sum += v[u];
        int tot;
        int run = s_base + block_excl_scan(sum, &tot, sh);
#pragma unroll
        for (int u = 0; u < kPer; ++u) {  // counts -> starts
            const int x = v[u];
            v[u] = run;
            run += x;
        }
        if (b0 + kPer <= nblk) {
            int4 *qs = reinterpret_cast<int4 *>(c.blk_start + b0);
            int4 *qc = reinterpret_cast<int4 *>(c.blk_cnt + b0);
#pragma unroll
            for (int u = 0; u < kPer / 4; ++u) {
                qs[u] = make_int4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
                qc[u] = make_int4(0, 0, 0, 0);
            }
        } else {
#pragma unroll
            for (int u = 0; u < kPer; ++u) {
                if (b0 + u < nblk) {
                    c.blk_start[b0 + u] = v[u];
                    c.blk_cnt[b0 + u] = 0;
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0)
            s_base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0)
        c.blk_start[nblk] = s_base;
}

// Step 3: every chunk is entered in the list of each block it fills, with
// its first position relative to the block (+ 32, so a chunk that began in
// the block before stays positive) and its entry count.
__device__ __forceinline__ void blk_enter(const Ctx &c, int64_t bk, int64_t mc, int64_t pos0, int cnt) {
    const int64_t slot = (int64_t)c.blk_start[bk] + atomicAdd(&c.blk_cnt[bk], 1);
    const int rel = (int)(pos0 - (bk << kEmitLog2)) + 32;
    if (slot < (int64_t)c.blk_start[bk + 1] && slot < 2 * c.chunk_cap)
        c.blk_list[slot] = make_int2((int32_t)mc, rel | (cnt << 12));
    else
        set_status(c.status, kStOverflow);  // (inconsistent counts: cannot happen)
}

__global__ void __launch_bounds__(256) k_chunk_fill(Ctx c) {
    griddep_wait();
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t nchunks = min((int64_t)c.ctr->chunk_next.v, c.chunk_cap);
    for (int64_t mc = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; mc < nchunks;
         mc += (int64_t)gridDim.x * blockDim.x) {
        const int2 pc = c.chunk_pc[mc];
        if (pc.x < 0)
            continue;
        const int64_t bk = (int64_t)pc.x >> kEmitLog2;
        blk_enter(c, bk, mc, pc.x, pc.y);
        if ((((int64_t)pc.x + pc.y - 1) >> kEmitLog2) != bk)
            blk_enter(c, bk + 1, mc, pc.x, pc.y);
    }
}

// Step 4: one CTA per block of kEmitBlock positions.  Each warp takes its
// share of the block's chunk list (lane u holds the u-th entry; every
// chunk's 32 entries are read by the whole warp): with keys of 4 or 8 bytes
// by asynchronous copies into shared memory, all in flight at once, else
// kEmitBatch chunks at a time with the loads issued before the shared-memory
// stores.  Then the block is
// written to (ord_key, ord_idx) with 16-byte stores.  kHist (one list at
// position 0 on the 256-bucket passes): the CTA also counts the digits of the
// first pass's window [max(M - D, 0), M) and the AND/OR of the keys, as the
// first histogram kernel would (row b of the counts = tile b of the list).
constexpr int kEmitWarps = 8;
constexpr int kEmitBatch = 8;

template <typename KeyT, bool kHist>
__global__ void __launch_bounds__(32 * kEmitWarps) k_emit_blk(Ctx c) {
    griddep_wait();
    __shared__ __align__(16) KeyT sk[kEmitBlock];
    __shared__ __align__(16) int32_t si[kEmitBlock];
    __shared__ uint32_t sh_h[kHist ? kEmitWarps : 1][256];
    __shared__ unsigned long long s_and, s_or;
    if (*(volatile int32_t *)c.status)
        return;
    using U = typename KeyWord<KeyT>::U;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t nv = c.ctr->n_virt;
    const int64_t nblk = (nv + kEmitBlock - 1) >> kEmitLog2;
    const KeyT *ckey = reinterpret_cast<const KeyT *>(c.chunk_key);
    KeyT *okey = reinterpret_cast<KeyT *>(c.keyb[0]);
    int32_t *oidx = c.idxb[0];
    const int32_t CH = c.CH;
    int lo = 0;
    unsigned dmask = 0;
    if constexpr (kHist) {
        lo = max(c.M - c.D, 0);
        dmask = (1u << (c.M - lo)) - 1u;
#pragma unroll
        for (int x = 0; x < kEmitWarps; ++x)
            sh_h[x][tid] = 0;
        if (tid == 0) {
            s_and = ~0ull;
            s_or = 0ull;
        }
        __syncthreads();
    }
    long long my_elems = 0;
    for (int64_t bk = blockIdx.x; bk < nblk; bk += gridDim.x) {
        const int64_t p0 = bk << kEmitLog2;
        const int cnt_b = (int)min((int64_t)kEmitBlock, nv - p0);
        const int l0 = c.blk_start[bk], nl = c.blk_start[bk + 1] - l0;
        if constexpr (sizeof(KeyT) >= 4) {
            // keys of 4 or 8 bytes: asynchronous copies straight into shared
            // memory, so every chunk of the warp's share is in flight at once
            for (int k0 = wid; k0 < nl; k0 += kEmitWarps * 32) {
                const int k = k0 + lane * kEmitWarps;
                const int2 e = k < nl ? c.blk_list[l0 + k] : make_int2(-1, 0);
                const int ne = min(32, (nl - k0 + kEmitWarps - 1) / kEmitWarps);  // (warp-uniform)
                for (int u = 0; u < ne; ++u) {
                    const int m = __shfl_sync(kFull, e.x, u);
                    const int pk = __shfl_sync(kFull, e.y, u);
                    const int rel = (pk & 0xfff) - 32 + lane;
                    if (m >= 0 && lane < (pk >> 12) && rel >= 0 && rel < cnt_b) {
                        cp_async<(int)sizeof(KeyT)>(&sk[rel], ckey + (int64_t)m * CH + lane);
                        cp_async<4>(&si[rel], c.chunk_data + (int64_t)m * CH + lane);
                    }
                }
            }
            cp_async_commit();
            cp_async_wait_all();
        }
        for (int k0 = wid; sizeof(KeyT) < 4 && k0 < nl; k0 += kEmitWarps * kEmitBatch) {
            int2 e = make_int2(-1, 0);
            if (lane < kEmitBatch) {
                const int k = k0 + lane * kEmitWarps;
                if (k < nl)
                    e = c.blk_list[l0 + k];
            }
            KeyT kv[kEmitBatch];
            int32_t iv[kEmitBatch];
            int sp[kEmitBatch];
#pragma unroll
            for (int u = 0; u < kEmitBatch; ++u) {
                const int m = __shfl_sync(kFull, e.x, u);
                const int pk = __shfl_sync(kFull, e.y, u);
                const int rel = (pk & 0xfff) - 32 + lane;  // this lane's position in the block
                const bool ok = m >= 0 && lane < (pk >> 12) && rel >= 0 && rel < cnt_b;
                sp[u] = ok ? rel : -1;
                if (ok) {
                    kv[u] = ckey[(int64_t)m * CH + lane];
                    iv[u] = c.chunk_data[(int64_t)m * CH + lane];
                }
            }
#pragma unroll
            for (int u = 0; u < kEmitBatch; ++u) {
                if (sp[u] >= 0) {
                    sk[sp[u]] = kv[u];
                    si[sp[u]] = iv[u];
                }
            }
        }
        __syncthreads();
        my_elems += cnt_b;
        if constexpr (kHist) {
            U a_and = ~(U)0, a_or = 0;
#pragma unroll
            for (int u = 0; u < kEmitBlock / (32 * kEmitWarps); ++u) {
                const int j = u * 32 * kEmitWarps + tid;
                if (j < cnt_b) {
                    const U kk = (U)sk[j];
                    a_and &= kk;
                    a_or |= kk;
                    atomicAdd(&sh_h[wid][(unsigned)(kk >> lo) & dmask], 1u);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                a_and &= __shfl_xor_sync(kFull, a_and, o);
                a_or |= __shfl_xor_sync(kFull, a_or, o);
            }
            if (lane == 0) {  // keys are zero-extended to 64 bits
                atomicAnd(&s_and, (unsigned long long)a_and);
                atomicOr(&s_or, (unsigned long long)a_or);
            }
        }
        // write-out: whole blocks with 16-byte stores, the last one element-wise
        if (cnt_b == kEmitBlock) {
            constexpr int kKeyVec = kEmitBlock * (int)sizeof(KeyT) / 16;
            const uint4 *vk = reinterpret_cast<const uint4 *>(sk);
            uint4 *dk = reinterpret_cast<uint4 *>(okey + p0);
            for (int v = tid; v < kKeyVec; v += 32 * kEmitWarps)
                dk[v] = vk[v];
            const uint4 *vi = reinterpret_cast<const uint4 *>(si);
            uint4 *di = reinterpret_cast<uint4 *>(oidx + p0);
            for (int v = tid; v < kEmitBlock / 4; v += 32 * kEmitWarps)
                di[v] = vi[v];
        } else {
            for (int j = tid; j < cnt_b; j += 32 * kEmitWarps) {
                okey[p0 + j] = sk[j];
                oidx[p0 + j] = si[j];
            }
        }
        __syncthreads();
        if constexpr (kHist) {
            uint32_t sum = 0;
#pragma unroll
            for (int x = 0; x < kEmitWarps; ++x) {
                sum += sh_h[x][tid];
                sh_h[x][tid] = 0;
            }
            if (bk < c.row_cap)
                c.tcnt[0][bk * 256 + tid] = sum;
            else
                set_status(c.status, kStOverflow);
            if (tid == 0) {
                atomicAnd(&c.pand[0][0], s_and);
                atomicOr(&c.por[0][0], s_or);
                s_and = ~0ull;
                s_or = 0ull;
            }
            __syncthreads();  // counters and AND/OR reset before the next block counts
        }
    }
    if constexpr (kHist) {
        if (tid == 0 && my_elems)
            atomicAdd((unsigned long long *)&c.ctr->stat_elems[0], (unsigned long long)my_elems);
    }
}

// ---------------------------------------------------------------- launchers
void launch_setup(const Ctx &c, const int64_t *d_offsets, const int32_t *d_roots, int mode,
                  const ListDesc *tmpl, cudaStream_t s, int sms) {
    (void)sms;
    ListDesc t{};
    if (tmpl)
        t = *tmpl;
    launch_pdl(k_setup, dim3(1), dim3(1024), 0, s, c, t, d_offsets, d_roots, mode);
    prof_mark("setup", s);
}

void launch_pack(const Ctx &c, cudaStream_t s, int sms) {
    if (!c.pack)
        return;
    const unsigned blocks = (unsigned)max((int64_t)1, min((int64_t)sms * 8, (c.ncap + 255) / 256));
    switch (c.key_bytes) {
    case 1: launch_pdl(k_pack<uint8_t>, dim3(blocks), dim3(256), 0, s, c); break;
    case 2: launch_pdl(k_pack<uint16_t>, dim3(blocks), dim3(256), 0, s, c); break;
    case 4: launch_pdl(k_pack<uint32_t>, dim3(blocks), dim3(256), 0, s, c); break;
    default: launch_pdl(k_pack<unsigned long long>, dim3(blocks), dim3(256), 0, s, c); break;
    }
    prof_mark("pack", s);
}

void launch_walk(const Ctx &c, cudaStream_t s, int sms) {
    const int64_t warps_needed = (c.Rcap + 31) / 32;  // at least one task per lane
    // Once the records no longer fit in L2 the walk is bound by the rate of
    // random DRAM accesses, which 32 warps per SM already reach; more only
    // add contention (measured at 2^25 nodes, CTAs per SM: 2 -> 1.07 ms,
    // 4 -> 0.87 ms, 6 -> 0.89 ms, 8 (1.33 waves) -> 0.99 ms).  Smaller pools,
    // read from L2, keep the larger grid.
    const int per_sm = c.ncap >= (1ll << 24) ? 4 : 8;
    const unsigned blocks = (unsigned)min((int64_t)sms * per_sm, max((int64_t)1, (warps_needed + 7) / 8));
    switch (c.key_bytes) {
    case 1: launch_pdl(k_walk<uint8_t>, dim3(blocks), dim3(256), 0, s, c); break;
    case 2: launch_pdl(k_walk<uint16_t>, dim3(blocks), dim3(256), 0, s, c); break;
    case 4: launch_pdl(k_walk<uint32_t>, dim3(blocks), dim3(256), 0, s, c); break;
    default: launch_pdl(k_walk<unsigned long long>, dim3(blocks), dim3(256), 0, s, c); break;
    }
    prof_mark("walk", s);
}

void launch_wyllie(const Ctx &c, cudaStream_t s, int sms, int rounds) {
    const int64_t wb = min((int64_t)sms * 8, max((int64_t)1, ((int64_t)c.Scap + 127) / 128));
    launch_pdl(k_ruler_walk, dim3((unsigned)wb), dim3(128), 0, s, c);
    prof_mark("wyllie", s);
    const int64_t rb = min((int64_t)sms * 8, max((int64_t)1, ((int64_t)c.Scap + 255) / 256));
    for (int r = 0; r < rounds; ++r) {
        launch_pdl(k_wy_round, dim3((unsigned)rb), dim3(256), 0, s, c.sw[r & 1], c.sw[(r & 1) ^ 1], c.Scap);
        prof_mark("wyllie", s);
    }
    const int64_t eb = min((int64_t)sms * 8, max((int64_t)1, ((int64_t)c.Rcap + 255) / 256));
    launch_pdl(k_ruler_expand, dim3((unsigned)eb), dim3(256), 0, s, c, rounds & 1);
    prof_mark("wyllie", s);
}

void launch_validate_emit(const Ctx &c, cudaStream_t s, int sms) {
    launch_pdl(k_validate, dim3(max(1, min(sms, (c.num_lists + 255) / 256))), dim3(256), 0, s, c);
    prof_mark("validate", s);
    const unsigned cb = (unsigned)max((int64_t)1, min((int64_t)sms * 8, (c.chunk_cap + 255) / 256));
    launch_pdl(k_chunk_place, dim3(cb), dim3(256), 0, s, c);
    launch_pdl(k_blk_scan, dim3(1), dim3(1024), 0, s, c);
    launch_pdl(k_chunk_fill, dim3(cb), dim3(256), 0, s, c);
    const unsigned eb = (unsigned)max((int64_t)1, min((int64_t)sms * 8, c.blk_cap));
    const dim3 et(32 * kEmitWarps);
    if (c.emit_hist) {
        switch (c.key_bytes) {
        case 1: launch_pdl(k_emit_blk<uint8_t, true>, dim3(eb), et, 0, s, c); break;
        case 2: launch_pdl(k_emit_blk<uint16_t, true>, dim3(eb), et, 0, s, c); break;
        case 4: launch_pdl(k_emit_blk<uint32_t, true>, dim3(eb), et, 0, s, c); break;
        default: launch_pdl(k_emit_blk<unsigned long long, true>, dim3(eb), et, 0, s, c); break;
        }
    } else {
        switch (c.key_bytes) {
        case 1: launch_pdl(k_emit_blk<uint8_t, false>, dim3(eb), et, 0, s, c); break;
        case 2: launch_pdl(k_emit_blk<uint16_t, false>, dim3(eb), et, 0, s, c); break;
        case 4: launch_pdl(k_emit_blk<uint32_t, false>, dim3(eb), et, 0, s, c); break;
        default: launch_pdl(k_emit_blk<unsigned long long, false>, dim3(eb), et, 0, s, c); break;
        }
    }
    prof_mark("emit", s);
}

}  // namespace pbit
