// rank.cu -- stage (a): list ranking.  Turns list order into array order:
// ord_idx[r] / ord_key[r] = node and sort key at list rank r.  In the paper
// this is what the split loop gets by walking L = L->next (Sec.
// "Implementation in C++"); on the GPU the walk is cut into many short
// sub-walks by a sparse ruling set so that thousands of them run at once.
//
//   setup     list descriptors, hash rulers, the root task of every list
//   walk      every ruler walks next[] to the next ruler, writing the nodes it
//             visits into chunks (one dependent gather per hop)
//   wyllie    pointer jumping over the ruler sublists -> offset of each sublist
//   validate  the root's ruler chain must end at NULL after exactly n nodes
//   emit      chunks -> (ord_idx, ord_key) at their ranks, keys gathered and
//             mapped to unsigned sort keys
#include "pbit_internal.cuh"

namespace pbit {

// ------------------------------------------------------------------ setup
// mode 0: lists from device offsets/roots over one pool (pool fields in t)
// mode 1: desc[] already filled by the host (serving)
// mode 2: a single list described by t
__global__ void __launch_bounds__(1024) k_setup(Ctx c, ListDesc t, const int64_t *offsets,
                                                const int32_t *roots, int mode) {
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

// ------------------------------------------------------------------- walk
// Warps own a static block of tasks; idle lanes refill from it, so a long
// sub-walk keeps one lane busy instead of a whole block.  Chunks of CH node
// ids are taken from a per-warp super-chunk of kSuper chunks, so the global
// bump allocator sees one atomic per kSuper chunks.
constexpr int kSuper = 64;

__global__ void __launch_bounds__(256) k_walk(Ctx c) {
    if (*(volatile int32_t *)c.status)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t ntask = c.Rcap;
    const int32_t per = (int32_t)((ntask + nwarps - 1) / nwarps);
    const int32_t t_begin = (int32_t)min((int64_t)ntask, gwarp * per);
    const int32_t t_end = (int32_t)min((int64_t)ntask, (int64_t)t_begin + per);
    const int32_t nv = c.ctr->n_virt;
    const int32_t log2S = c.log2S;
    const int32_t CH = c.CH;
    const unsigned lt = lanemask_lt();

    int32_t next_t = t_begin;  // warp-uniform
    int32_t pool_next = 0, pool_end = 0;  // warp-uniform

    int32_t t = -1, v = 0, j = 0, chunk = 0;
    int32_t saved = -1, power = 1, lam = 0;  // Brent cycle detection
    int32_t *nxt = nullptr;
    int64_t nstride = 4;
    int32_t dn = 0, did = 0, dob = 0;

    while (true) {
        // ---- refill idle lanes with the warp's next tasks
        bool idle = (t < 0);
        unsigned im = __ballot_sync(kFull, idle);
        if (im != 0 && next_t < t_end) {
            int32_t cand = next_t + __popc(im & lt);
            next_t += __popc(im);
            if (idle && cand < t_end) {
                // find the start node of task cand
                int32_t p = -1, lst = -1;
                if (cand < c.R0) {
                    if (((int64_t)cand << log2S) < nv) {
                        p = ruler_of_block(cand, log2S, nv);
                        lst = upper_index(c.out_base, c.num_lists, p);
                    }
                } else {
                    int32_t i = cand - c.R0;
                    if (c.root_task[i] == cand) {
                        lst = i;
                        p = c.desc[i].out_base + c.desc[i].root;
                    }
                }
                if (p >= 0) {
                    const ListDesc &d = c.desc[lst];
                    t = cand;
                    nxt = d.next;
                    nstride = d.next_stride;
                    dn = d.n;
                    did = d.id_base;
                    dob = d.out_base;
                    v = p - dob;
                    j = 0;
                    saved = -1;
                    power = 1;
                    lam = 0;
                    c.task_list[cand] = lst;
                }
            }
        }
        bool active = (t >= 0);
        if (!__any_sync(kFull, active)) {
            if (next_t >= t_end)
                break;
            continue;
        }
        // ---- chunk allocation for lanes starting a new chunk
        bool need = active && (j % CH == 0);
        unsigned nm = __ballot_sync(kFull, need);
        if (nm) {
            const int32_t cnt = __popc(nm);
            const int32_t avail = pool_end - pool_next;
            const int32_t r = __popc(nm & lt);
            if (need)
                chunk = pool_next + r;  // lanes ranked below `avail` use the current super-chunk
            if (avail < cnt) {
                int32_t base = 0;
                if (lane == 0)
                    base = atomicAdd(&c.ctr->chunk_next, kSuper);
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
            c.chunk_data[(int64_t)chunk * CH + (j % CH)] = dob + v;
            ++j;
            int32_t raw = *(const int32_t *)((const unsigned char *)nxt + (int64_t)(did + v) * nstride);
            bool done = false;
            int32_t succ = -1;
            if (raw == -1) {
                done = true;
            } else {
                int32_t w = raw - did;
                if (raw < did || w >= dn) {
                    set_status(c.status, PBIT_EBADLIST);
                    done = true;
                } else {
                    int32_t p = dob + w;
                    if (is_ruler(p, log2S, nv)) {
                        succ = p >> log2S;
                        done = true;
                    } else if (w == saved || j >= dn) {
                        set_status(c.status, PBIT_EBADLIST);  // cycle or longer than the list
                        done = true;
                    } else {
                        if (lam == power) {
                            saved = w;
                            power <<= 1;
                            lam = 0;
                        }
                        ++lam;
                        v = w;
                    }
                }
            }
            if (done) {
                c.task_len[t] = j;
                c.task_succ[t] = succ;
                t = -1;
            }
        }
    }
}

// ----------------------------------------------------------------- wyllie
__global__ void k_wy_init(Ctx c) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < c.Rcap;
         t += (int64_t)gridDim.x * blockDim.x) {
        int32_t s = c.task_succ[t];
        uint32_t l = (uint32_t)c.task_len[t];
        c.wy[0][t] = (int64_t)(((uint64_t)(uint32_t)s << 32) | l);
    }
}

// One pointer-jumping round: (s, v) <- (succ(s), v + v(s)).
__global__ void k_wy_round(Ctx c, int in) {
    const int64_t *a = c.wy[in];
    int64_t *b = c.wy[in ^ 1];
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < c.Rcap;
         t += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = (uint64_t)a[t];
        int32_t s = (int32_t)(x >> 32);
        if (s >= 0) {
            uint64_t y = (uint64_t)a[s];
            uint32_t val = (uint32_t)x + (uint32_t)y;
            x = (y & 0xffffffff00000000ull) | val;
        }
        b[t] = (int64_t)x;
    }
}

// --------------------------------------------------------- validate + emit
__global__ void k_validate(Ctx c, int fin) {
    if (*(volatile int32_t *)c.status)
        return;
    const int64_t *w = c.wy[fin];
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

template <typename KeyT>
__global__ void __launch_bounds__(256) k_emit(Ctx c, int fin) {
    if (*(volatile int32_t *)c.status)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t nchunks = min((int64_t)c.ctr->chunk_next, c.chunk_cap);
    const int64_t *w = c.wy[fin];
    KeyT *okey = reinterpret_cast<KeyT *>(c.keyb[0]);
    int32_t *oidx = c.idxb[0];
    const int CH = c.CH;  // == 32
    for (int64_t ch = gwarp; ch < nchunks; ch += nwarps) {
        int32_t t = c.chunk_task[ch];
        if (t < 0)
            continue;
        int32_t j0 = c.chunk_j0[ch];
        int32_t len = c.task_len[t];
        int32_t lst = c.task_list[t];
        const ListDesc &d = c.desc[lst];
        uint32_t suffix = (uint32_t)((uint64_t)w[t]);
        int32_t cnt = min(CH, len - j0);
        int64_t pos0 = (int64_t)d.out_base + ((int64_t)d.n - (int64_t)suffix) + j0;
        if (lane < cnt) {
            int32_t p = c.chunk_data[ch * CH + lane];
            int64_t pos = pos0 + lane;
            if (pos < d.out_base || pos >= (int64_t)d.out_base + d.n) {
                set_status(c.status, PBIT_EBADLIST);
            } else {
                int32_t loc = p - d.out_base;
                KeyT k = load_key_raw<KeyT>(d.key + (int64_t)(d.id_base + loc) * d.key_stride);
                okey[pos] = sort_key<KeyT>(k, c.flags, c.M);
                oidx[pos] = p;
            }
        }
    }
}

// ---------------------------------------------------------------- launchers
void launch_setup(const Ctx &c, const int64_t *d_offsets, const int32_t *d_roots, int mode,
                  const ListDesc *tmpl, cudaStream_t s, int sms) {
    (void)sms;
    ListDesc t{};
    if (tmpl)
        t = *tmpl;
    k_setup<<<1, 1024, 0, s>>>(c, t, d_offsets, d_roots, mode);
}

void launch_walk(const Ctx &c, cudaStream_t s, int sms) {
    int64_t warps_needed = (c.Rcap + 31) / 32;  // at least one task per lane
    int64_t blocks = min((int64_t)sms * 8, max((int64_t)1, (warps_needed + 7) / 8));
    k_walk<<<(unsigned)blocks, 256, 0, s>>>(c);
}

void launch_wyllie(const Ctx &c, cudaStream_t s, int sms, int rounds) {
    int64_t blocks = min((int64_t)sms * 8, max((int64_t)1, ((int64_t)c.Rcap + 255) / 256));
    k_wy_init<<<(unsigned)blocks, 256, 0, s>>>(c);
    for (int r = 0; r < rounds; ++r)
        k_wy_round<<<(unsigned)blocks, 256, 0, s>>>(c, r & 1);
}

void launch_validate_emit(const Ctx &c, int fin, cudaStream_t s, int sms) {
    k_validate<<<max(1, min(sms, (c.num_lists + 255) / 256)), 256, 0, s>>>(c, fin);
    unsigned blocks = (unsigned)(sms * 8);
    switch (c.key_bytes) {
    case 1: k_emit<uint8_t><<<blocks, 256, 0, s>>>(c, fin); break;
    case 2: k_emit<uint16_t><<<blocks, 256, 0, s>>>(c, fin); break;
    case 4: k_emit<uint32_t><<<blocks, 256, 0, s>>>(c, fin); break;
    default: k_emit<unsigned long long><<<blocks, 256, 0, s>>>(c, fin); break;
    }
}

}  // namespace pbit
