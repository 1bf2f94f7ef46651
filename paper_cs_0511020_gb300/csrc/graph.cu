// graph.cu -- sort calls captured once as a CUDA graph and replayed, and the
// autotuner that picks the tune for a pool shape by timing the candidates.
//
// A sort call's launch sequence depends only on the pool size, the number of
// lists, the key width, M and the tune: the data (list order, keys, list
// lengths inside the pool) is read by the kernels at run time.  So one
// capture of the ~100 memsets and kernels serves every later sort of any
// lists laid out in the same pool, and replaying it costs one graph launch
// instead of one host launch per kernel.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "engine.h"

struct pbit_graph {
    int device = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int32_t *status = nullptr;    // device, in the workspace
    int32_t *new_root = nullptr;  // device: head of a single-list graph
    bool single = false;
    int64_t nodes = 0;            // graph nodes (memsets + kernels)
    int32_t *h_out = nullptr;     // pinned: status, root
};

namespace pbit {

// ------------------------------------------------------------ tune cache
// Key: device (SM count and compute capability), key width and the size
// class (ceil log2 of the pool size and of the number of lists).
struct TuneEntry {
    int sms, cc, kb, lg_n, lg_l;
    pbit_tune t;
    float ms;
};

static std::mutex g_tune_mu;
static std::vector<TuneEntry> g_tune;
static bool g_tune_loaded = false;

static int lg(int64_t x) {
    int r = 0;
    while ((1ll << r) < x)
        ++r;
    return r;
}

static int device_cc() {
    int dev = 0, ma = 0, mi = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&ma, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&mi, cudaDevAttrComputeCapabilityMinor, dev);
    return ma * 10 + mi;
}

static void tune_load_locked() {
    if (g_tune_loaded)
        return;
    g_tune_loaded = true;
    const char *path = std::getenv("PBIT_TUNE_FILE");
    if (!path || !*path)
        return;
    FILE *f = std::fopen(path, "r");
    if (!f)
        return;
    char line[256];
    while (std::fgets(line, sizeof line, f)) {
        TuneEntry e{};
        if (std::sscanf(line, "pbit-tune sms=%d cc=%d kb=%d lg_n=%d lg_l=%d cutoff=%d stride=%d ms=%f", &e.sms,
                        &e.cc, &e.kb, &e.lg_n, &e.lg_l, &e.t.smem_cutoff, &e.t.ruler_stride, &e.ms) == 8)
            g_tune.push_back(e);  // later lines win (searched from the back)
    }
    std::fclose(f);
}

bool tune_cache_lookup(int64_t pool_size, int32_t num_lists, int kb, pbit_tune *out) {
    const int sms = device_sms(), cc = device_cc(), ln = lg(pool_size), ll = lg(num_lists);
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    for (size_t i = g_tune.size(); i-- > 0;) {
        const TuneEntry &e = g_tune[i];
        if (e.sms == sms && e.cc == cc && e.kb == kb && e.lg_n == ln && e.lg_l == ll) {
            *out = e.t;
            return true;
        }
    }
    return false;
}

void tune_cache_store(int64_t pool_size, int32_t num_lists, int kb, const pbit_tune &t, float ms) {
    TuneEntry e{device_sms(), device_cc(), kb, lg(pool_size), lg(num_lists), t, ms};
    std::lock_guard<std::mutex> g(g_tune_mu);
    tune_load_locked();
    g_tune.push_back(e);
    const char *path = std::getenv("PBIT_TUNE_FILE");
    if (!path || !*path)
        return;
    if (FILE *f = std::fopen(path, "a")) {
        std::fprintf(f, "pbit-tune sms=%d cc=%d kb=%d lg_n=%d lg_l=%d cutoff=%d stride=%d ms=%.4f\n", e.sms, e.cc,
                     e.kb, e.lg_n, e.lg_l, t.smem_cutoff, t.ruler_stride, ms);
        std::fclose(f);
    }
}

// The candidates the autotuner times: the shared-memory cutoff and the
// ruler stride of the list ranking.  (The pass digit width and tile are
// compile-time constants of the pass kernel.)
static const int kDigits[] = {4, 8};
static const int kCutoffs[] = {128, 256, 512};
static const int kStrides[] = {16, 32, 64, 128};

static size_t candidate_ws_max(int64_t pool_size, int32_t num_lists, int kb) {
    size_t m = 0;
    for (int d : kDigits)
        for (int c : kCutoffs)
            for (int r : kStrides) {
                pbit_tune t{d, c, r, 0};
                size_t w = 0;
                if (pbit_workspace_size(pool_size, num_lists, kb, &t, &w) == PBIT_OK)
                    m = std::max(m, w);
            }
    size_t w = 0;
    if (pbit_workspace_size(pool_size, num_lists, kb, nullptr, &w) == PBIT_OK)
        m = std::max(m, w);
    return m;
}

static bool check_batch_args(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                             const int64_t *d_offsets, int32_t M, int32_t K, const int32_t *d_new_roots) {
    return check_pool(pool, M, K) && num_lists >= 1 && d_roots && d_offsets && d_new_roots;
}

// Capture one sort call into g (batched when d_offsets != nullptr, else one
// list given by root and n).
static pbit_status capture(pbit_graph *g, const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                           const int64_t *d_offsets, int32_t root, int64_t n, int32_t M, int32_t K,
                           int32_t *d_new_roots, const pbit_tune *tune, void *ws, size_t ws_bytes) {
    if (cudaGetDevice(&g->device) != cudaSuccess)
        return PBIT_ECUDA;
    cudaStream_t cs = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess)
        return PBIT_ECUDA;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaStreamDestroy(cs);
        return PBIT_ECUDA;
    }
    const bool prof = prof_set(false);  // timing events are not part of a graph
    Ctx c;
    pbit_status rc = enqueue_pool(pool, num_lists, d_roots, d_offsets, root, n, M, K, d_new_roots, tune, ws,
                                  ws_bytes, cs, &c);
    prof_set(prof);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cs, &graph);  // always ends the capture
    cudaStreamDestroy(cs);
    if (rc == PBIT_OK && (e != cudaSuccess || !graph))
        rc = PBIT_ECUDA;
    if (rc != PBIT_OK) {
        if (graph)
            cudaGraphDestroy(graph);
        return rc;
    }
    g->graph = graph;
    if (cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess)
        return PBIT_ECUDA;
    size_t nn = 0;
    if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess)
        g->nodes = (int64_t)nn;
    g->status = c.status;
    g->new_root = c.new_roots;
    return PBIT_OK;
}

}  // namespace pbit

using namespace pbit;

extern "C" {

pbit_status pbit_graph_create_batched(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                      const int64_t *d_offsets, int32_t M, int32_t K, int32_t *d_new_roots,
                                      const pbit_tune *tune, void *ws, size_t ws_bytes, pbit_graph **out) {
    if (!out || !check_batch_args(pool, num_lists, d_roots, d_offsets, M, K, d_new_roots))
        return PBIT_EINVAL;
    pbit_graph *g = new pbit_graph();
    pbit_status rc = capture(g, pool, num_lists, d_roots, d_offsets, 0, 0, M, K, d_new_roots, tune, ws, ws_bytes);
    if (rc == PBIT_OK && cudaMallocHost((void **)&g->h_out, 64) != cudaSuccess)
        rc = PBIT_ECUDA;
    if (rc != PBIT_OK) {
        pbit_graph_destroy(g);
        return rc;
    }
    *out = g;
    return PBIT_OK;
}

pbit_status pbit_graph_create_single(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                     const pbit_tune *tune, void *ws, size_t ws_bytes, pbit_graph **out) {
    if (!out || !check_pool(pool, M, K) || n != pool->pool_size || n < 1)
        return PBIT_EINVAL;
    if (root < 0 || root >= n)
        return PBIT_EBADLIST;
    pbit_graph *g = new pbit_graph();
    g->single = true;
    pbit_status rc = capture(g, pool, 1, nullptr, nullptr, root, n, M, K, nullptr, tune, ws, ws_bytes);
    if (rc == PBIT_OK && cudaMallocHost((void **)&g->h_out, 64) != cudaSuccess)
        rc = PBIT_ECUDA;
    if (rc != PBIT_OK) {
        pbit_graph_destroy(g);
        return rc;
    }
    *out = g;
    return PBIT_OK;
}

pbit_status pbit_graph_launch(pbit_graph *g, void *stream) {
    if (!g || !g->exec)
        return PBIT_EINVAL;
    return cudaGraphLaunch(g->exec, (cudaStream_t)stream) == cudaSuccess ? PBIT_OK : PBIT_ECUDA;
}

pbit_status pbit_graph_result(pbit_graph *g, void *stream, int32_t *new_root_host) {
    if (!g || !g->exec)
        return PBIT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemcpyAsync(g->h_out, g->status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        (g->single && cudaMemcpyAsync(g->h_out + 1, g->new_root, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PBIT_ECUDA;
    const pbit_status st = map_status(g->h_out[0]);
    if (st == PBIT_OK && g->single && new_root_host)
        *new_root_host = g->h_out[1];
    return st;
}

int64_t pbit_graph_node_count(const pbit_graph *g) { return g ? g->nodes : 0; }

void pbit_graph_destroy(pbit_graph *g) {
    if (!g)
        return;
    if (g->exec)
        cudaGraphExecDestroy(g->exec);
    if (g->graph)
        cudaGraphDestroy(g->graph);
    if (g->h_out)
        cudaFreeHost(g->h_out);
    delete g;
}

pbit_status pbit_autotune_workspace_size(int64_t pool_size, int32_t num_lists, int32_t key_type, size_t *bytes) {
    if (!bytes || pool_size < 0 || pool_size >= (1ll << 31) || num_lists < 1)
        return PBIT_EINVAL;
    if (key_type != 1 && key_type != 2 && key_type != 4 && key_type != 8)
        return PBIT_EINVAL;
    *bytes = candidate_ws_max(pool_size, num_lists, key_type);
    return *bytes ? PBIT_OK : PBIT_EINVAL;
}

pbit_status pbit_autotune_batched(const pbit_pool *pool, int32_t num_lists, const int32_t *d_roots,
                                  const int64_t *d_offsets, int32_t M, int32_t K, int32_t *d_new_roots, void *ws,
                                  size_t ws_bytes, int32_t reps, void *stream, pbit_tune *best, float *best_ms) {
    if (!best || reps < 1 || reps > 64 || !check_batch_args(pool, num_lists, d_roots, d_offsets, M, K, d_new_roots))
        return PBIT_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    const PoolSpan sp = pool_span(pool);
    // every trial sorts the caller's lists from their input state: save next[]
    // (and prev[]) once and restore them before each trial and at the end
    unsigned char *save = nullptr;
    const size_t save_bytes = sp.next_bytes + sp.prev_bytes;
    if (save_bytes && cudaMalloc((void **)&save, save_bytes) != cudaSuccess)
        return PBIT_ENOMEM;
    auto copy_all = [&](bool restore) -> bool {
        unsigned char *nx = (unsigned char *)pool->next, *pv = (unsigned char *)pool->prev;
        if (sp.next_bytes && cudaMemcpyAsync(restore ? nx : save, restore ? save : nx, sp.next_bytes,
                                             cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return false;
        if (sp.prev_bytes && cudaMemcpyAsync(restore ? pv : save + sp.next_bytes, restore ? save + sp.next_bytes : pv,
                                             sp.prev_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
            return false;
        return true;
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    pbit_status rc = PBIT_OK;
    if (!copy_all(false) || cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        rc = PBIT_ECUDA;
    float best_t = INFINITY;
    pbit_tune best_c{};
    pbit_status last_err = PBIT_ENOMEM;
    constexpr int nd = (int)(sizeof kDigits / sizeof *kDigits), nc = (int)(sizeof kCutoffs / sizeof *kCutoffs),
                  nr = (int)(sizeof kStrides / sizeof *kStrides);
    for (int ci = 0; rc == PBIT_OK && ci < nd * nc; ++ci) {
        for (int ri = 0; rc == PBIT_OK && ri < nr; ++ri) {
            const pbit_tune cand{kDigits[ci / nc], kCutoffs[ci % nc], kStrides[ri], 0};
            size_t need = 0;
            if (pbit_workspace_size(pool->pool_size, num_lists, pool->key_type, &cand, &need) != PBIT_OK ||
                need > ws_bytes)
                continue;
            std::vector<float> times;
            pbit_status st = PBIT_OK;
            for (int r = 0; r <= reps && st == PBIT_OK; ++r) {  // r == 0 warms up
                Ctx c;
                if (!copy_all(true) || cudaEventRecord(e0, s) != cudaSuccess) {
                    rc = PBIT_ECUDA;
                    break;
                }
                st = enqueue_pool(pool, num_lists, d_roots, d_offsets, 0, 0, M, K, d_new_roots, &cand, ws, ws_bytes,
                                  s, &c);
                int32_t dev_st = 0;
                if (st == PBIT_OK &&
                    (cudaEventRecord(e1, s) != cudaSuccess ||
                     cudaMemcpyAsync(&dev_st, c.status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                     cudaStreamSynchronize(s) != cudaSuccess)) {
                    rc = PBIT_ECUDA;
                    break;
                }
                if (st == PBIT_OK)
                    st = map_status(dev_st);
                float ms = 0.f;
                if (st == PBIT_OK && r > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    times.push_back(ms);
            }
            if (st != PBIT_OK) {
                last_err = st;
                if (st == PBIT_EBADLIST || st == PBIT_ECUDA || st == PBIT_ETIMEOUT)
                    rc = st;  // the input or the device is at fault, not the candidate
                continue;
            }
            if (times.empty())
                continue;
            std::sort(times.begin(), times.end());
            const float med = times[times.size() / 2];
            if (med < best_t) {
                best_t = med;
                best_c = cand;
            }
        }
    }
    if (save) {
        if (!copy_all(true) || cudaStreamSynchronize(s) != cudaSuccess)
            rc = PBIT_ECUDA;
        cudaFree(save);
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    if (rc != PBIT_OK)
        return rc;
    if (!std::isfinite(best_t))
        return last_err;
    *best = best_c;
    if (best_ms)
        *best_ms = best_t;
    tune_cache_store(pool->pool_size, num_lists, pool->key_type, best_c, best_t);
    return PBIT_OK;
}

}  // extern "C"
