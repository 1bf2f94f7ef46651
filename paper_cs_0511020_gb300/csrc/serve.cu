// serve.cu -- request server: continuous batching of sort requests.
//
// Callers submit lists that live in their own device pools.  A scheduler
// thread forms batches from the queue and launches each one as soon as a
// CUDA stream is free and its workspace fits in the free part of the device
// arena (the memory budget): the arena is carved per batch, first fit, and
// given back when the batch completes, so the sum of the workspaces in
// flight never exceeds the budget, and a large request waits only until
// enough memory has been freed (batches are formed from the head of the
// queue, in arrival order, so no request waits behind later ones).
// Requests that arrive while other batches run on the GPU join the next
// batch; up to `streams` batches overlap on the device.  A batch is one sort
// call whose lists are its requests (each list with its own pool, relinked in
// place); requests of one batch share key type, flags, M and K.  If a batch
// fails (a malformed list), its requests are retried one by one so each gets
// its own status.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.h"

namespace pbit {

struct SrvReq {
    uint64_t ticket;
    pbit_pool pool;
    int32_t root;
    int64_t n;
    int M, K;
    bool solo = false;      // retry alone (its batch failed)
    int status = PBIT_EPENDING;
    int32_t new_root = -1;
    int64_t submit_ns = 0, done_ns = 0;  // host steady clock
};

static int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

// One CUDA stream and what a batch in flight on it holds.
struct SrvSlot {
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    ListDesc *h_desc = nullptr;  // pinned, max_batch entries
    int32_t *h_out = nullptr;    // pinned: status, then one head per list
    std::vector<SrvReq *> reqs;
    size_t ws_off = 0, ws_bytes = 0;  // its workspace in the arena
    bool busy = false;
};

static bool compatible(const SrvReq *a, const SrvReq *b) {
    return a->pool.key_type == b->pool.key_type && a->pool.flags == b->pool.flags && a->M == b->M && a->K == b->K &&
           !a->solo && !b->solo;
}

// First-fit allocator over the arena's byte range (256-byte granules).
struct ArenaMap {
    std::map<size_t, size_t> free_;  // offset -> length, coalesced
    void init(size_t bytes) {
        free_.clear();
        if (bytes)
            free_[0] = bytes;
    }
    size_t largest() const {
        size_t m = 0;
        for (const auto &kv : free_)
            m = std::max(m, kv.second);
        return m;
    }
    bool take(size_t bytes, size_t *off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes)
                continue;
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t at = it->first + bytes;
            free_.erase(it);
            if (rest)
                free_[at] = rest;
            return true;
        }
        return false;
    }
    void give(size_t off, size_t bytes) {
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {  // merge with the next range
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {  // and with the previous one
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

}  // namespace pbit

using namespace pbit;

struct pbit_server {
    int device = 0;
    int max_batch = 64;
    unsigned char *arena = nullptr;
    size_t arena_bytes = 0;
    ArenaMap amap;
    bool has_tune = false;
    pbit_tune tune{};
    std::vector<SrvSlot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<SrvReq *> queue;
    std::unordered_map<uint64_t, SrvReq *> reqs;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    int64_t submitted = 0, completed = 0, batches = 0, max_in_batch = 0, peak_bytes = 0, in_flight_bytes = 0;
};

namespace pbit {

// Workspace bytes of a batch of `lists` lists with `nodes` nodes in all.
static size_t batch_ws(const pbit_server *s, int64_t nodes, int32_t lists, const SrvReq *r) {
    Tune t;
    if (!resolve_tune(s->has_tune ? &s->tune : nullptr, nodes, r->pool.key_type, r->K, &t))
        return (size_t)-1;
    return bind(compute_sizes(nodes, lists, r->pool.key_type, t, device_sms()), nullptr, nullptr, nullptr);
}

// Take a batch from the head of the queue whose workspace fits the largest
// free range of the arena (lock held).  Returns an empty batch when the
// head does not fit yet: it waits for memory, and nothing overtakes it.
static std::vector<SrvReq *> take_batch(pbit_server *s, int64_t *nodes_out, size_t *ws_out) {
    std::vector<SrvReq *> b;
    if (s->queue.empty())
        return b;
    const size_t room = s->amap.largest();
    SrvReq *first = s->queue.front();
    int64_t nodes = first->n;
    size_t need = batch_ws(s, nodes, 1, first);
    if (need > room)
        return b;
    b.push_back(first);
    s->queue.pop_front();
    if (!first->solo) {
        const size_t window = 256;  // how far down the queue to look for companions
        for (size_t i = 0; i < s->queue.size() && i < window && (int)b.size() < s->max_batch;) {
            SrvReq *r = s->queue[i];
            size_t w = 0;
            if (compatible(first, r) && (w = batch_ws(s, nodes + r->n, (int32_t)b.size() + 1, r)) <= room) {
                b.push_back(r);
                nodes += r->n;
                need = w;
                s->queue.erase(s->queue.begin() + (ptrdiff_t)i);
            } else {
                ++i;
            }
        }
    }
    *nodes_out = nodes;
    *ws_out = (need + 255) & ~(size_t)255;
    return b;
}

static pbit_status launch_batch(pbit_server *s, SrvSlot &slot, const std::vector<SrvReq *> &b, int64_t nodes) {
    const SrvReq *r0 = b[0];
    const int L = (int)b.size();
    int32_t ob = 0;
    for (int i = 0; i < L; ++i) {
        ListDesc d = pool_template(&b[i]->pool);
        d.n = (int32_t)b[i]->n;
        d.root = b[i]->root;
        d.id_base = 0;
        d.out_base = ob;
        ob += d.n;
        slot.h_desc[i] = d;
    }
    Tune t;
    if (!resolve_tune(s->has_tune ? &s->tune : nullptr, nodes, r0->pool.key_type, r0->K, &t))
        return PBIT_EINVAL;
    const int sms = device_sms();
    Sizes z = compute_sizes(nodes, L, r0->pool.key_type, t, sms);
    Ctx c;
    MemsetList ms;
    if (bind(z, s->arena + slot.ws_off, &c, &ms) > slot.ws_bytes)
        return PBIT_ENOMEM;
    c.flags = r0->pool.flags;
    c.shared_pool = 0;
    c.desc_next_stride = 4;
    if (cudaMemcpyAsync(c.desc, slot.h_desc, sizeof(ListDesc) * (size_t)L, cudaMemcpyHostToDevice, slot.stream) !=
        cudaSuccess)
        return PBIT_ECUDA;
    bool small = true;  // every request short: one kernel sorts each in shared memory
    for (int i = 0; i < L; ++i)
        small &= b[i]->n <= kSmallList;
    pbit_status rc = enqueue_sort(c, ms, 1, nullptr, nullptr, nullptr, r0->M, slot.stream, sms, nullptr, small);
    if (rc != PBIT_OK)
        return rc;
    if (cudaMemcpyAsync(slot.h_out, c.status, 4, cudaMemcpyDeviceToHost, slot.stream) != cudaSuccess ||
        cudaMemcpyAsync(slot.h_out + 1, c.new_roots, 4 * (size_t)L, cudaMemcpyDeviceToHost, slot.stream) !=
            cudaSuccess ||
        cudaEventRecord(slot.ev, slot.stream) != cudaSuccess)
        return PBIT_ECUDA;
    return PBIT_OK;
}

static void serve_loop(pbit_server *s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        bool progress = false;
        // completions
        for (SrvSlot &slot : s->slots) {
            if (!slot.busy || cudaEventQuery(slot.ev) != cudaSuccess)
                continue;
            const pbit_status st = map_status(slot.h_out[0]);
            if (st == PBIT_OK || slot.reqs.size() == 1) {
                const int64_t t = now_ns();
                for (size_t i = 0; i < slot.reqs.size(); ++i) {
                    SrvReq *r = slot.reqs[i];
                    r->status = st;
                    r->new_root = st == PBIT_OK ? slot.h_out[1 + i] : -1;
                    r->done_ns = t;
                    ++s->completed;
                }
            } else {  // isolate the failing request(s): retry each alone, in order
                for (size_t i = slot.reqs.size(); i-- > 0;) {
                    slot.reqs[i]->solo = true;
                    s->queue.push_front(slot.reqs[i]);
                }
            }
            s->in_flight_bytes -= (int64_t)slot.ws_bytes;
            s->amap.give(slot.ws_off, slot.ws_bytes);
            slot.ws_bytes = 0;
            slot.reqs.clear();
            slot.busy = false;
            progress = true;
            s->cv_done.notify_all();
        }
        // admissions
        for (SrvSlot &slot : s->slots) {
            if (slot.busy || s->queue.empty())
                continue;
            int64_t nodes = 0;
            size_t need = 0;
            std::vector<SrvReq *> b = take_batch(s, &nodes, &need);
            if (b.empty())
                break;  // the head waits for memory
            size_t off = 0;
            if (!s->amap.take(need, &off)) {  // (take_batch checked the room: cannot happen)
                for (size_t i = b.size(); i-- > 0;)
                    s->queue.push_front(b[i]);
                break;
            }
            slot.ws_off = off;
            slot.ws_bytes = need;
            slot.busy = true;  // owned by this thread while the lock is released
            lk.unlock();       // launching takes a while: let submitters in
            const pbit_status rc = launch_batch(s, slot, b, nodes);
            lk.lock();
            slot.busy = false;
            if (rc != PBIT_OK) {
                s->amap.give(slot.ws_off, slot.ws_bytes);
                slot.ws_bytes = 0;
                for (SrvReq *r : b) {
                    r->status = rc;
                    r->done_ns = now_ns();
                    ++s->completed;
                }
                s->cv_done.notify_all();
                continue;
            }
            slot.reqs = b;
            slot.busy = true;
            ++s->batches;
            s->max_in_batch = std::max<int64_t>(s->max_in_batch, (int64_t)b.size());
            s->in_flight_bytes += (int64_t)slot.ws_bytes;
            s->peak_bytes = std::max(s->peak_bytes, s->in_flight_bytes);
            progress = true;
        }
        if (!progress) {
            bool any_busy = false;
            for (const SrvSlot &slot : s->slots)
                any_busy |= slot.busy;
            // idle: sleep until a submit; busy: poll the events again shortly
            s->cv_work.wait_for(lk, any_busy ? std::chrono::microseconds(20) : std::chrono::milliseconds(50));
        }
    }
}

}  // namespace pbit

extern "C" {

pbit_status pbit_serve_create(pbit_server **out, size_t mem_budget_bytes, int32_t device, int32_t streams,
                              int32_t max_batch, const pbit_tune *tune) {
    if (!out || streams < 1 || streams > 16 || max_batch < 1 || mem_budget_bytes < (1u << 20))
        return PBIT_EINVAL;
    Tune probe;
    if (tune && !resolve_tune(tune, 1 << 20, 4, 4, &probe))
        return PBIT_EINVAL;
    if (cudaSetDevice(device) != cudaSuccess)
        return PBIT_ECUDA;
    pbit_server *s = new pbit_server();
    s->device = device;
    s->max_batch = max_batch;
    if (tune) {
        s->has_tune = true;
        s->tune = *tune;
    }
    s->arena_bytes = mem_budget_bytes & ~(size_t)255;
    if (cudaMalloc((void **)&s->arena, s->arena_bytes) != cudaSuccess) {
        delete s;
        return PBIT_ENOMEM;
    }
    s->amap.init(s->arena_bytes);
    s->slots.resize((size_t)streams);
    for (int i = 0; i < streams; ++i) {
        SrvSlot &sl = s->slots[(size_t)i];
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void **)&sl.h_desc, sizeof(ListDesc) * (size_t)max_batch) != cudaSuccess ||
            cudaMallocHost((void **)&sl.h_out, 4 * (size_t)(max_batch + 1)) != cudaSuccess) {
            pbit_serve_destroy(s);
            return PBIT_ECUDA;
        }
    }
    s->worker = std::thread(serve_loop, s);
    *out = s;
    return PBIT_OK;
}

pbit_status pbit_serve_submit(pbit_server *s, const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                              uint64_t *ticket) {
    if (!s || !pool || !ticket || !check_pool(pool, M, K) || n != pool->pool_size)
        return PBIT_EINVAL;
    if (n > 0 && (root < 0 || root >= n))
        return PBIT_EBADLIST;
    if (n == 0 && root != -1)
        return PBIT_EBADLIST;
    SrvReq *r = new SrvReq();
    r->pool = *pool;
    r->root = root;
    r->n = n;
    r->M = M;
    r->K = K;
    r->submit_ns = now_ns();
    if (n > 0 && batch_ws(s, n, 1, r) > s->arena_bytes) {
        delete r;
        return PBIT_EAGAIN;  // can never fit the budget
    }
    {
        std::lock_guard<std::mutex> g(s->mu);
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        ++s->submitted;
        if (n == 0) {  // an empty list is done at once (the paper returns NULL)
            r->status = PBIT_OK;
            r->new_root = -1;
            r->done_ns = r->submit_ns;
            ++s->completed;
        } else {
            s->queue.push_back(r);
        }
    }
    s->cv_work.notify_one();
    *ticket = r->ticket;
    return PBIT_OK;
}

pbit_status pbit_serve_poll(pbit_server *s, uint64_t ticket, int32_t *new_root) {
    if (!s)
        return PBIT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return PBIT_EINVAL;
    const SrvReq *r = it->second;
    if (r->status == PBIT_OK && new_root)
        *new_root = r->new_root;
    return (pbit_status)r->status;
}

pbit_status pbit_serve_wait(pbit_server *s, uint64_t ticket, int32_t *new_root, int64_t timeout_ms) {
    if (!s)
        return PBIT_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return PBIT_EINVAL;
    const SrvReq *r = it->second;
    s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms),
                        [&] { return r->status != PBIT_EPENDING; });
    if (r->status == PBIT_OK && new_root)
        *new_root = r->new_root;
    return (pbit_status)r->status;
}

pbit_status pbit_serve_times(pbit_server *s, uint64_t ticket, int64_t *submit_ns, int64_t *done_ns) {
    if (!s)
        return PBIT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return PBIT_EINVAL;
    if (submit_ns)
        *submit_ns = it->second->submit_ns;
    if (done_ns)
        *done_ns = it->second->done_ns;
    return PBIT_OK;
}

pbit_status pbit_serve_release(pbit_server *s, uint64_t ticket) {
    if (!s)
        return PBIT_EINVAL;
    std::lock_guard<std::mutex> g(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end())
        return PBIT_EINVAL;
    if (it->second->status == PBIT_EPENDING)
        return PBIT_EPENDING;
    delete it->second;
    s->reqs.erase(it);
    return PBIT_OK;
}

void pbit_serve_stats(pbit_server *s, int64_t *out5) {
    if (!s || !out5)
        return;
    std::lock_guard<std::mutex> g(s->mu);
    out5[0] = s->submitted;
    out5[1] = s->completed;
    out5[2] = s->batches;
    out5[3] = s->max_in_batch;
    out5[4] = s->peak_bytes;
}

void pbit_serve_destroy(pbit_server *s) {
    if (!s)
        return;
    {
        std::lock_guard<std::mutex> g(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->worker.joinable())
        s->worker.join();
    for (SrvSlot &sl : s->slots) {
        if (sl.stream)
            cudaStreamSynchronize(sl.stream);
        if (sl.ev)
            cudaEventDestroy(sl.ev);
        if (sl.stream)
            cudaStreamDestroy(sl.stream);
        if (sl.h_desc)
            cudaFreeHost(sl.h_desc);
        if (sl.h_out)
            cudaFreeHost(sl.h_out);
    }
    if (s->arena)
        cudaFree(s->arena);
    for (auto &kv : s->reqs)
        delete kv.second;
    delete s;
}

}  // extern "C"
