// noalloc.cu -- pbit_sort_list_noalloc: the single-list sort for callers that
// cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or any allocator) when they want to
// sort: code that runs while its process's allocator has handed all device
// memory to a framework's pool, code in a latency-critical loop where an
// allocation (and its implicit synchronization) is not acceptable, or a thin C
// wrapper whose own API has no place for a workspace buffer.  This entry point
// needs no workspace from the caller: its scratch space is a fixed array in the
// library's device image, sized for lists of up to kNoAllocMaxNodes nodes.
// Every GPU that loads the library holds that array (kScratchBytes) until the
// process exits.
#include <mutex>

#include "engine.h"

namespace pbit {

constexpr int64_t kNoAllocMaxNodes = 1 << 16;   // longest list this entry point sorts
constexpr size_t kScratchBytes = 8u << 20;      // 8 MiB: the workspace of 2^16 nodes with 8-byte keys is 6.1 MiB

// The scratch array.  In host code its name is only a host-side stand-in,
// never a device address: the address a kernel may use comes from
// cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_mu;
static unsigned char *g_scratch_dev[kMaxDevices];  // device address of g_scratch, per device
static int g_sms[kMaxDevices];

// Set-up, once per device, with that device current: look up the device
// address of the scratch array and the SM count.
static pbit_status scratch_for_current_device(unsigned char **ptr, int *sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess)
        return PBIT_ECUDA;
    if (dev < 0 || dev >= kMaxDevices)
        return PBIT_EINVAL;
    std::lock_guard<std::mutex> g(g_mu);
    if (!g_scratch_dev[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p)
            return PBIT_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            return PBIT_ECUDA;
        g_sms[dev] = n;
        g_scratch_dev[dev] = static_cast<unsigned char *>(p);
    }
    *ptr = g_scratch_dev[dev];
    *sms = g_sms[dev];
    return PBIT_OK;
}

}  // namespace pbit

using namespace pbit;

extern "C" pbit_status pbit_sort_list_noalloc(const pbit_pool *pool, int32_t root, int64_t n, int32_t M, int32_t K,
                                              int32_t *new_root_host, void *stream) {
    if (!check_pool(pool, M, K) || !new_root_host || n != pool->pool_size)
        return PBIT_EINVAL;
    if (n == 0) {
        if (root != -1)
            return PBIT_EBADLIST;
        *new_root_host = -1;
        return PBIT_OK;
    }
    if (root < 0 || root >= n)
        return PBIT_EBADLIST;
    if (n > kNoAllocMaxNodes)
        return PBIT_ENOMEM;  // longer than the static scratch array allows
    unsigned char *scratch = nullptr;
    int sms = 0;
    pbit_status rc = scratch_for_current_device(&scratch, &sms);
    if (rc != PBIT_OK)
        return rc;
    Tune t;
    const pbit_tune sparse{0, 0, 32, 0};  // sparse rulers: fewer walk warps, less chunk slack to fit the array
    if (!resolve_tune(&sparse, n, pool->key_type, K, &t))
        return PBIT_EINVAL;
    const Sizes z = compute_sizes(n, 1, pool->key_type, t, sms);
    if (bind(z, nullptr, nullptr, nullptr) > kScratchBytes)
        return PBIT_ENOMEM;
    Ctx c;
    MemsetList ms;
    bind(z, scratch, &c, &ms);  // every region that must start at zero is cleared by the call itself
    c.flags = pool->flags;
    c.shared_pool = 1;
    c.desc_next_stride = pool->next_stride_bytes;
    ListDesc d = pool_template(pool);
    d.n = (int32_t)n;
    d.root = root;
    d.id_base = 0;
    d.out_base = 0;
    cudaStream_t s = (cudaStream_t)stream;
    // No timing events (creating them allocates): this call records no
    // per-kernel profile, and the profile of an earlier call is dropped so it
    // is not mistaken for this one.
    const bool prof = prof_set(false);
    prof_forget();
    rc = enqueue_sort(c, ms, 2, &d, nullptr, nullptr, M, s, sms, last_launches_slot(), n <= kSmallList);
    prof_set(prof);
    if (rc != PBIT_OK)
        return rc;
    int32_t st = -1, r = -1;  // read back into the caller's stack: no pinned buffer
    if (cudaMemcpyAsync(&st, c.status, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&r, c.new_roots, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return PBIT_ECUDA;
    rc = map_status(st);
    if (rc == PBIT_OK)
        *new_root_host = r;
    return rc;
}
