// vi_pool.cu -- per-process cache of the device blocks, pinned host blocks and
// streams that problem handles use.
//
// A handle allocates its tables, value ping-pong buffer, staging buffers and a
// pinned mirror of its solve state, and frees them when it is destroyed.  With
// cudaMalloc / cudaFree / cudaMallocHost that cost about 1 ms per handle on
// B300 (pinning host pages and unmapping device memory dominate), which is a
// tenth of a 4M-state solve when an application creates a handle per problem.
// Released blocks are therefore kept, up to a cap, and handed to the next
// request of a close size on the same device.  vi_release_cached_memory()
// frees all of them.
//
// The caller of a release guarantees that no queued work still uses the block
// (vi_problem_destroy synchronises the device first, as cudaFree would).

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "vi_pool.h"

namespace vip {
namespace {

struct Block {
    size_t bytes;
    int device;   // -1: pinned host memory
};

constexpr size_t kDevCap = (size_t)8 << 30;    // cached device bytes kept at most
constexpr size_t kHostCap = (size_t)256 << 20; // cached pinned bytes kept at most

std::mutex g_mu;
std::unordered_map<void *, Block> g_live;                  // handed out
std::multimap<std::pair<int, size_t>, void *> g_free;      // (device, bytes) -> block
size_t g_cached_dev = 0, g_cached_host = 0;
std::multimap<int, cudaStream_t> g_streams;                // device -> idle stream

// sizes are rounded so that shapes of similar size share blocks
size_t round_bytes(size_t b) {
    if (b == 0) return 256;
    const size_t q = b >= ((size_t)1 << 20) ? ((size_t)2 << 20) : 256;
    return (b + q - 1) / q * q;
}

// a cached block of the device (or host, device = -1) between bytes and 5/4 bytes
void *take_cached(int device, size_t bytes) {
    auto it = g_free.lower_bound({device, bytes});
    if (it == g_free.end() || it->first.first != device || it->first.second > bytes + bytes / 4) return nullptr;
    void *p = it->second;
    const size_t got = it->first.second;
    g_free.erase(it);
    (device < 0 ? g_cached_host : g_cached_dev) -= got;
    g_live[p] = Block{got, device};
    return p;
}

cudaError_t alloc_impl(void **p, size_t bytes, bool host) {
    *p = nullptr;
    int dev = -1;
    if (!host) {
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
    }
    const size_t rb = round_bytes(bytes);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if ((*p = take_cached(dev, rb)) != nullptr) return cudaSuccess;
    }
    cudaError_t e = host ? cudaMallocHost(p, rb) : cudaMalloc(p, rb);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        trim();
        e = host ? cudaMallocHost(p, rb) : cudaMalloc(p, rb);
    }
    if (e != cudaSuccess) {
        *p = nullptr;
        return e;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    g_live[*p] = Block{rb, dev};
    return cudaSuccess;
}

}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes) { return alloc_impl(p, bytes, false); }
cudaError_t host_alloc(void **p, size_t bytes) { return alloc_impl(p, bytes, true); }

void release(void *p) {
    if (!p) return;
    Block b;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_live.find(p);
        if (it == g_live.end()) return;   // not ours
        b = it->second;
        g_live.erase(it);
        size_t &cached = b.device < 0 ? g_cached_host : g_cached_dev;
        if (cached + b.bytes <= (b.device < 0 ? kHostCap : kDevCap)) {
            g_free.insert({{b.device, b.bytes}, p});
            cached += b.bytes;
            return;
        }
    }
    if (b.device < 0) {
        cudaFreeHost(p);
    } else {
        int cur = 0;
        cudaGetDevice(&cur);
        if (cur != b.device) cudaSetDevice(b.device);
        cudaFree(p);
        if (cur != b.device) cudaSetDevice(cur);
    }
}

cudaError_t stream_get(cudaStream_t *s) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_streams.find(dev);
        if (it != g_streams.end()) {
            *s = it->second;
            g_streams.erase(it);
            return cudaSuccess;
        }
    }
    return cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}

void stream_put(cudaStream_t s) {
    if (!s) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaStreamDestroy(s);
        return;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_streams.size() < 64) {
        g_streams.insert({dev, s});
        return;
    }
    cudaStreamDestroy(s);   // a bounded number of idle streams is kept
}

size_t trim() {
    std::vector<std::pair<Block, void *>> blocks;
    std::vector<std::pair<int, cudaStream_t>> streams;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (auto &kv : g_free) blocks.push_back({Block{kv.first.second, kv.first.first}, kv.second});
        g_free.clear();
        g_cached_dev = g_cached_host = 0;
        for (auto &kv : g_streams) streams.push_back(kv);
        g_streams.clear();
    }
    int cur = 0;
    cudaGetDevice(&cur);
    size_t freed = 0;
    for (auto &bp : blocks) {
        if (bp.first.device < 0) {
            cudaFreeHost(bp.second);
        } else {
            cudaSetDevice(bp.first.device);
            cudaFree(bp.second);
        }
        freed += bp.first.bytes;
    }
    for (auto &ds : streams) {
        cudaSetDevice(ds.first);
        cudaStreamDestroy(ds.second);
    }
    cudaSetDevice(cur);
    return freed;
}

size_t cached_bytes() {
    std::lock_guard<std::mutex> lk(g_mu);
    return g_cached_dev + g_cached_host;
}

}  // namespace vip

extern "C" vi_status vi_release_cached_memory(size_t *bytes_released) {
    const size_t n = vip::trim();
    if (bytes_released) *bytes_released = n;
    return VI_OK;
}

extern "C" vi_status vi_cached_memory(size_t *bytes) {
    if (!bytes) return VI_EINVAL;
    *bytes = vip::cached_bytes();
    return VI_OK;
}
