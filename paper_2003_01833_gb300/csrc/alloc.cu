// Caching device allocator behind DevBuf.
//
// Building a tree and running a Green step need several dozen device buffers;
// cudaMalloc / cudaFree per buffer (cudaFree synchronises the device) would
// cost milliseconds per step.  Freed blocks are kept in per-(device, stream)
// free lists binned by size (8 bins per power of two, so a block is at most
// 12.5% larger than asked) and handed out again to allocations on the same
// stream: work queued on one stream runs in order, so a block released by
// earlier work on that stream is free for later work on it.  Entry points set
// the stream with AllocStream; tagi_trim_cache returns every cached block.
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tagi_internal.cuh"

namespace tagi {
namespace {

struct Key {
    int dev;
    cudaStream_t stream;
    size_t bytes;
    bool operator<(const Key& o) const
    {
        return std::tie(dev, stream, bytes) < std::tie(o.dev, o.stream, o.bytes);
    }
};

std::mutex g_mu;
std::map<Key, std::vector<void*>> g_free;
thread_local cudaStream_t t_stream = nullptr;

size_t bin_size(size_t n)
{
    if (n < 256) return 256;
    size_t p = 1;
    while ((p << 1) <= n) p <<= 1;  // p = largest power of two <= n
    const size_t step = p >= 8 ? p / 8 : 1;
    return (n + step - 1) / step * step;
}

}  // namespace

AllocStream::AllocStream(cudaStream_t s) : prev(t_stream) { t_stream = s; }
AllocStream::~AllocStream() { t_stream = prev; }

void DevBuf::release()
{
    if (p) {
        std::lock_guard<std::mutex> lk(g_mu);
        g_free[Key{dev, stream, bytes}].push_back(p);
    }
    p = nullptr;
    bytes = 0;
}

void DevBuf::ensure(size_t nbytes)
{
    if (nbytes <= bytes && p) return;
    release();
    const size_t b = bin_size(nbytes);
    int d = 0;
    TAGI_CUDA(cudaGetDevice(&d));
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_free.find(Key{d, t_stream, b});
        if (it != g_free.end() && !it->second.empty()) {
            p = it->second.back();
            it->second.pop_back();
        }
    }
    if (!p) {
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaErrorMemoryAllocation) {
            // give the cache back and retry once
            cudaGetLastError();
            trim_cache();
            e = cudaMalloc(&p, b);
        }
        if (e != cudaSuccess) {
            p = nullptr;
            throw Error(e == cudaErrorMemoryAllocation ? TAGI_ERR_OOM : TAGI_ERR_CUDA,
                        std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
    }
    bytes = b;
    dev = d;
    stream = t_stream;
}

void trim_cache()
{
    std::lock_guard<std::mutex> lk(g_mu);
    cudaDeviceSynchronize();
    for (auto& kv : g_free)
        for (void* q : kv.second) cudaFree(q);
    g_free.clear();
}

}  // namespace tagi

extern "C" tagi_status tagi_trim_cache(void)
{
    tagi::trim_cache();
    return TAGI_OK;
}
