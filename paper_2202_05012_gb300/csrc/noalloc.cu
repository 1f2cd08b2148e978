// noalloc.cu -- shower offsets without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs while another
// component owns every allocation (a host framework with its own memory pool
// that forbids outside allocations), code on a path that must never block on
// the allocator, or code that may not touch the device heap at all.  For
// them this file gives one entry point that turns per-shower hit counts into
// the int64 first-hit offsets of every shower (the same exclusive scan the
// batch runs after each simulation) with its scratch -- the per-block totals
// of the scan -- in a fixed array that is part of the library's device image.
//
// That array is loaded with the module on every GPU that loads the library
// and stays there until the process exits.  Host code must not pass the
// array's name to a kernel: on the host it is only a stand-in for the symbol,
// not a device address.  The device address is looked up once per device (on
// the first call on that device, with that device current) with
// cudaGetSymbolAddress and cached.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "supa_internal.cuh"

namespace supa {
namespace {

// Per-block totals of the scan: one entry per 4,096 showers plus two.
constexpr int kNoAllocScratch = 4096;
static __device__ __align__(256) unsigned long long g_scan_scratch[kNoAllocScratch];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long *g_scratch_addr[kMaxDevices] = {};

}  // namespace
}  // namespace supa

using namespace supa;

extern "C" {

int supa_shower_offsets_noalloc(const uint32_t *counts_dev, int64_t n, int64_t *offsets_dev, void *stream) {
    if (!offsets_dev || (!counts_dev && n > 0))
        return set_last_error(SUPA_ERR_INVALID_ARG, "supa_shower_offsets_noalloc: null argument");
    const int64_t max_n = (int64_t)(kNoAllocScratch - 2) * 4096;
    if (n < 0 || n > max_n) {
        char msg[160];
        snprintf(msg, sizeof(msg),
                 "supa_shower_offsets_noalloc: n = %lld is outside [0, %lld], the size its fixed scratch covers",
                 (long long)n, (long long)max_n);
        return set_last_error(SUPA_ERR_INVALID_ARG, msg);
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return set_last_error(SUPA_ERR_CUDA, cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return set_last_error(SUPA_ERR_INVALID_ARG, "device index out of range");
    unsigned long long *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        if (!g_scratch_addr[dev]) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scan_scratch);
            if (e != cudaSuccess) return set_last_error(SUPA_ERR_CUDA, cudaGetErrorString(e));
            g_scratch_addr[dev] = static_cast<unsigned long long *>(p);
        }
        scratch = g_scratch_addr[dev];
    }
    // Every entry the scan reads is written earlier in the same call, so the
    // scratch needs no clearing between calls.
    e = launch_scan_counts(counts_dev, n, offsets_dev, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_last_error(SUPA_ERR_CUDA, cudaGetErrorString(e));
    return SUPA_OK;
}

}  // extern "C"
