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
// not a device address.  The device address is looked up once per device and
// context (on the first call on that device, with that device current) with
// cudaGetSymbolAddress and cached together with the id of the context it
// belongs to; when the device's context has changed since (after
// cudaDeviceReset the module is loaded again and the array may move), the
// next call looks the address up again.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "supa_internal.cuh"

namespace supa {
namespace {

// Per-block totals of the scan: one entry per kScanTile showers plus one for
// the total (scan_tmp_elems), 32 KiB in all.
constexpr int kNoAllocScratch = 4096;
static __device__ __align__(256) unsigned long long g_scan_scratch[kNoAllocScratch];
constexpr int64_t kNoAllocMaxShowers = (int64_t)(kNoAllocScratch - 2) * kScanTile;
static_assert(kScanTile == 4096, "the documented limit of 16,769,024 showers assumes 4,096-shower scan tiles");
static_assert((kNoAllocMaxShowers + kScanTile - 1) / kScanTile + 1 <= kNoAllocScratch,
              "the largest accepted n must fit the scan's per-block totals into the fixed array");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
struct CachedAddr {
    unsigned long long ctx_id;  // id of the context the address belongs to
    bool valid;
    unsigned long long *addr;
};
CachedAddr g_scratch[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext *);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 with ok = false when there
// is none yet, or the driver entry points are unavailable).
unsigned long long current_ctx_id(bool &ok) {
    static CtxGetCurrentFn get_cur = nullptr;
    static CtxGetIdFn get_id = nullptr;
    static bool looked_up = false;
    ok = false;
    if (!looked_up) {
        void *f0 = nullptr, *f1 = nullptr;
        cudaDriverEntryPointQueryResult q0, q1;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0) == cudaSuccess &&
            q0 == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess) {
            get_cur = reinterpret_cast<CtxGetCurrentFn>(f0);
            get_id = reinterpret_cast<CtxGetIdFn>(f1);
        }
        looked_up = true;
    }
    if (!get_cur || !get_id) return 0;
    CUcontext ctx = nullptr;
    if (get_cur(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    unsigned long long id = 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    ok = true;
    return id;
}

}  // namespace
}  // namespace supa

using namespace supa;

extern "C" {

int supa_shower_offsets_noalloc(const uint32_t *counts_dev, int64_t n, int64_t *offsets_dev, void *stream) {
    if (!offsets_dev || (!counts_dev && n > 0))
        return set_last_error(SUPA_ERR_INVALID_ARG, "supa_shower_offsets_noalloc: null argument");
    const int64_t max_n = kNoAllocMaxShowers;
    if (n < 0 || n > max_n || scan_tmp_elems(n) > (size_t)kNoAllocScratch) {
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
        bool have_ctx = false;
        const unsigned long long id = current_ctx_id(have_ctx);
        CachedAddr &c = g_scratch[dev];
        if (!c.valid || !have_ctx || c.ctx_id != id) {
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, g_scan_scratch);
            if (e != cudaSuccess) return set_last_error(SUPA_ERR_CUDA, cudaGetErrorString(e));
            // the lookup makes the device's context current if it was not yet
            bool ok = false;
            const unsigned long long id2 = current_ctx_id(ok);
            c.addr = static_cast<unsigned long long *>(p);
            c.ctx_id = id2;
            c.valid = ok;  // without a context id the address is looked up on every call
        }
        scratch = c.addr;
    }
    // Every entry the scan reads is written earlier in the same call, so the
    // scratch needs no clearing between calls.
    e = launch_scan_counts(counts_dev, n, offsets_dev, scratch, (cudaStream_t)stream);
    if (e != cudaSuccess) return set_last_error(SUPA_ERR_CUDA, cudaGetErrorString(e));
    return SUPA_OK;
}

}  // extern "C"
