// tc_gemm.cu -- the grouped tcgen05 / TMA weight-gradient GEMM of the
// surrogate's training pass, tensor-map helpers and the bounded-wait probe
// (see tc_gemm.cuh).
#include <cudaTypedefs.h>

#include <algorithm>

#include "supa_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_prims.cuh"

namespace supa {

namespace {

using namespace tc;

// Warp roles: 0 issues TMA loads, 1 owns tensor memory and issues the MMAs,
// 4..11 run the epilogue (warps 4+q and 8+q read TMEM lanes 32q..32q+31, one
// half of the columns each); 2 and 3 only take part in the block barriers.
constexpr int kWgThreads = 384;
constexpr int kWgStages = 4;
constexpr uint32_t kWgBox = 64 * 128;          // one box: 64 rows (K) x 64 columns (M or N), bf16
constexpr uint32_t kWgA = 2 * kWgBox;          // 128 columns of G
constexpr uint32_t kWgStage = kWgA + 4 * kWgBox;  // + up to 256 columns of H

struct WgradMaps {
    CUtensorMap g[kWgradMax], h[kWgradMax], o[kWgradMax];
};
struct WgradPlan {
    int splits[kWgradMax];      // K splits of each problem
    int kbps[kWgradMax];        // K-blocks (64 rows) per split
    int item0[kWgradMax + 1];   // first CTA of each problem
};

// One CTA = one item: problem p, 128-row block mt of dW_p, K-blocks
// [kb0, kb0 + nkb) of the rows.  Per K-block a stage holds G rows r0..r0+63,
// columns 128 mt..+127 (two boxes) and H rows r0..r0+63, all N columns (N/64
// boxes); both are MN-major operands, so dW_p[m][n] = sum_r G[r][m] H[r][n]
// needs no transposed copy.
__global__ void __launch_bounds__(kWgThreads, 1)
    wgrad_kernel(const __grid_constant__ WgradMaps mp, const __grid_constant__ WgradArgs g,
                 const __grid_constant__ WgradPlan pl) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kWgStages];
    __shared__ __align__(8) uint64_t empty_bar[kWgStages];
    __shared__ __align__(8) uint64_t done_bar;
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int item = (int)blockIdx.x;
    int items = 0;
#pragma unroll
    for (int i = 1; i <= kWgradMax; ++i)
        if (i == g.nprob) items = pl.item0[i];
    if (item >= items) return;
    // this CTA's problem (constant indices, so the parameters stay in place)
    int p = 0, first = 0, splits = 1, kbps = 1, N = 64;
#pragma unroll
    for (int i = 0; i < kWgradMax; ++i)
        if (i < g.nprob && item >= pl.item0[i]) {
            p = i;
            first = pl.item0[i];
            splits = pl.splits[i];
            kbps = pl.kbps[i];
            N = g.p[i].N;
        }
    const int local = item - first;
    const int mt = local / splits, sp = local % splits;
    const int kb0 = sp * kbps;
    const int nkb = min(kbps, g.B / 64 - kb0);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kWgStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(256)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // the training pass that wrote the operands (and the Adam update that
    // cleared the gradients) are done from here on
    pdl_wait();
    pdl_trigger();
    __syncwarp();  // lanes that ran a one-lane role rejoin: the block barrier is warp-aligned
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    volatile int *abort_v = &abort_flag;

    int issued = 0;
    if (warp == 0 && lane == 0 && nkb > 0) {
        // TMA producer
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kWgStages;
            if (kb >= kWgStages && !mbar_wait(&empty_bar[s], ((kb / kWgStages) - 1) & 1)) {
                *abort_v = 1;
                break;
            }
            if (*abort_v) break;
            uint8_t *st = base + s * kWgStage;
            const int r0 = (kb0 + kb) * 64;
            mbar_expect_tx(&full_bar[s], kWgA + (uint32_t)(N / 64) * kWgBox);
            tma_load_2d(st, &mp.g[p], mt * 128, r0, &full_bar[s]);
            tma_load_2d(st + kWgBox, &mp.g[p], mt * 128 + 64, r0, &full_bar[s]);
            for (int j = 0; j < N / 64; ++j) tma_load_2d(st + kWgA + j * kWgBox, &mp.h[p], j * 64, r0, &full_bar[s]);
            issued = kb + 1;
        }
    } else if (warp == 1 && lane == 0 && nkb > 0) {
        // MMA issuer: 4 MMAs of K = 16 (16 rows: 2048 bytes of each box) per stage
        const uint32_t idesc = idesc_bf16_mn(128, N);
        bool ok = true;
        for (int kb = 0; kb < nkb; ++kb) {
            const int s = kb % kWgStages;
            if (*abort_v || !mbar_wait(&full_bar[s], (kb / kWgStages) & 1)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const uint32_t sa = smem_u32(base + s * kWgStage);
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma_bf16(tmem, sw128_mn_desc(sa + k * 2048, kWgBox), sw128_mn_desc(sa + kWgA + k * 2048, kWgBox), idesc,
                         (kb > 0 || k > 0) ? 1u : 0u);
            mma_commit(&empty_bar[s]);
        }
        if (!ok) *abort_v = 1;
        // on success done_bar completes with the last MMA; after an abort it
        // still completes, once every MMA issued has finished
        mma_commit(&done_bar);
    } else if (warp >= 4) {
        // ---- epilogue: add the partial product to dW_p with 4-float vector reductions ----
        const int q = warp & 3, h = (warp - 4) >> 2;
        const bool ok = __all_sync(0xFFFFFFFFu, nkb > 0 && mbar_wait(&done_bar, 0) && !*abort_v);
        fence_after_sync();
        if (!ok) {
            if (lane == 0 && nkb > 0) atomicOr(g.error, kErrTimeout);
            *abort_v = 1;
        } else {
            // The partial product leaves by TMA reductions: each warp stages its
            // 32-row x 32-column blocks in the 128-byte-swizzled layout of the
            // output map (16 KB a warp in the idle stage buffers) and one lane
            // adds them to dW_p -- whole lines per request, where per-thread
            // vector reductions sent one 16-byte request per row.
            const uint32_t lane_addr = tmem + ((uint32_t)(q * 32) << 16);
            uint8_t *wbuf = base + (warp - 4) * 4 * 4096;
            const int chunks = N / 64;
#pragma unroll 1
            for (int ci = 0; ci < chunks; ++ci) {
                const int c0 = h * (N / 2) + ci * 32;
                float v[32];
                tmem_ld32(lane_addr + c0, v);
                uint8_t *blk = wbuf + ci * 4096;
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<float4 *>(blk + lane * 128 + ((i ^ (lane & 7)) << 4)) =
                        make_float4(v[4 * i], v[4 * i + 1], v[4 * i + 2], v[4 * i + 3]);
            }
            fence_smem_to_async();
            __syncwarp();
            if (lane == 0) {
                for (int ci = 0; ci < chunks; ++ci)
                    tma_reduce_add_2d(&mp.o[p], wbuf + ci * 4096, h * (N / 2) + ci * 32, mt * 128 + q * 32);
                bulk_commit();
                bulk_wait_all();
            }
            __syncwarp();
        }
    }

    // drain TMA loads still in flight after an abort (bounded), then free TMEM
    if (warp == 0 && lane == 0 && *abort_v)
        for (int i = max(0, issued - kWgStages); i < issued; ++i)
            mbar_wait(&full_bar[i % kWgStages], (i / kWgStages) & 1);
    __syncwarp();  // lanes that ran a one-lane role rejoin: the block barrier is warp-aligned
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(256) : "memory");
    }
}

constexpr size_t kWgSmem = (size_t)kWgStages * kWgStage + 1024;

}  // namespace

cudaError_t launch_weight_grads(const CUtensorMap *g_maps, const CUtensorMap *h_maps, const CUtensorMap *out_maps,
                                const WgradArgs &a, cudaStream_t st) {
    if (a.B < 64 || a.B % 64 != 0 || a.nprob < 1 || a.nprob > kWgradMax) return cudaErrorInvalidValue;
    const int kbt = a.B / 64;
    WgradMaps m;
    WgradPlan pl{};
    // Work in units of one 128 x 256 K-block (a 64-column K-block is bound by
    // its loads and counts half): each problem gets K splits of about the
    // same number of units per CTA, about one CTA per SM in all.
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double units = 0.0;
    for (int i = 0; i < a.nprob; ++i) {
        const WgradProblem &q = a.p[i];
        if (q.M < 128 || q.M % 128 || (q.N != 64 && q.N != 128 && q.N != 256) || !q.out || q.ld < q.N || q.ld % 4 ||
            ((uintptr_t)q.out & 15))
            return cudaErrorInvalidValue;
        units += (q.M / 128) * (q.N == 256 ? 1.0 : 0.5);
    }
    const double per_item = std::max(1.0, std::ceil(kbt * units / std::max(1, sms - 4)));
    int items = 0;
    for (int i = 0; i < a.nprob; ++i) {
        const WgradProblem &q = a.p[i];
        const int want = std::min(kbt, (int)(per_item / (q.N == 256 ? 1.0 : 0.5)));
        const int splits = (kbt + std::max(1, want) - 1) / std::max(1, want);
        pl.splits[i] = splits;
        pl.kbps[i] = (kbt + splits - 1) / splits;
        pl.item0[i] = items;
        items += (q.M / 128) * splits;
        m.g[i] = g_maps[i];
        m.h[i] = h_maps[i];
        m.o[i] = out_maps[i];
    }
    pl.item0[a.nprob] = items;
    cudaError_t e = cudaFuncSetAttribute(wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgSmem);
    if (e != cudaSuccess) return e;
    return launch_pdl(wgrad_kernel, dim3(items), dim3(kWgThreads), kWgSmem, st, m, a, pl);
}

namespace {
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return nullptr;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    return encode;
}
}  // namespace

int make_bf16_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return -1;
    if (((uintptr_t)base & 15) || (cols * 2) % 16 || box_rows > 256 || box_rows < 1) return -2;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

int make_f32_store_map(CUtensorMap *map, void *base, uint64_t rows, uint64_t cols, uint64_t ld) {
    const PFN_cuTensorMapEncodeTiled_v12000 encode = tensor_map_encoder();
    if (!encode) return -1;
    if (((uintptr_t)base & 15) || (ld * 4) % 16 || cols < 1 || cols > ld || rows < 1) return -2;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 4};
    cuuint32_t box[2] = {32, 32};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, base, dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -3;
}

namespace {
// A wait on a barrier that nothing completes: the bounded wait must give up
// after `limit` cycles and report it (the kernel returns normally).
__global__ void wait_expiry_probe(long long limit, int *status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const bool done = mbar_wait_for(&bar, 0, limit);
    *status = done ? 0 : 1;
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_u32(&bar)) : "memory");
}
}  // namespace

cudaError_t launch_wait_expiry_probe(long long limit_cycles, int *status, cudaStream_t st) {
    wait_expiry_probe<<<1, 32, 0, st>>>(limit_cycles, status);
    return cudaGetLastError();
}

}  // namespace supa
