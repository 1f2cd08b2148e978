// tc_gemm.cu -- tcgen05 / TMA BF16 GEMM with fused epilogues (see tc_gemm.cuh).
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_prims.cuh"

namespace supa {

namespace {

using namespace tc;

// Warp roles: 0 issues TMA loads, 1 owns tensor memory and issues the MMAs,
// 4..11 run the epilogue (warps 4+q and 8+q read TMEM lanes 32q..32q+31, one
// half of the columns each); 2 and 3 only take part in the block barriers.
constexpr int kGemmThreads = 384;

template <int N>
__global__ void __launch_bounds__(kGemmThreads, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, const GemmArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kGemmStages];
    __shared__ __align__(8) uint64_t empty_bar[kGemmStages];
    __shared__ __align__(8) uint64_t done_bar[2];   // accumulator b holds a finished tile
    __shared__ __align__(8) uint64_t free_bar[2];   // the epilogue has read accumulator b
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    constexpr uint32_t kABytes = kTileM * 128;
    constexpr uint32_t kBBytes = N * 128;
    constexpr uint32_t kStage = kABytes + kBBytes;
    constexpr uint32_t kCols = 2 * N;  // two accumulators; a power of two >= 32

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // rows present: M, or fewer when a device-side count says so; a CTA with
    // no tile leaves before touching barriers or tensor memory
    int M = g.M;
    if (g.m_dev) M = (int)min((unsigned)M, *g.m_dev);
    const int tiles = (M + kTileM - 1) / kTileM;
    if ((int)blockIdx.x >= tiles) return;
    const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int kb0 = blockIdx.y * g.k_blocks_per_split;
    const int nkb = min(g.k_blocks_per_split, g.K / kTileK - kb0);
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&done_bar[b], 1);
            mbar_init(&free_bar[b], 8);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(kCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = tmem_slot;
    volatile int *abort_v = &abort_flag;

    int issued = 0;
    if (warp == 0 && lane == 0 && nkb > 0) {
        // TMA producer: one stage = A tile (128 x 64) + B tile (N x 64)
        for (int t = 0; t < my_tiles && !*abort_v; ++t) {
            const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * kTileM;
            for (int kb = 0; kb < nkb; ++kb) {
                const int c = t * nkb + kb, s = c % kGemmStages;
                if (c >= kGemmStages && !mbar_wait(&empty_bar[s], ((c / kGemmStages) - 1) & 1)) {
                    *abort_v = 1;
                    break;
                }
                if (*abort_v) break;
                uint8_t *sa = base + s * kStage;
                mbar_expect_tx(&full_bar[s], kStage);
                tma_load_2d(sa, &ta, (kb0 + kb) * kTileK, m0, &full_bar[s]);
                tma_load_2d(sa + kABytes, &tb, (kb0 + kb) * kTileK, 0, &full_bar[s]);
                issued = c + 1;
            }
        }
    } else if (warp == 1 && lane == 0 && nkb > 0) {
        // MMA issuer: 4 MMAs of K = 16 per stage into accumulator t % 2
        constexpr uint32_t idesc = idesc_bf16(kTileM, N);
        for (int t = 0; t < my_tiles && !*abort_v; ++t) {
            const int b = t & 1;
            if (t >= 2 && !mbar_wait(&free_bar[b], ((t >> 1) - 1) & 1)) {
                *abort_v = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            const uint32_t acc = tmem + (uint32_t)(b * N);
            for (int kb = 0; kb < nkb; ++kb) {
                const int c = t * nkb + kb, s = c % kGemmStages;
                if (*abort_v || !mbar_wait(&full_bar[s], (c / kGemmStages) & 1)) {
                    *abort_v = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
                const uint32_t sa = smem_u32(base + s * kStage);
#pragma unroll
                for (int k = 0; k < kTileK / 16; ++k)
                    mma_bf16(acc, sw128_desc(sa + k * 32), sw128_desc(sa + kABytes + k * 32), idesc,
                             (kb > 0 || k > 0) ? 1u : 0u);
                mma_commit(&empty_bar[s]);
            }
            mma_commit(&done_bar[b]);
        }
    } else if (warp >= 4) {
        // ---- epilogue: one tile at a time, accumulators alternate ----
        const int quarter = warp & 3, half = (warp - 4) >> 2;
        for (int t = 0; t < my_tiles; ++t) {
            const int b = t & 1;
            // warp-uniform, so that the .sync.aligned TMEM loads see the whole warp
            const bool ok =
                __all_sync(0xFFFFFFFFu, nkb > 0 && !*abort_v && mbar_wait(&done_bar[b], (t >> 1) & 1) && !*abort_v);
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) {
                if (lane == 0 && nkb > 0) atomicOr(g.error, kErrTimeout);
                *abort_v = 1;
                break;
            }
            const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * kTileM;
            const int row = m0 + quarter * 32 + lane;
            const bool live = row < M;
            const uint32_t lane_addr = tmem + (uint32_t)(b * N) + ((uint32_t)(quarter * 32) << 16);
#pragma unroll 1
            for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 32) {
                float v[32];
                tmem_ld32(lane_addr + c0, v);
                if (g.epi == EPI_ATOMIC_F32) {
                    // split-K partial products: vector reductions of 4 floats
                    if (live) {
                        float *o = g.out_f32 + (size_t)row * g.ld + c0;
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(o + 4 * j),
                                         "f"(v[4 * j]), "f"(v[4 * j + 1]), "f"(v[4 * j + 2]), "f"(v[4 * j + 3])
                                         : "memory");
                    }
                } else if (g.epi == EPI_BIAS_F32) {
                    if (live) {
                        float4 *o = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            o[j] = make_float4(v[4 * j] + g.bias[c0 + 4 * j], v[4 * j + 1] + g.bias[c0 + 4 * j + 1],
                                               v[4 * j + 2] + g.bias[c0 + 4 * j + 2],
                                               v[4 * j + 3] + g.bias[c0 + 4 * j + 3]);
                    }
                } else if (g.epi == EPI_BIAS_GELU) {
                    float h[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        v[j] += g.bias[c0 + j];
                        h[j] = gelu(v[j]);
                    }
                    if (live) {
                        float4 *z = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            z[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        uint4 *o = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = make_uint4(pack_bf16(h[8 * j], h[8 * j + 1]), pack_bf16(h[8 * j + 2], h[8 * j + 3]),
                                              pack_bf16(h[8 * j + 4], h[8 * j + 5]),
                                              pack_bf16(h[8 * j + 6], h[8 * j + 7]));
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            g.outT_bf16[(size_t)(c0 + j) * g.ldT + row] = __float2bfloat16_rn(h[j]);
                    }
                } else if (g.epi == EPI_GELU_BWD) {
                    float d[32];
                    if (live) {
                        const float4 *zi = reinterpret_cast<const float4 *>(g.z_in + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j) {
                            const float4 z = zi[j];
                            d[4 * j] = v[4 * j] * gelu_grad(z.x);
                            d[4 * j + 1] = v[4 * j + 1] * gelu_grad(z.y);
                            d[4 * j + 2] = v[4 * j + 2] * gelu_grad(z.z);
                            d[4 * j + 3] = v[4 * j + 3] * gelu_grad(z.w);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) d[j] = 0.0f;
                    }
                    if (live) {
                        uint4 *o = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = make_uint4(pack_bf16(d[8 * j], d[8 * j + 1]), pack_bf16(d[8 * j + 2], d[8 * j + 3]),
                                              pack_bf16(d[8 * j + 4], d[8 * j + 5]),
                                              pack_bf16(d[8 * j + 6], d[8 * j + 7]));
#pragma unroll
                        for (int j = 0; j < 32; ++j)
                            g.outT_bf16[(size_t)(c0 + j) * g.ldT + row] = __float2bfloat16_rn(d[j]);
                    }
                    // column sums over the 32 rows of this warp (bias gradient):
                    // a butterfly that halves the columns a lane keeps at every
                    // step, so lane j ends with the sum of column j
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) {
                        const bool upper = (lane & o) != 0;
#pragma unroll
                        for (int i = 0; i < o; ++i) {
                            const float give = upper ? d[i] : d[i + o];
                            const float keep = upper ? d[i + o] : d[i];
                            d[i] = keep + __shfl_xor_sync(0xFFFFFFFFu, give, o);
                        }
                    }
                    atomicAdd(&g.colsum[c0 + lane], d[0]);
                }
            }
            // hand the accumulator back to the MMA issuer
            asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&free_bar[b]);
        }
    }

    // drain TMA loads still in flight after an abort (bounded), then free TMEM
    if (warp == 0 && lane == 0 && *abort_v)
        for (int i = max(0, issued - kGemmStages); i < issued; ++i)
            mbar_wait(&full_bar[i % kGemmStages], (i / kGemmStages) & 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    if (warp == 1) {
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols) : "memory");
    }
}

template <int N>
cudaError_t launch_n(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &a, int splits, cudaStream_t st) {
    const size_t smem = gemm_smem_bytes(N);
    cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // persistent over M tiles: at most one CTA per SM per K split
    const int tiles = (a.M + kTileM - 1) / kTileM;
    dim3 grid(std::min(tiles, std::max(1, sms / splits)), splits);
    tc_gemm_kernel<N><<<grid, kGemmThreads, smem, st>>>(ta, tb, a);
    return cudaGetLastError();
}

}  // namespace

size_t gemm_smem_bytes(int N) { return (size_t)kGemmStages * (kTileM * 128 + N * 128) + 1024; }

cudaError_t launch_gemm(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &a, int splits, cudaStream_t st) {
    if (a.K % kTileK != 0 || a.M < 1 || splits < 1) return cudaErrorInvalidValue;
    switch (a.N) {
        case 64: return launch_n<64>(ta, tb, a, splits, st);
        case 128: return launch_n<128>(ta, tb, a, splits, st);
        case 256: return launch_n<256>(ta, tb, a, splits, st);
        default: return cudaErrorInvalidValue;
    }
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
