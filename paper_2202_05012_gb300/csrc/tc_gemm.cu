// tc_gemm.cu -- tcgen05 / TMA BF16 GEMM with fused epilogues (see tc_gemm.cuh).
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_gemm.cuh"

namespace supa {

namespace {

constexpr int kErrGemmTimeout = 8;
constexpr long long kWaitCycles = 4000000000ll;  // about two seconds at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Wait until the phase of parity `parity` of the barrier has completed.
// Bounded: returns false after about two seconds.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];\n" ::"r"(smem_u32(dst)),
        "l"((uint64_t)map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile stored as rows of 128
// bytes with the 128-byte swizzle (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_128B): 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address / 16
    d |= (uint64_t)1 << 16;                            // leading byte offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;                  // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;                            // descriptor version of tcgen05
    d |= (uint64_t)2 << 61;                            // 128-byte swizzle
    return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator, both
// operands K-major, M x N tile.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem_d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// erf for the GELU epilogues: the rational approximation of Abramowitz &
// Stegun, Handbook of Mathematical Functions (1964), formula 7.1.26 (after
// Hastings), |error| <= 1.5e-7 for x >= 0, extended by odd symmetry -- far
// below the BF16 resolution of the stored activations.
__device__ __forceinline__ float erf_as(float x) {
    const float a = fabsf(x);
    const float t = __frcp_rn(fmaf(0.3275911f, a, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    return copysignf(1.0f - poly * __expf(-a * a), x);
}

// GELU(z) = z Phi(z) with Phi(z) = (1 + erf(z / sqrt 2)) / 2; its derivative
// Phi(z) + z phi(z), phi the standard normal density.
__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erf_as(z * 0.70710678118654752f)); }

__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erf_as(z * 0.70710678118654752f)) + z * __expf(-0.5f * z * z) * 0.39894228040143268f;
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(bar)) : "memory");
}

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
            const bool ok = nkb > 0 && !*abort_v && mbar_wait(&done_bar[b], (t >> 1) & 1) && !*abort_v;
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
            if (!ok) {
                if (lane == 0 && nkb > 0) atomicOr(g.error, kErrGemmTimeout);
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
                    if (live)
#pragma unroll
                        for (int j = 0; j < 32; ++j) atomicAdd(&g.out_f32[(size_t)row * g.ld + c0 + j], v[j]);
                } else if (g.epi == EPI_BIAS_F32) {
                    if (live) {
                        float4 *o = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            o[j] = make_float4(v[4 * j] + g.bias[c0 + 4 * j], v[4 * j + 1] + g.bias[c0 + 4 * j + 1],
                                               v[4 * j + 2] + g.bias[c0 + 4 * j + 2],
                                               v[4 * j + 3] + g.bias[c0 + 4 * j + 3]);
                    }
                } else if (g.epi == EPI_BIAS_GELU || g.epi == EPI_GELU_ONLY) {
                    float h[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        v[j] += g.bias[c0 + j];
                        h[j] = gelu(v[j]);
                    }
                    if (live) {
                        if (g.epi == EPI_BIAS_GELU) {
                            float4 *z = reinterpret_cast<float4 *>(g.out_f32 + (size_t)row * g.ld + c0);
#pragma unroll
                            for (int j = 0; j < 8; ++j)
                                z[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                        }
                        uint4 *o = reinterpret_cast<uint4 *>(g.out_bf16 + (size_t)row * g.ld + c0);
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            o[j] = make_uint4(pack_bf16(h[8 * j], h[8 * j + 1]), pack_bf16(h[8 * j + 2], h[8 * j + 3]),
                                              pack_bf16(h[8 * j + 4], h[8 * j + 5]),
                                              pack_bf16(h[8 * j + 6], h[8 * j + 7]));
                        if (g.epi == EPI_BIAS_GELU)
#pragma unroll
                            for (int j = 0; j < 32; ++j)
                                g.outT_bf16[(size_t)(c0 + j) * g.ldT + row] = __float2bfloat16_rn(h[j]);
                    }
                } else if (g.epi == EPI_GELU_BWD) {
                    float d[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        d[j] = live ? v[j] * gelu_grad(g.z_in[(size_t)row * g.ld + c0 + j]) : 0.0f;
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
                    // column sums over the 32 rows of this warp (bias gradient)
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        float s = d[j];
#pragma unroll
                        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                        if (lane == 0) atomicAdd(&g.colsum[c0 + j], s);
                    }
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

int make_bf16_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void *fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return -1;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
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

}  // namespace supa
