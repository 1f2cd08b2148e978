// sur_mlp.cu -- inference of the surrogate network 6 -> 256 -> 256 -> 256 ->
// 96 (90 used) in one persistent kernel: the activations of a 128-row tile
// never leave the SM.
//
// Two row tiles are in flight per CTA (slots A and B, each with its own
// 256-column accumulator in tensor memory and its own activation buffer H),
// and their layers alternate: while the epilogue warps turn slot A's layer-l
// accumulator into activations (bias, GELU, BF16, written straight into
// shared memory in the 128-byte-swizzled K-major layout the next MMA reads),
// the tensor core runs slot B's layer, and the other way round.  A slot's
// next layer starts once the epilogue has read all of its accumulator (the
// layer overwrites it).  Only the 6 inputs (24 B) and the outputs of a row
// touch HBM.
//
// Shared memory (209,920 B with alignment slack, plus the 3 KB of hidden-layer
// biases read by the epilogue):
//   X   16 KB       inputs of a tile (bf16, columns 0..15 used, K = 16), one
//                   tile at a time: the next is packed once layer 1 read it
//   H   2 x 64 KB   hidden activations of slots A and B, 4 K-blocks of 128
//                   rows x 64 columns each; a slot's output tile is staged
//                   in its H buffer and written out coalesced
//   S   2 x 32 KB   ring of weight K-blocks, TMA, in the order the MMAs use
//                   them: W1 (both slots), then per layer and slot the 4
//                   K-blocks of W2, W3 (256 rows x 64 columns) or W4 (96 rows)
// Warps: 0 TMA producer, 1 tensor-memory owner and MMA issuer, 2-3 pack the
// inputs of each tile, 4-19 epilogue (warp w reads TMEM lanes 32(w%4)..+31
// and columns 16((w-4)/4)..+15 of every K-block; 32((w-4)/4)..+31 of the
// output layer, w < 16).
//
// Every wait is bounded (about two seconds): on expiry the CTA sets the error
// word, stops, lets its TMA loads and MMAs finish (bounded), frees tensor
// memory and returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "tc_gemm.cuh"
#include "tc_prims.cuh"

namespace supa {

namespace {

using namespace tc;

constexpr int kMlpThreads = 640;
constexpr int kRows = 128;
constexpr uint32_t kXBytes = kRows * 128;    // one input tile
constexpr uint32_t kHBlk = kRows * 128;      // one K-block of H
constexpr uint32_t kHBytes = 4 * kHBlk;      // one slot's H
constexpr uint32_t kWBlk = 256 * 128;        // one K-block of a 256-row weight (a ring stage)
constexpr int kOutN = 96;                    // output-layer width
constexpr uint32_t kW4Blk = kOutN * 128;     // one K-block of W4
constexpr uint32_t oX = 0, oH = kXBytes, oS = oH + 2 * kHBytes;
constexpr uint32_t kMlpSmem = oS + 2 * kWBlk + 1024;
constexpr int kEpiWarps = 16;

// kTmaOut: the output rows are 16-byte aligned (ld a multiple of 4), and each
// epilogue warp writes its 32 x 32 output block with one TMA store (tout);
// otherwise the output tile is staged in shared memory and written out with
// coalesced plain stores by all epilogue warps together.
template <bool kTmaOut>
__global__ void __launch_bounds__(kMlpThreads, 1)
    sur_mlp_kernel(const __grid_constant__ CUtensorMap tw1, const __grid_constant__ CUtensorMap tw2,
                   const __grid_constant__ CUtensorMap tw3, const __grid_constant__ CUtensorMap tw4,
                   const __grid_constant__ CUtensorMap tout, const MlpInferArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t w_full[2];      // ring stage holds a K-block
    __shared__ __align__(8) uint64_t w_empty[2];     // the MMAs have read the stage
    __shared__ __align__(8) uint64_t x_full;         // input tile packed
    __shared__ __align__(8) uint64_t x_empty;        // layer-1 MMA has read it
    __shared__ __align__(8) uint64_t h_ready[2];     // slot: H written, accumulator read
    __shared__ __align__(8) uint64_t acc_full[2];    // slot: a layer's accumulator is final
    __shared__ __align__(8) uint64_t drain;          // all MMAs of this CTA done
    __shared__ __align__(8) uint64_t out_staged[2];  // slot: every epilogue warp read its output block
    __shared__ __align__(8) uint64_t out_done[2];    // slot: every epilogue warp wrote its share out
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float sbias[3 * 256];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int M = g.rows;
    if (g.count) M = (int)min((unsigned)M, *g.count);
    const int tiles = (M + kRows - 1) / kRows;
    if ((int)blockIdx.x >= tiles) return;
    const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    const int my_pairs = (my_tiles + 1) / 2;  // tile 2p in slot A, tile 2p+1 (if any) in slot B
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&w_full[i], 1);
            mbar_init(&w_empty[i], 1);
            mbar_init(&h_ready[i], kEpiWarps);
            mbar_init(&acc_full[i], 1);
            mbar_init(&out_staged[i], kEpiWarps);
            mbar_init(&out_done[i], kEpiWarps);
        }
        mbar_init(&x_full, 2);
        mbar_init(&x_empty, 1);
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // hidden-layer biases, read by the epilogue from shared memory (global
    // loads in the GELU loop stalled it on their latency)
    for (int i = threadIdx.x; i < 3 * 256; i += blockDim.x)
        sbias[i] = i < 256 ? g.b1[i] : i < 512 ? g.b2[i - 256] : g.b3[i - 512];
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    __syncwarp();  // lanes that ran a one-lane role rejoin: the block barrier is warp-aligned
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;  // slot X's accumulator: columns 256 X .. 256 X + 255
    volatile int *abort_v = &abort_flag;
    auto fail = [&]() {
        if (!*abort_v) atomicOr(g.error, kErrTimeout);
        *abort_v = 1;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: the weight K-blocks in the order the MMAs use them ----
            int issued = 0;
            auto load = [&](const CUtensorMap *m, int kcol, uint32_t bytes) -> bool {
                const int c = issued, s = c & 1;
                if (c >= 2 && !mbar_wait(&w_empty[s], ((c >> 1) - 1) & 1)) {
                    fail();
                    return false;
                }
                if (*abort_v) return false;
                mbar_expect_tx(&w_full[s], bytes);
                tma_load_2d(base + oS + s * kWBlk, m, kcol, 0, &w_full[s]);
                issued = c + 1;
                return true;
            };
            bool ok = true;
            for (int pr = 0; pr < my_pairs && ok && !*abort_v; ++pr) {
                const int nx = 2 * pr + 1 < my_tiles ? 2 : 1;
                ok = load(&tw1, 0, kWBlk);
                for (int layer = 2; layer <= 4 && ok; ++layer)
                    for (int x = 0; x < nx && ok; ++x)
                        for (int kb = 0; kb < 4 && ok; ++kb)
                            ok = layer == 2 ? load(&tw2, kb * 64, kWBlk)
                                 : layer == 3 ? load(&tw3, kb * 64, kWBlk)
                                              : load(&tw4, kb * 64, kW4Blk);
            }
            if (*abort_v) {
                // let the loads in flight land before the CTA exits
                for (int i = max(0, issued - 2); i < issued; ++i) mbar_wait(&w_full[i & 1], (i >> 1) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            constexpr uint32_t id256 = idesc_bf16(kRows, 256), idout = idesc_bf16(kRows, kOutN);
            const uint32_t sX = smem_u32(base + oX), sH = smem_u32(base + oH), sS = smem_u32(base + oS);
            bool ok = true;
            int wc = 0;                    // ring stages consumed
            int xc = 0;                    // input tiles consumed
            uint32_t hc[2] = {0u, 0u};     // completions of h_ready consumed, per slot
            for (int pr = 0; pr < my_pairs && ok && !*abort_v; ++pr) {
                const int nx = 2 * pr + 1 < my_tiles ? 2 : 1;
                // layer 1: K = 16 (6 inputs, zero padded), W1 from the ring, both slots
                int s = wc & 1;
                if (!mbar_wait(&w_full[s], (wc >> 1) & 1)) {
                    fail();
                    break;
                }
                for (int x = 0; x < nx && ok; ++x) {
                    // the slot's accumulator is free once the previous tile's
                    // output epilogue has read it
                    if (!mbar_wait(&x_full, xc & 1) || (pr > 0 && !mbar_wait(&out_staged[x], (pr - 1) & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    ++xc;
                    fence_after_sync();
                    mma_bf16(tmem + 256 * x, sw128_desc(sX), sw128_desc(sS + s * kWBlk), id256, 0u);
                    mma_commit(&x_empty);
                    mma_commit(&acc_full[x]);
                }
                if (!ok) break;
                mma_commit(&w_empty[s]);
                ++wc;
                // layers 2-4, alternating slots: a slot's layer starts once the
                // epilogue has read all of its previous accumulator
                for (int layer = 2; layer <= 4 && ok; ++layer) {
                    for (int x = 0; x < nx && ok; ++x) {
                        if (*abort_v || !mbar_wait(&h_ready[x], hc[x] & 1)) {
                            fail();
                            ok = false;
                            break;
                        }
                        ++hc[x];
                        const uint32_t acc = tmem + 256 * x, hx = sH + x * kHBytes;
                        for (int kb = 0; kb < 4; ++kb) {
                            s = wc & 1;
                            if (*abort_v || !mbar_wait(&w_full[s], (wc >> 1) & 1)) {
                                fail();
                                ok = false;
                                break;
                            }
                            fence_after_sync();
#pragma unroll
                            for (int k = 0; k < 4; ++k)
                                mma_bf16(acc, sw128_desc(hx + kb * kHBlk + k * 32), sw128_desc(sS + s * kWBlk + k * 32),
                                         layer == 4 ? idout : id256, (kb > 0 || k > 0) ? 1u : 0u);
                            mma_commit(&w_empty[s]);
                            ++wc;
                        }
                        if (ok) mma_commit(&acc_full[x]);
                    }
                }
            }
            // every MMA issued by this thread completes before tensor memory is freed
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
    } else if (warp < 4) {
        // ---- input packing: 6 features -> bf16, columns 6..15 zero ----
        const int tid = threadIdx.x - 64;
        for (int t = 0; t < my_tiles; ++t) {
            // warp-uniform decision (both warps of the packer take the same path)
            if (!__all_sync(0xFFFFFFFFu, !*abort_v && (t < 1 || mbar_wait(&x_empty, (t - 1) & 1)))) {
                fail();
                break;
            }
            const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * kRows;
            uint8_t *xs = base + oX;
            for (int r = tid; r < kRows; r += 64) {
                const int row = m0 + r;
                float f[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
                if (row < M) {
                    const float2 *src = reinterpret_cast<const float2 *>(g.x + (size_t)row * 6);
                    const float2 a = src[0], b = src[1], c = src[2];
                    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y; f[4] = c.x; f[5] = c.y;
                }
                *reinterpret_cast<uint4 *>(xs + sw128_offset(r, 0)) =
                    make_uint4(pack_bf16(f[0], f[1]), pack_bf16(f[2], f[3]), pack_bf16(f[4], f[5]), 0u);
                *reinterpret_cast<uint4 *>(xs + sw128_offset(r, 1)) = make_uint4(0u, 0u, 0u, 0u);
            }
            fence_smem_to_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&x_full);
        }
    } else {
        // ---- epilogue: 16 warps; warp (q, h) owns rows 32q.. and columns 16h.. of each K-block ----
        const int q = warp & 3, h = (warp - 4) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        uint32_t ac[2] = {0u, 0u};  // completions of acc_full consumed, per slot
        bool ok = true;
        for (int pr = 0; pr < my_pairs && ok; ++pr) {
            const int nx = 2 * pr + 1 < my_tiles ? 2 : 1;
            for (int layer = 1; layer <= 3 && ok; ++layer) {
                for (int x = 0; x < nx; ++x) {
                    // warp-uniform, so that the .sync.aligned TMEM loads see the whole warp
                    if (!__all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&acc_full[x], ac[x] & 1))) {
                        fail();
                        ok = false;
                        break;
                    }
                    ++ac[x];
                    fence_after_sync();
                    const uint32_t acc = tmem + 256 * x + lane_off;
                    uint8_t *hs = base + oH + x * kHBytes;
                    // the next K-block's columns load from tensor memory while
                    // this one's GELU runs
                    uint32_t rv[2][16];
                    tmem_ld16_issue(acc + h * 16, rv[0]);
                    tmem_ld_wait(rv[0]);
#pragma unroll
                    for (int kb = 0; kb < 4; ++kb) {
                        const int c0 = kb * 64 + h * 16;
                        if (kb < 3) tmem_ld16_issue(acc + c0 + 64, rv[(kb + 1) & 1]);
                        const float4 *b4 = reinterpret_cast<const float4 *>(sbias + (layer - 1) * 256 + c0);
                        const uint32_t *u = rv[kb & 1];
                        uint32_t p[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const float4 bb = b4[i];
                            p[2 * i] = gelu2_bf16(__fadd2_rn(
                                make_float2(__uint_as_float(u[4 * i]), __uint_as_float(u[4 * i + 1])),
                                make_float2(bb.x, bb.y)));
                            p[2 * i + 1] = gelu2_bf16(__fadd2_rn(
                                make_float2(__uint_as_float(u[4 * i + 2]), __uint_as_float(u[4 * i + 3])),
                                make_float2(bb.z, bb.w)));
                        }
                        uint8_t *blk = hs + kb * kHBlk;
                        *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h)) = make_uint4(p[0], p[1], p[2], p[3]);
                        *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h + 1)) =
                            make_uint4(p[4], p[5], p[6], p[7]);
                        if (kb < 3) tmem_ld_wait(rv[(kb + 1) & 1]);
                    }
                    // the next layer's MMAs overwrite the whole accumulator, so
                    // they wait for all of H: one hand-off per layer
                    fence_smem_to_async();
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&h_ready[x]);
                }
            }
            for (int x = 0; x < nx && ok; ++x) {
                if (!__all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&acc_full[x], ac[x] & 1))) {
                    fail();
                    ok = false;
                    break;
                }
                ++ac[x];
                fence_after_sync();
                const int m0 = ((int)blockIdx.x + (2 * pr + x) * (int)gridDim.x) * kRows;
                if constexpr (kTmaOut) {
                    // Output layer, TMA path: warp (q, h < 3) holds rows 32q.. and
                    // columns 32h.. of the tile; it stages them as one 4 KB block
                    // in the 128-byte-swizzled layout of tout (inside the slot's
                    // idle H buffer, its own block) and stores the block with
                    // one TMA store.  Rows past M (a ragged last tile) go out
                    // with plain stores; columns past ncols are clipped by tout.
                    // The warp arrives on out_staged once the TMA engine has
                    // read its block: the slot's next tile writes H only after
                    // the MMA issuer has seen every warp arrive.
                    const int c0 = h * 32, row0 = m0 + q * 32;
                    if (c0 < kOutN && row0 < M) {
                        float v[32];
                        tmem_ld32(tmem + 256 * x + lane_off + c0, v);
                        const float4 *b4 = reinterpret_cast<const float4 *>(g.b4 + c0);
                        if (row0 + 32 <= M) {
                            uint8_t *blk = base + oH + x * kHBytes + (h * 4 + q) * 4096;
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const float4 bb = __ldg(b4 + i);
                                *reinterpret_cast<float4 *>(blk + lane * 128 + ((i ^ (lane & 7)) << 4)) =
                                    make_float4(v[4 * i] + bb.x, v[4 * i + 1] + bb.y, v[4 * i + 2] + bb.z,
                                                v[4 * i + 3] + bb.w);
                            }
                            fence_smem_to_async();
                            __syncwarp();
                            if (lane == 0) {
                                tma_store_2d(&tout, blk, c0, row0);
                                bulk_commit();
                                bulk_wait_read_all();
                            }
                            __syncwarp();
                        } else if (row0 + lane < M) {
                            float *o = g.out + (size_t)(row0 + lane) * g.ld + c0;
#pragma unroll
                            for (int i = 0; i < 8; ++i) {
                                const float4 bb = __ldg(b4 + i);
                                const float w4[4] = {v[4 * i] + bb.x, v[4 * i + 1] + bb.y, v[4 * i + 2] + bb.z,
                                                     v[4 * i + 3] + bb.w};
                                if (c0 + 4 * i + 4 <= g.ncols)
                                    *reinterpret_cast<float4 *>(o + 4 * i) = make_float4(w4[0], w4[1], w4[2], w4[3]);
                                else
                                    for (int j = 0; j < 4 && c0 + 4 * i + j < g.ncols; ++j) o[4 * i + j] = w4[j];
                            }
                        }
                    }
                    fence_before_sync();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&out_staged[x]);
                    continue;
                }
                // Output layer, plain path: stage the 128 x 96 tile in the
                // slot's H buffer (idle now: layer 4's MMAs are done, and the
                // next tile of the slot writes H only after every warp has
                // passed out_done), then write it out row by row, coalesced.
                // Row pitch 100 floats: the float4 stores of 8 consecutive
                // rows hit distinct banks.
                float *stage = reinterpret_cast<float *>(base + oH + x * kHBytes);
                constexpr int kPitch = 100;
                const int c0 = h * 32;
                if (c0 < kOutN) {
                    float v[32];
                    tmem_ld32(tmem + 256 * x + lane_off + c0, v);
                    const float4 *b4 = reinterpret_cast<const float4 *>(g.b4 + c0);
                    float4 *dst = reinterpret_cast<float4 *>(stage + r * kPitch + c0);
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float4 bb = __ldg(b4 + i);
                        dst[i] = make_float4(v[4 * i] + bb.x, v[4 * i + 1] + bb.y, v[4 * i + 2] + bb.z,
                                             v[4 * i + 3] + bb.w);
                    }
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&out_staged[x]);
                if (!__all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&out_staged[x], pr & 1))) {
                    fail();
                    ok = false;
                    break;
                }
                const int e = (warp - 4) * 32 + lane;  // 0..511 over the epilogue warps
                const bool vec = (g.ld & 3) == 0 && ((uintptr_t)g.out & 15) == 0;
                for (int idx = e; idx < kRows * (kOutN / 4); idx += kEpiWarps * 32) {
                    const int rr = idx / (kOutN / 4), c = (idx % (kOutN / 4)) * 4;
                    if (m0 + rr >= M || c >= g.ncols) continue;
                    const float4 val = *reinterpret_cast<const float4 *>(stage + rr * kPitch + c);
                    float *o = g.out + (size_t)(m0 + rr) * g.ld + c;
                    if (vec && c + 4 <= g.ncols) {
                        *reinterpret_cast<float4 *>(o) = val;
                    } else {
                        const float w4[4] = {val.x, val.y, val.z, val.w};
                        for (int j = 0; j < 4 && c + j < g.ncols; ++j) o[j] = w4[j];
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&out_done[x]);
                if (!__all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&out_done[x], pr & 1))) {
                    fail();
                    ok = false;
                    break;
                }
            }
        }
    }

    if constexpr (kTmaOut) {
        if (warp >= 4 && lane == 0) bulk_wait_all();
    }
    __syncwarp();  // lanes that ran a one-lane role rejoin: the block barrier is warp-aligned
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(512) : "memory");
    }
}

}  // namespace

cudaError_t launch_sur_mlp(const CUtensorMap &w1, const CUtensorMap &w2, const CUtensorMap &w3,
                           const CUtensorMap &w4, const MlpInferArgs &a, cudaStream_t st) {
    if (a.rows < 0 || a.ncols < 0 || a.ncols > kOutN || a.ld < a.ncols || !a.x || !a.out || !a.error ||
        ((uintptr_t)a.x & 7))
        return cudaErrorInvalidValue;
    if (a.rows == 0) return cudaSuccess;
    // rows of a 16-byte multiple pitch at a 16-byte aligned base, whole
    // 16-byte column groups written: TMA stores (a TMA store writes a 16-byte
    // group that straddles the column bound whole)
    CUtensorMap tout{};
    const bool tma_out = (a.ld & 3) == 0 && ((uintptr_t)a.out & 15) == 0 && a.ncols > 0 && (a.ncols & 3) == 0;
    if (tma_out && make_f32_store_map(&tout, a.out, (uint64_t)a.rows, (uint64_t)a.ncols, (uint64_t)a.ld) != 0)
        return cudaErrorInvalidValue;
    auto kernel = tma_out ? sur_mlp_kernel<true> : sur_mlp_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMlpSmem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = (a.rows + kRows - 1) / kRows;
    kernel<<<std::max(1, std::min(tiles, sms)), kMlpThreads, kMlpSmem, st>>>(w1, w2, w3, w4, tout, a);
    return cudaGetLastError();
}

}  // namespace supa
