// train_mlp.cu -- the surrogate network's training pass up to the weight
// gradients, one 128-row tile at a time per CTA in one kernel: the forward
// through the four layers, the loss gradient, and the data-gradient chain
// back through layers 4, 3 and 2, with the tile's activations (and then its
// gradients) kept in shared memory as the A operand of the next tcgen05 MMA.
// Per layer and tile the tensor core takes the operand from shared memory,
// the 16 epilogue warps turn its TMEM accumulator into the next operand.
//
// Gathers its minibatch rows of x itself (one warp packs them into the input
// tile); the targets come staged by stage_targets (once an epoch) in the
// order the loss phase reads them, each warp's loads whole 512-byte runs.
// Writes what the weight-gradient GEMM and the optimiser need: every operand
// tile it builds -- the packed inputs, the activations H1..H3, the output
// gradient d out and the hidden gradients G3..G1 -- leaves shared memory
// row-major through TMA stores issued by one thread (the weight-gradient GEMM
// reads them as MN-major operands, so no transposed copy is written);
// GELU'(z) of the hidden layers (bf16, B x 256, in thread order: each warp's
// two 16-byte stores per K-block are whole 512-byte runs, read back by the
// same thread in the backward); the bias gradients (column sums) and the
// minibatch loss.  The
// per-layer launches it replaces each gave every CTA one 128-row tile and
// spent most of their 15-20 us on the latency of one tile's loads, MMAs and
// stores.
//
// Loss (mean over rows and the 30 layers), network outputs o_j, s_j, rho_j:
//   (y_j - mu_j)^2 / (2 v_j) + ln(v_j) / 2 + y_j (rho_j - R_j)^2 / 2,
//   mu_j = exp(o_j - 4), v_j = exp(s_j) + 1e-8.
//
// Shared memory (209 KB): X 16 KB (the tile's inputs, bf16, K = 64 with 6
// used), A 64 KB (activations or gradients, 4 K-blocks of 128 rows x 64
// columns, 128-byte swizzle; after the output layer it holds d out, K = 128,
// columns 90.. zero), and a 4-stage ring of 32 KB weight K-blocks -- one
// hidden layer's weights, loaded during the epilogue before the layer -- in
// the order the MMAs use them: W1, W2 (4), W3 (4), W4 (4, 128 rows), then
// for the backward W4 (2), W3 (4), W2 (4) again as MN-major B operands (the
// transposes W^T without a transposed copy: 64 rows of W, the K block, in
// four boxes of 64 columns).  The loss reads the outputs straight from TMEM.
// Warps: 0 TMA producer, 1 TMEM owner and MMA issuer, 2 TMA stores of the
// operand tiles, 3 gathers the minibatch rows of the inputs into the input
// tile, 4-19 epilogue (warp w reads TMEM lanes 32 (w % 4).. and columns
// 16 ((w - 4) / 4).. of each 64-column block).
// Two TMEM accumulators (512 columns) alternate between consecutive layers,
// and each 64-column K-block of an operand is handed to the MMA issuer (and
// to the stores) as soon as the epilogue has written it: the next layer's
// MMAs run while the epilogue finishes the current one.
// Barriers: acc_full completes once per MMA layer (7 per tile); a_ready[kb]
// once per epilogue phase (7 per tile: K-block kb of the operand is written,
// and the epilogue is past reading the accumulator before the current one);
// a_free once per phase after the stores of its operand have read shared
// memory, before the next phase overwrites it.
// Every wait is bounded; on expiry the CTA sets the error word, stops, lets
// its loads, MMAs and stores finish (bounded), frees TMEM, returns.
#include <cudaTypedefs.h>

#include <algorithm>

#include "supa_internal.cuh"
#include "tc_gemm.cuh"
#include "tc_prims.cuh"

namespace supa {

namespace {

using namespace tc;

constexpr int kTThreads = 640;  // 20 warps (5 per scheduler: 96 registers a thread)
constexpr int kTRows = 128;
constexpr int kLayersOut = 30;
constexpr int kStagedPerTile = 2048;  // float4 of staged targets per 128-row tile
constexpr uint32_t kXBytes = kTRows * 128;    // input tile
constexpr uint32_t kABlk = kTRows * 128;      // one K-block of a 128-row operand
constexpr uint32_t kABytes = 4 * kABlk;
constexpr uint32_t kStageBytes = 256 * 128;   // one weight K-block (256 rows x 64 columns)
constexpr int kRing = 4;
constexpr uint32_t oX = 0, oA = kXBytes, oS = oA + kABytes;
constexpr uint32_t kTrainSmem = oS + kRing * kStageBytes + 1024;
constexpr int kEpi = 16;
constexpr int kPhases = 7;    // epilogue phases per tile: H1, H2, H3, d out, G3, G2, G1
constexpr int kHandOff = 2;  // K-blocks per hand-off of an operand to the MMAs (1, 2 or 4)

// The weight K-block loads of one tile, in MMA order.
struct LoadPlan {
    int map;     // 0 w1, 1 w2, 2 w3, 3 w4 (K-major B operands), 4 w4, 5 w3, 6 w2 (MN-major, backward)
    int kb;      // column block
    uint32_t bytes;
};
__device__ __forceinline__ LoadPlan plan(int i) {
    if (i == 0) return {0, 0, 256 * 128};
    if (i < 5) return {1, i - 1, 256 * 128};
    if (i < 9) return {2, i - 5, 256 * 128};
    if (i < 13) return {3, i - 9, 128 * 128};
    if (i < 15) return {4, i - 13, 256 * 128};
    if (i < 19) return {5, i - 15, 256 * 128};
    return {6, i - 19, 256 * 128};
}
constexpr int kLoads = 23;

// Targets in the loss phase's thread order (layout with launch_stage_targets):
// per tile the 128 rows are read whole (30 lanes x 8 bytes a row, 16 rows of a
// warp in flight) into shared memory, then written out as the tile's 2048
// float4 in order.  Grid-stride over the tiles.
__global__ void __launch_bounds__(256) stage_targets(const float *__restrict__ y, int64_t n, int64_t i0, uint64_t a,
                                                     uint64_t c, int64_t tiles, float4 *__restrict__ yt) {
    __shared__ float rows[kTRows][2 * kLayersOut + 5];  // odd stride: the column reads below are conflict-free
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        // lane k < 16 finds the source of row warp + 8 k
        const int64_t my_src =
            (int64_t)((a * (uint64_t)(i0 + tile * kTRows + warp + 8 * (lane & 15)) + c) % (uint64_t)n);
        float2 v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int64_t src = __shfl_sync(0xFFFFFFFFu, my_src, k);
            v[k] = lane < kLayersOut ? *reinterpret_cast<const float2 *>(y + src * (2 * kLayersOut) + 2 * lane)
                                     : make_float2(0.0f, 0.0f);  // lanes 30, 31: columns 60..63 zero
        }
        __syncthreads();  // the previous tile's rows are written out
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            rows[warp + 8 * k][2 * lane] = v[k].x;
            rows[warp + 8 * k][2 * lane + 1] = v[k].y;
        }
        __syncthreads();
        float4 *out = yt + tile * kStagedPerTile;
        for (int i = threadIdx.x; i < kStagedPerTile; i += 256) {
            const int ln = i & 31, k = (i >> 5) & 3, q = (i >> 7) & 3, h = i >> 9;
            const float *row = rows[32 * q + ln] + (k < 2 ? 0 : kLayersOut) + 8 * h + 4 * (k & 1);
            out[i] = make_float4(row[0], row[1], row[2], row[3]);
        }
    }
}

__global__ void __launch_bounds__(kTThreads, 1)
    train_mlp_kernel(const __grid_constant__ TrainMapSet mp, const TrainPassArgs g) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t w_full[kRing], w_empty[kRing];
    __shared__ __align__(8) uint64_t x_full, x_empty, x_read;  // input tile: gathered, read by layer 1, stored
    __shared__ __align__(8) uint64_t acc_full;  // a layer's accumulator is final
    __shared__ __align__(8) uint64_t a_ready[4];  // K-block kb of the next operand is written
    __shared__ __align__(8) uint64_t a_free;    // the stores of that operand have read it
    __shared__ __align__(8) uint64_t drain;
    __shared__ uint32_t tmem_slot;
    __shared__ __align__(16) float sbias[3 * 256 + 128];
    __shared__ int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles = g.B / kTRows;
    if ((int)blockIdx.x >= tiles) return;
    const int my_tiles = (tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));

    if (threadIdx.x == 0) {
        for (int i = 0; i < kRing; ++i) {
            mbar_init(&w_full[i], 1);
            mbar_init(&w_empty[i], 1);
        }
        mbar_init(&x_full, 1);
        mbar_init(&x_empty, 1);
        mbar_init(&x_read, 1);
        mbar_init(&acc_full, 1);
        for (int kb = 0; kb < 4; ++kb) mbar_init(&a_ready[kb], kEpi);
        mbar_init(&a_free, 1);
        mbar_init(&drain, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    // the input tile's columns 8..63 stay zero (the gather writes columns 0..7)
    for (int i = threadIdx.x; i < kTRows * 7; i += blockDim.x)
        *reinterpret_cast<uint4 *>(base + oX + sw128_offset(i / 7, 1 + i % 7)) = make_uint4(0u, 0u, 0u, 0u);
    // the rows of x of tile t packed to bf16 into columns 0..7 of the input
    // tile (x is not written by the kernels before this one: the first tile is
    // gathered before waiting for them)
    auto gather_tile = [&](int t) {
        const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * kTRows;
        float v[4][6];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int64_t src =
                (int64_t)((g.perm_a * (uint64_t)(g.i0 + m0 + lane + 32 * k) + g.perm_c) % (uint64_t)g.n);
#pragma unroll
            for (int j = 0; j < 6; ++j) v[k][j] = __ldg(g.x + src * 6 + j);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            *reinterpret_cast<uint4 *>(base + oX + sw128_offset(lane + 32 * k, 0)) =
                make_uint4(pack_bf16(v[k][0], v[k][1]), pack_bf16(v[k][2], v[k][3]), pack_bf16(v[k][4], v[k][5]), 0u);
        fence_smem_to_async();
    };
    if (warp == 3) gather_tile(0);
    fence_smem_to_async();
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    // the earlier kernels of the stream (the last Adam update: weights and
    // biases; the last weight gradients: readers of the buffers written here)
    // are done from here on
    pdl_wait();
    pdl_trigger();
    for (int i = threadIdx.x; i < 3 * 256 + 128; i += blockDim.x)
        sbias[i] = i < 256 ? g.b1[i] : i < 512 ? g.b2[i - 256] : i < 768 ? g.b3[i - 512] : g.b4[i - 768];
    __syncwarp();  // lanes that ran a one-lane role rejoin: the block barrier is warp-aligned
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;
    volatile int *abort_v = &abort_flag;
    auto fail = [&]() {
        if (!*abort_v) atomicOr(g.error, kErrTimeout);
        *abort_v = 1;
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---- TMA producer: each tile's 23 weight K-blocks ----
            int issued = 0;
            bool ok = true;
            for (int t = 0; t < my_tiles && ok && !*abort_v; ++t) {
                for (int i = 0; i < kLoads && ok; ++i) {
                    const int c = t * kLoads + i, s = c % kRing;
                    if (c >= kRing && !mbar_wait(&w_empty[s], ((c / kRing) - 1) & 1)) {
                        fail();
                        ok = false;
                        break;
                    }
                    if (*abort_v) {
                        ok = false;
                        break;
                    }
                    const LoadPlan pl = plan(i);
                    mbar_expect_tx(&w_full[s], pl.bytes);
                    if (pl.map < 4) {
                        // forward: 64 columns (K) of all rows (N) of W
                        const CUtensorMap *m = pl.map == 0 ? &mp.w1 : pl.map == 1 ? &mp.w2 : pl.map == 2 ? &mp.w3 : &mp.w4;
                        tma_load_2d(base + oS + s * kStageBytes, m, pl.kb * 64, 0, &w_full[s]);
                    } else {
                        // backward: 64 rows (K) of W, all 256 columns (N) in four boxes
                        const CUtensorMap *m = pl.map == 4 ? &mp.w4m : pl.map == 5 ? &mp.w3m : &mp.w2m;
                        for (int j = 0; j < 4; ++j)
                            tma_load_2d(base + oS + s * kStageBytes + j * 8192, m, j * 64, pl.kb * 64, &w_full[s]);
                    }
                    issued = c + 1;
                }
            }
            if (*abort_v) {
                // let the loads in flight land before the CTA exits
                for (int i = max(0, issued - kRing); i < issued; ++i) mbar_wait(&w_full[i % kRing], (i / kRing) & 1);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---- MMA issuer ----
            constexpr uint32_t id256 = idesc_bf16(kTRows, 256), id128 = idesc_bf16(kTRows, 128);
            constexpr uint32_t id256m = idesc_bf16(kTRows, 256) | (1u << 16);  // B MN-major
            const uint32_t sX = smem_u32(base + oX), sA = smem_u32(base + oA), sS = smem_u32(base + oS);
            bool ok = true;
            uint32_t m = 0;  // MMA layers issued: layer m accumulates in TMEM columns 256 (m % 2)..
            int c = 0;       // weight stages consumed
            // one layer: `nkb` K-blocks of the operand at `a_base` against the next ring
            // stages; with `wait_op`, K-block kb waits until the epilogue of the previous
            // layer has written it (which also means that epilogue is past reading the
            // accumulator this layer overwrites)
            auto layer = [&](uint32_t a_base, int nkb, uint32_t idesc, int k_steps_first, bool wait_op,
                             bool b_mn = false) -> bool {
                const uint32_t acc = tmem + (m & 1u) * 256u;
                for (int kb = 0; kb < nkb; ++kb) {
                    if (wait_op && (*abort_v || !mbar_wait(&a_ready[kb], (m - 1) & 1))) return false;
                    const int s = c % kRing;
                    if (*abort_v || !mbar_wait(&w_full[s], (c / kRing) & 1)) return false;
                    fence_after_sync();
                    const int ks = kb == 0 ? k_steps_first : 4;
                    const uint32_t sb = sS + s * kStageBytes;
                    for (int k = 0; k < ks; ++k)
                        mma_bf16(acc, sw128_desc(a_base + kb * kABlk + k * 32),
                                 b_mn ? sw128_mn_desc(sb + k * 2048, 8192) : sw128_desc(sb + k * 32), idesc,
                                 (kb > 0 || k > 0) ? 1u : 0u);
                    mma_commit(&w_empty[s]);
                    ++c;
                }
                mma_commit(&acc_full);
                ++m;
                return true;
            };
            for (int t = 0; t < my_tiles && ok; ++t) {
                // layer 1 (K = 16: 6 inputs, zero padded) reads the input tile; its
                // accumulator is free once the previous tile's last epilogue has begun
                if (t > 0 && (*abort_v || !mbar_wait(&a_ready[0], (m - 1) & 1))) { ok = false; break; }
                if (*abort_v || !mbar_wait(&x_full, t & 1)) { ok = false; break; }
                fence_after_sync();
                ok = layer(sX, 1, id256, 1, false);
                if (!ok) break;
                mma_commit(&x_empty);
                ok = layer(sA, 4, id256, 4, true)      // layer 2
                     && layer(sA, 4, id256, 4, true)   // layer 3
                     && layer(sA, 4, id128, 4, true)   // layer 4 (128 output columns)
                     && layer(sA, 2, id256m, 4, true, true)   // d out W4: K = 128
                     && layer(sA, 4, id256m, 4, true, true)   // d H3 W3
                     && layer(sA, 4, id256m, 4, true, true);  // d H2 W2
            }
            if (!ok) fail();
            // every MMA issued by this thread completes before tensor memory is freed
            mma_commit(&drain);
            mbar_wait(&drain, 0);
        }
    } else if (warp == 2) {
        if (lane == 0) {
            // ---- stores: each phase's operand tile to its row-major matrix ----
            uint32_t n = 0;  // epilogue phases seen
            bool ok = true;
            for (int t = 0; t < my_tiles && ok; ++t) {
                const int m0 = ((int)blockIdx.x + t * (int)gridDim.x) * kTRows;
                // the packed input tile (the B operand of dW1)
                if (*abort_v || !mbar_wait(&x_full, t & 1)) {
                    ok = false;
                    break;
                }
                tma_store_2d(&mp.x0, base + oX, 0, m0);
                bulk_commit();
                bulk_wait_read_all();
                mbar_arrive(&x_read);
                for (int ph = 0; ph < kPhases && ok; ++ph, ++n) {
                    const CUtensorMap *m = ph == 0 ? &mp.h1 : ph == 1 ? &mp.h2 : ph == 2 ? &mp.h3 : ph == 3 ? &mp.g4
                                         : ph == 4 ? &mp.g3 : ph == 5 ? &mp.g2 : &mp.g1;
                    // each K-block leaves as soon as it is written (d out has two)
#pragma unroll 1
                    for (int kb = 0; kb < 4; ++kb) {
                        if (*abort_v || !mbar_wait(&a_ready[kb], n & 1)) {
                            ok = false;
                            break;
                        }
                        if (ph != 3 || kb < 2) tma_store_2d(m, base + oA + kb * kABlk, kb * 64, m0);
                    }
                    if (!ok) break;
                    bulk_commit();
                    bulk_wait_read_all();
                    mbar_arrive(&a_free);
                }
            }
            if (!ok) fail();
            // the stores complete before the CTA (and its shared memory) goes away
            bulk_wait_all();
        }
    } else if (warp == 3) {
        // ---- gather: each tile's rows of x into the input tile (the first one is there) ----
        bool ok = true;
        for (int t = 0; t < my_tiles && ok; ++t) {
            if (t > 0) {
                // the previous tile's input was read by layer 1 and by its store
                if (!__all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&x_empty, (t - 1) & 1) &&
                                                 mbar_wait(&x_read, (t - 1) & 1))) {
                    ok = false;
                    break;
                }
                gather_tile(t);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&x_full);
        }
        if (!ok) fail();
    } else if (warp >= 4) {
        // ---- epilogue: warp (q, h) owns rows 32q.. and columns 16h.. of each K-block ----
        const int q = warp & 3, h = (warp - 4) >> 2;
        const int r = q * 32 + lane;
        const uint32_t lane_off = (uint32_t)(q * 32) << 16;
        const float inv = 1.0f / (float)(g.B * kLayersOut);
        uint8_t *A = base + oA;
        int ph = 0;   // acc_full completions consumed
        int np = 0;   // phases handed off (a_free completions to come)
        bool ok = true;
        // the accumulator of the next layer is final, and the previous phase's
        // operand has been read by its stores (warp-uniform, so that the
        // .sync.aligned TMEM loads see the whole warp)
        auto wait_acc = [&]() -> bool {
            const bool w = __all_sync(0xFFFFFFFFu, !*abort_v && mbar_wait(&acc_full, ph & 1) &&
                                                       (np == 0 || mbar_wait(&a_free, (np - 1) & 1)));
            ++ph;
            fence_after_sync();
            return w;
        };
        // K-blocks up to kb of the next operand are written (and this warp is
        // past its reads of the previous accumulator): every kHandOff K-blocks,
        // one fence for the group
        auto hand_off_kb = [&](int kb) {
            if ((kb + 1) % kHandOff != 0) return;
            fence_smem_to_async();
            fence_before_sync();
            __syncwarp();
            if (lane == 0)
                for (int k = kb + 1 - kHandOff; k <= kb; ++k) mbar_arrive(&a_ready[k]);
        };
        for (int t = 0; t < my_tiles && ok; ++t) {
            const int tile = (int)blockIdx.x + t * (int)gridDim.x;
            // GELU'(z) is kept in thread order, so that each warp's stores and loads of it are
            // whole 512-byte runs: per layer and tile 64 KB, [epilogue warp][K-block][half][lane]
            // x 16 bytes (the same thread reads back what it wrote)
            const uint32_t gp_at = (uint32_t)tile * (kTRows * 256 / 8) + (uint32_t)(warp - 4) * 256u + (uint32_t)lane;
            // ---- forward: z = acc + b; GELU(z) to the operand, GELU'(z) kept for the backward ----
            for (int l = 0; l < 3 && ok; ++l) {
                if (!wait_acc()) { ok = false; break; }
                uint4 *gp = reinterpret_cast<uint4 *>(l == 0 ? g.GP1 : l == 1 ? g.GP2 : g.GP3) + gp_at;
                const uint32_t acc = tmem + lane_off + (uint32_t)(np & 1) * 256u;
                // the next K-block's accumulator columns load while this one is processed
                uint32_t raw[16], nxt[16];
                tmem_ld16_issue(acc + h * 16, raw);
                tmem_ld_wait(raw);
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    const int c0 = kb * 64 + h * 16;
                    if (kb < 3) tmem_ld16_issue(acc + c0 + 64, nxt);
                    float v[16];
                    const float *bb = sbias + l * 256 + c0;
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(raw[i]) + bb[i];
                    uint32_t p[8], d[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) gelu2_grad2_bf16(make_float2(v[2 * i], v[2 * i + 1]), p[i], d[i]);
                    uint8_t *blk = A + kb * kABlk;
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h)) = make_uint4(p[0], p[1], p[2], p[3]);
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h + 1)) = make_uint4(p[4], p[5], p[6], p[7]);
                    gp[kb * 64] = make_uint4(d[0], d[1], d[2], d[3]);
                    gp[kb * 64 + 32] = make_uint4(d[4], d[5], d[6], d[7]);
                    hand_off_kb(kb);
                    if (kb < 3) {
                        tmem_ld_wait(nxt);
#pragma unroll
                        for (int i = 0; i < 16; ++i) raw[i] = nxt[i];
                    }
                }
                ++np;
            }
            if (!ok) break;
            // ---- output layer and loss gradient: thread (q, h) takes row r and layers
            //      j = 8h .. 8h + 7 (< 30), its outputs o_j, s_j, rho_j read from TMEM, and
            //      writes d out (bf16) into the A buffer as the operand of d out W4 ----
            {
                const int j0 = 8 * h, nj = h < 3 ? 8 : kLayersOut - 24;
                // the targets load while the output layer's MMAs run: staged in thread
                // order, each warp's four loads are whole 512-byte runs
                const float4 *yt = g.yt + (size_t)tile * kStagedPerTile + (size_t)((h * 4 + q) * 4) * 32 + lane;
                const float4 ya = yt[0], yb = yt[32], yc = yt[64], yd = yt[96];
                const float yv[8] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
                const float yr[8] = {yc.x, yc.y, yc.z, yc.w, yd.x, yd.y, yd.z, yd.w};
                if (!wait_acc()) { ok = false; break; }
                const uint32_t acc = tmem + lane_off + (uint32_t)(np & 1) * 256u;
                float om[8], os[8], orh[8];
                tmem_ld8x3(acc + j0, acc + kLayersOut + j0, acc + 2 * kLayersOut + j0, om, os, orh);
                float gd[16], gr[8];  // d out of the means and log-variances, of the distances
                float l = 0.0f;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    gd[i] = gd[8 + i] = gr[i] = 0.0f;
                    if (i < nj) {
                        const int j = j0 + i;
                        // hardware exp2 / log2 based exp and log: a relative error of a few
                        // ulp, far below the BF16 rounding of the gradient
                        const float mu = __expf(om[i] + sbias[768 + j] - kMuShift);
                        const float es = __expf(os[i] + sbias[768 + kLayersOut + j]);
                        const float dr = orh[i] + sbias[768 + 2 * kLayersOut + j] - yr[i];
                        const float res = yv[i] - mu;
                        const float vv = es + kVarFloor;
                        const float iv = __frcp_rn(vv);
                        l += 0.5f * (res * res * iv + __logf(vv) + yv[i] * dr * dr);
                        gd[i] = -res * iv * mu * inv;
                        gd[8 + i] = 0.5f * es * iv * (1.0f - res * res * iv) * inv;
                        gr[i] = yv[i] * dr * inv;
                    }
                }
                // d out into the operand: row r, columns j, 30 + j, 60 + j (2-byte stores);
                // the padding columns 90..127 are zeroed by the h = 3 threads
                uint8_t *Arow = A;
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    if (i < nj) {
#pragma unroll
                        for (int w3 = 0; w3 < 3; ++w3) {
                            const int col = w3 * kLayersOut + j0 + i;
                            const float v = w3 == 0 ? gd[i] : w3 == 1 ? gd[8 + i] : gr[i];
                            *reinterpret_cast<__nv_bfloat16 *>(Arow + (col >> 6) * kABlk +
                                                               sw128_offset(r, (col & 63) >> 3) + (col & 7) * 2) =
                                __float2bfloat16_rn(v);
                        }
                    }
                }
                if (h == 3) {
                    uint8_t *blk = Arow + kABlk;  // columns 64..127
#pragma unroll
                    for (int col = 90; col < 96; ++col)
                        *reinterpret_cast<__nv_bfloat16 *>(blk + sw128_offset(r, (col - 64) >> 3) + (col & 7) * 2) =
                            __float2bfloat16_rn(0.0f);
#pragma unroll
                    for (int u = 4; u < 8; ++u) *reinterpret_cast<uint4 *>(blk + sw128_offset(r, u)) = make_uint4(0u, 0u, 0u, 0u);
                }
                // bias gradient of the output layer: column sums over the warp's rows
                const float s16 = warp_column_sums<16>(gd, lane);
                const float s8 = warp_column_sums<8>(gr, lane);
                if (lane < 16 && (lane & 7) < nj)
                    atomicAdd(&g.gb4[(lane < 8 ? 0 : kLayersOut) + j0 + (lane & 7)], s16);
                if (lane < 8 && lane < nj) atomicAdd(&g.gb4[2 * kLayersOut + j0 + lane], s8);
#pragma unroll
                for (int o2 = 16; o2 > 0; o2 >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o2);
                if (lane == 0) atomicAdd(g.loss_sum, (double)l / (double)(g.B * kLayersOut));
            }
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) hand_off_kb(kb);
            ++np;
            // ---- backward: g = acc * GELU'(z), to the operand, column sums ----
            for (int l = 2; l >= 0 && ok; --l) {
                const uint4 *gpv = reinterpret_cast<const uint4 *>(l == 0 ? g.GP1 : l == 1 ? g.GP2 : g.GP3) + gp_at;
                float *gb = l == 0 ? g.gb1 : l == 1 ? g.gb2 : g.gb3;
                if (!wait_acc()) { ok = false; break; }
                // GELU'(z) and the accumulator columns of the next K-block load
                // while this one is processed
                uint4 gp0 = gpv[0], gp1 = gpv[32];
                const uint32_t acc = tmem + lane_off + (uint32_t)(np & 1) * 256u;
                uint32_t raw[16], nxt[16];
                tmem_ld16_issue(acc + h * 16, raw);
                tmem_ld_wait(raw);
#pragma unroll
                for (int kb = 0; kb < 4; ++kb) {
                    const int c0 = kb * 64 + h * 16;
                    uint4 np0 = gp0, np1 = gp1;
                    if (kb < 3) {
                        tmem_ld16_issue(acc + c0 + 64, nxt);
                        np0 = gpv[64 * (kb + 1)];
                        np1 = gpv[64 * (kb + 1) + 32];
                    }
                    float d[16];
                    const uint32_t gw[8] = {gp0.x, gp0.y, gp0.z, gp0.w, gp1.x, gp1.y, gp1.z, gp1.w};
                    uint32_t p[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float2 s = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&gw[i]));
                        d[2 * i] = __uint_as_float(raw[2 * i]) * s.x;
                        d[2 * i + 1] = __uint_as_float(raw[2 * i + 1]) * s.y;
                        p[i] = pack_bf16(d[2 * i], d[2 * i + 1]);
                    }
                    uint8_t *blk = A + kb * kABlk;
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h)) = make_uint4(p[0], p[1], p[2], p[3]);
                    *reinterpret_cast<uint4 *>(blk + sw128_offset(r, 2 * h + 1)) = make_uint4(p[4], p[5], p[6], p[7]);
                    // column sums over the warp's 32 rows (bias gradient)
                    const float cs = warp_column_sums<16>(d, lane);
                    if (lane < 16) atomicAdd(&gb[c0 + lane], cs);
                    hand_off_kb(kb);
                    if (kb < 3) {
                        tmem_ld_wait(nxt);
#pragma unroll
                        for (int i = 0; i < 16; ++i) raw[i] = nxt[i];
                        gp0 = np0;
                        gp1 = np1;
                    }
                }
                ++np;
            }
        }
        if (!ok) fail();
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

cudaError_t launch_stage_targets(const float *y, int64_t n, int64_t i0, uint64_t a, uint64_t c, int64_t tiles,
                                 float4 *yt, cudaStream_t st) {
    if (tiles < 1 || n < 1) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)sms * 8);
    stage_targets<<<(unsigned)grid, 256, 0, st>>>(y, n, i0, a, c, tiles, yt);
    return cudaGetLastError();
}

cudaError_t launch_train_pass(const TrainMapSet &maps, const TrainPassArgs &a, cudaStream_t st) {
    if (a.B < kTRows || a.B % kTRows) return cudaErrorInvalidValue;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaFuncSetAttribute(train_mlp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e != cudaSuccess) return e;
    const int tiles = a.B / kTRows;
    return launch_pdl(train_mlp_kernel, dim3(std::min(tiles, sms)), dim3(kTThreads), kTrainSmem, st, maps, a);
}

}  // namespace supa
