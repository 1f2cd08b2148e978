// tc_gemm.cuh -- tensor-core kernels of the surrogate network on sm_103a:
// tcgen05.mma with FP32 accumulation in tensor memory (TMEM), operands staged
// in shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle), stages
// released through mbarriers.
//
// Every mbarrier wait is bounded: on expiry the CTA records an error code,
// stops issuing work, drains what it issued (again bounded), frees its TMEM
// and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace supa {

// Weight gradients of a training minibatch, up to four problems in one launch
// (tc_gemm.cu): dW_p[M_p][N_p] += sum over the B rows r of G_p[r][m] H_p[r][n],
// G_p [B][>= M_p] and H_p [B][N_p] row-major bf16 (the layout the training
// pass writes), read through tensor maps with boxes of 64 columns x 64 rows
// (make_bf16_map(..., 64)).  Each CTA takes one (problem, 128-row block of
// dW_p, run of 64-row K-blocks) and adds its partial product to out_p with TMA
// reductions through out_maps[p] (make_f32_store_map over out_p: 32 x 32
// boxes); the runs are sized so that there is about one CTA per SM.
constexpr int kWgradMax = 4;
struct WgradProblem {
    int M;       // dW rows, a multiple of 128
    int N;       // dW columns: 64, 128 or 256
    float *out;  // [M][ld] (16-byte aligned, ld a multiple of 4), added to
    int ld;
};
struct WgradArgs {
    int B;       // rows contracted over, a multiple of 64
    int nprob;   // 1..kWgradMax
    WgradProblem p[kWgradMax];
    int *error;  // device error word (|= 8: a pipeline wait expired)
};
cudaError_t launch_weight_grads(const CUtensorMap *g_maps, const CUtensorMap *h_maps, const CUtensorMap *out_maps,
                                const WgradArgs &a, cudaStream_t st);
// One bounded mbarrier wait on a barrier nothing completes; *status (device)
// receives 1 when the wait gave up after limit_cycles, else 0.
cudaError_t launch_wait_expiry_probe(long long limit_cycles, int *status, cudaStream_t st);
// The whole network 6 -> 256 -> 256 -> 256 -> 96 (GELU after the hidden
// layers) in one persistent kernel for inference (sur_mlp.cu).
struct MlpInferArgs {
    const float *x;         // [rows][6] inputs
    int rows;               // rows present, or the capacity when `count` is set
    const unsigned *count;  // optional device row count: rows = min(rows, *count)
    const float *b1, *b2, *b3, *b4;  // biases [256], [256], [256], [96]
    float *out;             // [rows][ld] outputs, columns 0..ncols-1 (ncols <= 96) written
    int ld, ncols;
    int *error;             // device error word (|= 8: a pipeline wait expired)
};
// w1: [256][64] in boxes of 256 rows; w2, w3: [256][256] in boxes of 256
// rows; w4: [>= 96][256] in boxes of 96 rows (make_bf16_map, K contiguous).
cudaError_t launch_sur_mlp(const CUtensorMap &w1, const CUtensorMap &w2, const CUtensorMap &w3,
                           const CUtensorMap &w4, const MlpInferArgs &a, cudaStream_t st);

// Targets in the order the training pass's loss phase reads them: for tiles
// t < `tiles` of 128 rows, rows (a (i0 + 128 t + r) + c) mod n of y [n][60]
// (8-byte aligned) as 2048 float4 each at yt + 2048 t, [h][q][k][lane] for
// row 32 q + lane of the tile: k = 0, 1 the deposit fractions of layers
// 8 h + 4 k .. + 3, k = 2, 3 the mean distances of the same layers (layers
// past 29: unused).  A plain launch: it follows all earlier work on `st`.
cudaError_t launch_stage_targets(const float *y, int64_t n, int64_t i0, uint64_t a, uint64_t c, int64_t tiles,
                                 float4 *yt, cudaStream_t st);

// One training pass of a minibatch up to the weight gradients (train_mlp.cu):
// per 128-row tile the forward, the loss gradient and the data-gradient chain
// in one kernel.  The kernel gathers the minibatch rows itself; the packed
// inputs leave through the x0 map ([B][64] bf16, 128-row boxes, columns 6..
// zero: the B operand of dW1).  Weights (bf16, row-major [out][in]) through
// w1 ([256][64]), w2, w3 ([256][256]) in 256-row boxes and w4 ([128][256])
// in 128-row boxes for the forward, and through w4m, w3m, w2m (the same W4,
// W3, W2 in boxes of 64 x 64) for the backward.
// The activations H1..H3 ([B][256]) and the gradients d out (G4, [B][128],
// columns 90.. zero) and G3..G1 ([B][256]), all row-major bf16, leave through
// the store maps h1..h3, g4, g3..g1 (boxes of 64 columns x 128 rows).
struct TrainPassArgs {
    int B;                              // rows, a multiple of 128
    const float *b1, *b2, *b3, *b4;     // biases [256] x 3, [128]
    // the minibatch: row r is row (perm_a (i0 + r) + perm_c) mod n of the
    // inputs x [n][6] (gathered by the kernel) and of the targets, staged by
    // launch_stage_targets: yt is the minibatch's first tile
    const float *x;
    int64_t n, i0;
    uint64_t perm_a, perm_c;
    const float4 *yt;
    __nv_bfloat16 *GP1, *GP2, *GP3;     // B x 256 GELU'(z) of the hidden layers, in the pass's thread order (written, read back)
    float *gb1, *gb2, *gb3, *gb4;       // bias gradients (added to)
    double *loss_sum;                   // minibatch loss (added to)
    int *error;                         // device error word (|= 8: a pipeline wait expired)
};
struct TrainMapSet {
    CUtensorMap x0, w1, w2, w3, w4, w4m, w3m, w2m;  // loads (x0: store)
    CUtensorMap h1, h2, h3, g4, g3, g2, g1;         // stores
};
cudaError_t launch_train_pass(const TrainMapSet &maps, const TrainPassArgs &a, cudaStream_t st);

// Tensor map of a row-major bf16 matrix [rows][cols] (cols contiguous) read in
// boxes of 64 columns x box_rows rows with the 128-byte swizzle.
int make_bf16_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows);
// Tensor map of a row-major float32 matrix [rows][cols] with row pitch ld
// floats (ld a multiple of 4, base 16-byte aligned), written in boxes of
// 32 columns x 32 rows with the 128-byte swizzle; columns >= cols and rows
// >= rows of a box are not written.
int make_f32_store_map(CUtensorMap *map, void *base, uint64_t rows, uint64_t cols, uint64_t ld);

}  // namespace supa
