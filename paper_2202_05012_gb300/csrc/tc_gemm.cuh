// tc_gemm.cuh -- BF16 tensor-core GEMM for the surrogate network on sm_103a:
// tcgen05.mma with FP32 accumulation in tensor memory (TMEM), operands staged
// in shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle), stages
// released through mbarriers, fused epilogues.
//
//   C[M x N] = A[M x K] * B[N x K]^T      (A, B bf16, K contiguous)
//
// A persistent CTA walks 128-row tiles of C (all N <= 256 columns each)
// with two TMEM accumulators, so the epilogue of one tile overlaps the MMAs
// of the next; blockIdx.y splits K (split-K partial products are added with
// float atomics).  Warp 0 lane 0 issues TMA loads, warp 1 owns the TMEM
// allocation and its lane 0 issues the MMAs, warps 4..11 run the epilogue
// (warps 4+q and 8+q read TMEM lanes 32q..32q+31 = rows of the tile, one
// half of the columns each).
//
// Every mbarrier wait is bounded: on expiry the CTA records an error code,
// stops issuing work, drains what it issued (again bounded), frees its TMEM
// and returns.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

namespace supa {

enum GemmEpilogue : int {
    EPI_BIAS_GELU = 0,  // z = acc + bias; store z (f32), gelu(z) (bf16) and its transpose (bf16)
    EPI_BIAS_F32 = 1,   // acc + bias -> f32
    EPI_GELU_BWD = 2,   // g = acc * gelu'(z); store g (bf16), its transpose, column sums (bias gradient)
    EPI_ATOMIC_F32 = 3, // out += acc (split-K partial products)
};

struct GemmArgs {
    int M, N, K;        // N in {64, 128, 256}; K multiple of 64
    int k_blocks_per_split;
    int epi;
    const float *bias;  // [N]
    float *out_f32;     // [M][ld] (BIAS_F32, ATOMIC_F32) or z (BIAS_GELU)
    __nv_bfloat16 *out_bf16;   // [M][ld]
    __nv_bfloat16 *outT_bf16;  // [N][ldT]
    const float *z_in;  // [M][ld] (GELU_BWD)
    float *colsum;      // [N] (GELU_BWD)
    int ld, ldT;
    int *error;         // device error word
    const unsigned *m_dev;  // optional device row count: rows >= min(M, *m_dev) are skipped
};

constexpr int kGemmStages = 4;
constexpr int kTileM = 128;
constexpr int kTileK = 64;

size_t gemm_smem_bytes(int N);
cudaError_t launch_gemm(const CUtensorMap &ta, const CUtensorMap &tb, const GemmArgs &a, int splits, cudaStream_t st);
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

// One training pass of a minibatch up to the weight gradients (train_mlp.cu):
// per 128-row tile the forward, the loss gradient and the data-gradient chain
// in one kernel.  Inputs through the x0 map ([B][64] bf16, 128-row boxes),
// weights through w1 ([256][64]), w2, w3 ([256][256]), w4 ([128][256], 128-row
// boxes), w4t ([256][128]), w3t, w2t ([256][256]) -- 256-row boxes otherwise.
struct TrainPassArgs {
    int B;                           // rows, a multiple of 128
    const float *b1, *b2, *b3, *b4;  // biases [256] x 3, [128]
    const float *y;                  // [B][60] targets
    float *Z1, *Z2, *Z3;             // [256][B] pre-activations, transposed (written)
    __nv_bfloat16 *H1T, *H2T, *H3T;  // [256][B] transposed activations (written)
    __nv_bfloat16 *G4T;              // [128][B] transposed output gradient (rows 90.. left alone)
    __nv_bfloat16 *G3T, *G2T, *G1T;  // [256][B] transposed hidden gradients (written)
    float *gb1, *gb2, *gb3, *gb4;    // bias gradients (added to)
    double *loss_sum;                // minibatch loss (added to)
    int *error;                      // device error word (|= 8: a pipeline wait expired)
};
cudaError_t launch_train_pass(const CUtensorMap &x0, const CUtensorMap &w1, const CUtensorMap &w2,
                              const CUtensorMap &w3, const CUtensorMap &w4, const CUtensorMap &w4t,
                              const CUtensorMap &w3t, const CUtensorMap &w2t, const TrainPassArgs &a, cudaStream_t st);

// Tensor map of a row-major bf16 matrix [rows][cols] (cols contiguous) read in
// boxes of 64 columns x box_rows rows with the 128-byte swizzle.
int make_bf16_map(CUtensorMap *map, const void *base, uint64_t rows, uint64_t cols, uint32_t box_rows);
// Tensor map of a row-major float32 matrix [rows][cols] with row pitch ld
// floats (ld a multiple of 4, base 16-byte aligned), written in boxes of
// 32 columns x 32 rows with the 128-byte swizzle; columns >= cols and rows
// >= rows of a box are not written.
int make_f32_store_map(CUtensorMap *map, void *base, uint64_t rows, uint64_t cols, uint64_t ld);

}  // namespace supa
