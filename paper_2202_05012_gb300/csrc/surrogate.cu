// surrogate.cu -- the BF16 tensor-core surrogate network of the hybrid path
// (no counterpart in the SUPA paper): an MLP 6 -> 256 -> 256 -> 256 -> 90
// with GELU (tanh form) -- per layer j = 0..29 from the start layer the mean
// mu_j = exp(o_j - 4) (log link: output o_j) and log-variance s_j of the
// deposit fraction and the mean lateral distance rho_j of the deposits from
// the particle's axis -- trained with Adam on
//   L = mean (1/30) sum_j [(y_j - mu_j)^2 / (2 v_j) + ln(v_j) / 2
//                          + y_j (rho_j - R_j)^2 / 2],  v_j = e^s_j + 1e-8
// (targets: fractions y_j, energy-weighted mean distances R_j), evaluated
// in minibatches of `batch` rows.
//
// Layout.  The training pass (train_mlp.cu) keeps a 128-row tile's
// activations in shared memory as the next layer's operand and writes them,
// and the gradients of the backward, row-major in BF16; the weight gradients
// dW = G^T H read those as MN-major operands (tc_gemm.cu).  Each weight is
// kept in BF16 (the backward's products with W^T read W as an MN-major
// operand), next to FP32 master weights and Adam moments.  The 6 inputs are padded to 64 columns
// and the 90 outputs to 128 rows; the padding stays exactly zero (zero inputs
// and zero output gradients give zero updates).
//
// Training step: the training pass (gathers its minibatch rows, forward,
// loss gradient, data-gradient chain, bias gradients) -> the four weight
// gradients in one grouped launch -> Adam, which also refreshes the BF16
// weight copies and clears the gradients.

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "supa_internal.cuh"
#include "tc_gemm.cuh"

using namespace supa;

namespace {

constexpr int kIn = 6, kInPad = 64, kHid = 256, kOut = 90, kOutPad = 128;
constexpr int kInferLd = 96;        // outputs written by the fused inference kernel (>= kOut; 90..95 are zero)
// packed user parameter vector: W1, b1, W2, b2, W3, b3, W4, b4
constexpr int kNParams = kHid * kIn + kHid + 2 * (kHid * kHid + kHid) + kOut * kHid + kOut;

// offsets of the padded FP32 master block
struct Off {
    static constexpr size_t W1 = 0, b1 = W1 + kHid * kInPad, W2 = b1 + kHid, b2 = W2 + kHid * kHid, W3 = b2 + kHid,
                            b3 = W3 + kHid * kHid, W4 = b3 + kHid, b4 = W4 + kOutPad * kHid, total = b4 + kOutPad;
};

template <typename T>
cudaError_t dalloc(T **p, size_t n) {
    *p = nullptr;
    return cudaMalloc((void **)p, std::max<size_t>(n, 1) * sizeof(T));
}

// Adam with bias correction (c1 = 1 - beta1^t, c2 = 1 - beta2^t).
// The BF16 copies of the four weight matrices that the tensor-core kernels
// read, refreshed by the Adam update itself.
struct WeightCopies {
    int off[4];   // offset of W in the master block
    int size[4];  // rows x columns
    __nv_bfloat16 *Wb[4];
};

// inv_c1 = 1 / c1, inv_sqrt_c2 = 1 / sqrt(c2): the step is
// lr (m / c1) / (sqrt(v / c2) + eps) = lr m inv_c1 / (sqrt(v) inv_sqrt_c2 + eps).
// With avg set, the updated parameters are also added to the running
// average avg with weight w (1 / (steps averaged + 1)).  Four parameters a
// thread (n, the offsets and sizes of the weight copies multiples of 4, all
// blocks 16-byte aligned): 16-byte loads and stores.
__device__ __forceinline__ float adam_one(float &p, float &m, float &v, float g, float lr, float b1, float b2,
                                          float eps, float inv_c1, float inv_sqrt_c2) {
    m = b1 * m + (1.0f - b1) * g;
    v = b2 * v + (1.0f - b2) * g * g;
    p = p - __fdividef(lr * m * inv_c1, fmaf(sqrtf(v), inv_sqrt_c2, eps));
    return p;
}

__global__ void adam_update(float *p, float *m, float *v, float *g, int n, float lr, float b1, float b2,
                            float eps, float inv_c1, float inv_sqrt_c2, const WeightCopies wc, float *avg, float w) {
    pdl_wait();  // the weight gradients are complete
    pdl_trigger();
    const int i = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= n) return;
    const float4 gi = *reinterpret_cast<const float4 *>(g + i);
    float4 pi = *reinterpret_cast<const float4 *>(p + i), mi = *reinterpret_cast<const float4 *>(m + i),
           vi = *reinterpret_cast<const float4 *>(v + i);
    adam_one(pi.x, mi.x, vi.x, gi.x, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam_one(pi.y, mi.y, vi.y, gi.y, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam_one(pi.z, mi.z, vi.z, gi.z, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    adam_one(pi.w, mi.w, vi.w, gi.w, lr, b1, b2, eps, inv_c1, inv_sqrt_c2);
    *reinterpret_cast<float4 *>(m + i) = mi;
    *reinterpret_cast<float4 *>(v + i) = vi;
    *reinterpret_cast<float4 *>(p + i) = pi;
    *reinterpret_cast<float4 *>(g + i) = make_float4(0.0f, 0.0f, 0.0f, 0.0f);  // ready for the next minibatch
    if (avg) {
        float4 a = *reinterpret_cast<const float4 *>(avg + i);
        a = make_float4(fmaf(w, pi.x - a.x, a.x), fmaf(w, pi.y - a.y, a.y), fmaf(w, pi.z - a.z, a.z),
                        fmaf(w, pi.w - a.w, a.w));
        *reinterpret_cast<float4 *>(avg + i) = a;
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int j = i - wc.off[c];
        if (j >= 0 && j < wc.size[c]) {
            __nv_bfloat162 lo = __floats2bfloat162_rn(pi.x, pi.y), hi = __floats2bfloat162_rn(pi.z, pi.w);
            uint2 u;
            u.x = *reinterpret_cast<uint32_t *>(&lo);
            u.y = *reinterpret_cast<uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(wc.Wb[c] + j) = u;
        }
    }
}

// BF16 copy of a master weight [rows][cols].
__global__ void cast_weight(const float *W, int n, __nv_bfloat16 *Wb) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Wb[i] = __float2bfloat16_rn(W[i]);
}

}  // namespace

struct supa_surrogate {
    int B = 0;
    int t = 0;  // Adam step count
    bool grad_zero = false;  // the gradient block holds zeros (the Adam update clears it)
    bool avg_on = false;     // iterate averaging: Adam steps are added to avg
    int64_t avg_n = 0;       // steps in the average
    float *avg = nullptr;    // running average of the master parameters
    float beta1 = 0.9f, beta2 = 0.999f, eps = 1e-8f;
    float *master = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
    __nv_bfloat16 *W1b, *W2b, *W3b, *W4b;
    __nv_bfloat16 *X0, *H1, *H2, *H3, *G4, *G3, *G2, *G1;  // row-major operands of the weight gradients
    __nv_bfloat16 *GP1, *GP2, *GP3;                           // GELU'(z) of the hidden layers
    float4 *yt = nullptr;       // one minibatch's targets in the training pass's order
    float4 *yt_epoch = nullptr;  // an epoch's, staged once before its first step
    int64_t yt_epoch_tiles = 0;
    double *loss_tmp = nullptr;
    int *error = nullptr;
    TrainMapSet tm;                                  // the training pass's loads and stores
    CUtensorMap dG[kWgradMax], dH[kWgradMax];        // weight-gradient operands (64-row boxes)
    CUtensorMap dO[kWgradMax];                       // weight gradients (f32, reduced into by TMA)
    CUtensorMap mW4i;  // W4 rows 0..95 for the fused inference kernel
    std::vector<void *> allocs;
};

namespace {

int sfail(int code, const std::string &m) { return set_last_error(code, m.c_str()); }

template <typename T>
bool grab(supa_surrogate *s, T **p, size_t n) {
    if (dalloc(p, n) != cudaSuccess) return false;
    s->allocs.push_back((void *)*p);
    return true;
}

void free_all(supa_surrogate *s) {
    for (void *p : s->allocs) cudaFree(p);
    s->allocs.clear();
    cudaFree(s->yt_epoch);
    s->yt_epoch = nullptr;
    s->yt_epoch_tiles = 0;
}

int weight_copies(supa_surrogate *s, cudaStream_t st) {
    const int T = 256;
    cast_weight<<<(kHid * kInPad + T - 1) / T, T, 0, st>>>(s->master + Off::W1, kHid * kInPad, s->W1b);
    cast_weight<<<(kHid * kHid + T - 1) / T, T, 0, st>>>(s->master + Off::W2, kHid * kHid, s->W2b);
    cast_weight<<<(kHid * kHid + T - 1) / T, T, 0, st>>>(s->master + Off::W3, kHid * kHid, s->W3b);
    cast_weight<<<(kOutPad * kHid + T - 1) / T, T, 0, st>>>(s->master + Off::W4, kOutPad * kHid, s->W4b);
    return cudaGetLastError() == cudaSuccess ? SUPA_OK : SUPA_ERR_CUDA;
}

// One minibatch -- rows (a (i0 + r) + c) mod n of the inputs x [n][6] and
// targets y [n][60] -- up to the gradients in s->grad (zeroed unless the last
// Adam update left it zero) and the loss added to *s->loss_tmp: the training
// pass per 128-row tile (gather, forward, loss gradient, data-gradient chain;
// bias gradients), then dW4 = G4^T H3, dW3 = G3^T H2, dW2 = G2^T H1,
// dW1 = G1^T X0 over the rows in one grouped launch.  The targets come staged
// (launch_stage_targets) at yt, or are staged here when yt is null.
cudaError_t train_pass(supa_surrogate *s, const float *x, const float *y, int64_t n, uint64_t a, uint64_t c,
                       int64_t i0, cudaStream_t st, const float4 *yt = nullptr) {
    const int B = s->B;
    cudaError_t e = cudaSuccess;
    if (!s->grad_zero && (e = cudaMemsetAsync(s->grad, 0, Off::total * sizeof(float), st)) != cudaSuccess) return e;
    s->grad_zero = false;
    TrainPassArgs t{};
    t.B = B;
    t.b1 = s->master + Off::b1;
    t.b2 = s->master + Off::b2;
    t.b3 = s->master + Off::b3;
    t.b4 = s->master + Off::b4;
    if (!yt) {
        if ((e = launch_stage_targets(y, n, i0, a, c, B / 128, s->yt, st)) != cudaSuccess) return e;
        yt = s->yt;
    }
    t.x = x;
    t.yt = yt;
    t.n = n;
    t.i0 = i0;
    t.perm_a = a;
    t.perm_c = c;
    t.GP1 = s->GP1; t.GP2 = s->GP2; t.GP3 = s->GP3;
    t.gb1 = s->grad + Off::b1; t.gb2 = s->grad + Off::b2; t.gb3 = s->grad + Off::b3; t.gb4 = s->grad + Off::b4;
    t.loss_sum = s->loss_tmp;
    t.error = s->error;
    if ((e = launch_train_pass(s->tm, t, st)) != cudaSuccess) return e;
    WgradArgs w{};
    w.B = B;
    w.nprob = 4;
    w.p[0] = {kOutPad, kHid, s->grad + Off::W4, kHid};
    w.p[1] = {kHid, kHid, s->grad + Off::W3, kHid};
    w.p[2] = {kHid, kHid, s->grad + Off::W2, kHid};
    w.p[3] = {kHid, kInPad, s->grad + Off::W1, kInPad};
    w.error = s->error;
    return launch_weight_grads(s->dG, s->dH, s->dO, w, st);
}

int check_error_word(supa_surrogate *s) {
    int h = 0;
    if (cudaMemcpy(&h, s->error, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return SUPA_ERR_CUDA;
    if (h) return sfail(SUPA_ERR_TIMEOUT, "a tensor-core GEMM gave up waiting on its pipeline (error word " +
                                              std::to_string(h) + ")");
    return SUPA_OK;
}

// packed user vector <-> padded master block (host side)
void unpack_params(const float *p, std::vector<float> &mst) {
    mst.assign(Off::total, 0.0f);
    size_t o = 0;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c < kIn; ++c) mst[Off::W1 + r * kInPad + c] = p[o++];
    for (int r = 0; r < kHid; ++r) mst[Off::b1 + r] = p[o++];
    for (int i = 0; i < kHid * kHid; ++i) mst[Off::W2 + i] = p[o++];
    for (int r = 0; r < kHid; ++r) mst[Off::b2 + r] = p[o++];
    for (int i = 0; i < kHid * kHid; ++i) mst[Off::W3 + i] = p[o++];
    for (int r = 0; r < kHid; ++r) mst[Off::b3 + r] = p[o++];
    for (int i = 0; i < kOut * kHid; ++i) mst[Off::W4 + i] = p[o++];
    for (int r = 0; r < kOut; ++r) mst[Off::b4 + r] = p[o++];
}

void pack_params(const std::vector<float> &mst, float *p) {
    size_t o = 0;
    for (int r = 0; r < kHid; ++r)
        for (int c = 0; c < kIn; ++c) p[o++] = mst[Off::W1 + r * kInPad + c];
    for (int r = 0; r < kHid; ++r) p[o++] = mst[Off::b1 + r];
    for (int i = 0; i < kHid * kHid; ++i) p[o++] = mst[Off::W2 + i];
    for (int r = 0; r < kHid; ++r) p[o++] = mst[Off::b2 + r];
    for (int i = 0; i < kHid * kHid; ++i) p[o++] = mst[Off::W3 + i];
    for (int r = 0; r < kHid; ++r) p[o++] = mst[Off::b3 + r];
    for (int i = 0; i < kOut * kHid; ++i) p[o++] = mst[Off::W4 + i];
    for (int r = 0; r < kOut; ++r) p[o++] = mst[Off::b4 + r];
}

}  // namespace

// ---- inference over a device-counted queue (hybrid path) -----------------

namespace supa {

void surrogate_infer_free(SurInfer *inf) {
    cudaFree(inf->OUT);
    inf->OUT = nullptr;
    inf->cap = 0;
}

int surrogate_infer_init(supa_surrogate *s, int cap, SurInfer *inf) {
    (void)s;
    inf->cap = cap;
    inf->ld = kInferLd;
    if (cudaMalloc((void **)&inf->OUT, (size_t)cap * kInferLd * 4) != cudaSuccess) {
        cudaGetLastError();
        surrogate_infer_free(inf);
        return set_last_error(SUPA_ERR_OOM, "surrogate queue buffers: out of device memory");
    }
    return SUPA_OK;
}

// The fused kernel over the first min(*count_dev, cap) rows of the queue.
cudaError_t surrogate_infer_run(supa_surrogate *s, SurInfer *inf, const float *feat, const unsigned *count_dev,
                                cudaStream_t st) {
    MlpInferArgs a{};
    a.x = feat;
    a.rows = inf->cap;
    a.count = count_dev;
    a.b1 = s->master + Off::b1;
    a.b2 = s->master + Off::b2;
    a.b3 = s->master + Off::b3;
    a.b4 = s->master + Off::b4;
    a.out = inf->OUT;
    a.ld = kInferLd;
    a.ncols = kInferLd;  // all 96 columns: whole-vector stores (W4, b4 rows 90..95 are zero)
    a.error = s->error;
    return launch_sur_mlp(s->tm.w1, s->tm.w2, s->tm.w3, s->mW4i, a, st);
}

}  // namespace supa

extern "C" {

int32_t supa_surrogate_param_count(void) { return kNParams; }

int supa_surrogate_destroy(supa_surrogate *s) {
    if (!s) return SUPA_OK;
    free_all(s);
    delete s;
    return SUPA_OK;
}

int supa_surrogate_create(int32_t batch, const float *params_host, supa_surrogate **out) {
    if (!out || !params_host) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_create: null argument");
    *out = nullptr;
    if (batch < 128 || batch % 128 != 0 || batch > (1 << 20))
        return sfail(SUPA_ERR_INVALID_ARG, "batch must be a positive multiple of 128 up to 2^20");
    supa_surrogate *s = new supa_surrogate();
    s->B = batch;
    const size_t B = batch;
    bool ok = grab(s, &s->master, Off::total) && grab(s, &s->m, Off::total) && grab(s, &s->v, Off::total) &&
              grab(s, &s->grad, Off::total) && grab(s, &s->W1b, (size_t)kHid * kInPad) &&
              grab(s, &s->W2b, (size_t)kHid * kHid) && grab(s, &s->W3b, (size_t)kHid * kHid) &&
              grab(s, &s->W4b, (size_t)kOutPad * kHid) &&
              grab(s, &s->X0, B * kInPad) && grab(s, &s->H1, B * kHid) && grab(s, &s->H2, B * kHid) &&
              grab(s, &s->H3, B * kHid) && grab(s, &s->G4, B * kOutPad) && grab(s, &s->G3, B * kHid) &&
              grab(s, &s->G2, B * kHid) && grab(s, &s->G1, B * kHid) && grab(s, &s->GP1, B * kHid) &&
              grab(s, &s->GP2, B * kHid) && grab(s, &s->GP3, B * kHid) && grab(s, &s->yt, B * 16) &&
              grab(s, &s->loss_tmp, 1) &&
              grab(s, &s->avg, Off::total) &&
              grab(s, &s->error, 1);
    if (!ok) {
        supa_surrogate_destroy(s);
        return sfail(SUPA_ERR_OOM, "supa_surrogate_create: out of device memory");
    }
    // tensor maps of the training pass: the input tile and its stores in
    // 128-row boxes, the weights in boxes of all their rows (forward) and of
    // 64 x 64 (backward)
    int rc = 0;
    TrainMapSet &tm = s->tm;
    rc |= make_bf16_map(&tm.x0, s->X0, B, kInPad, 128);
    rc |= make_bf16_map(&tm.w1, s->W1b, kHid, kInPad, kHid);
    rc |= make_bf16_map(&tm.w2, s->W2b, kHid, kHid, kHid);
    rc |= make_bf16_map(&tm.w3, s->W3b, kHid, kHid, kHid);
    rc |= make_bf16_map(&tm.w4, s->W4b, kOutPad, kHid, kOutPad);
    rc |= make_bf16_map(&tm.w4m, s->W4b, kOutPad, kHid, 64);
    rc |= make_bf16_map(&tm.w3m, s->W3b, kHid, kHid, 64);
    rc |= make_bf16_map(&tm.w2m, s->W2b, kHid, kHid, 64);
    rc |= make_bf16_map(&tm.h1, s->H1, B, kHid, 128);
    rc |= make_bf16_map(&tm.h2, s->H2, B, kHid, 128);
    rc |= make_bf16_map(&tm.h3, s->H3, B, kHid, 128);
    rc |= make_bf16_map(&tm.g4, s->G4, B, kOutPad, 128);
    rc |= make_bf16_map(&tm.g3, s->G3, B, kHid, 128);
    rc |= make_bf16_map(&tm.g2, s->G2, B, kHid, 128);
    rc |= make_bf16_map(&tm.g1, s->G1, B, kHid, 128);
    rc |= make_bf16_map(&s->mW4i, s->W4b, kOutPad, kHid, kInferLd);
    // the weight gradients read the same matrices in 64-row boxes
    const __nv_bfloat16 *gsrc[kWgradMax] = {s->G4, s->G3, s->G2, s->G1};
    const __nv_bfloat16 *hsrc[kWgradMax] = {s->H3, s->H2, s->H1, s->X0};
    const int gcols[kWgradMax] = {kOutPad, kHid, kHid, kHid}, hcols[kWgradMax] = {kHid, kHid, kHid, kInPad};
    float *gout[kWgradMax] = {s->grad + Off::W4, s->grad + Off::W3, s->grad + Off::W2, s->grad + Off::W1};
    const int orows[kWgradMax] = {kOutPad, kHid, kHid, kHid};
    for (int i = 0; i < kWgradMax; ++i) {
        rc |= make_bf16_map(&s->dG[i], gsrc[i], B, gcols[i], 64);
        rc |= make_bf16_map(&s->dH[i], hsrc[i], B, hcols[i], 64);
        rc |= make_f32_store_map(&s->dO[i], gout[i], orows[i], hcols[i], hcols[i]);
    }
    if (rc != 0) {
        supa_surrogate_destroy(s);
        return sfail(SUPA_ERR_CUDA, "supa_surrogate_create: cuTensorMapEncodeTiled failed");
    }
    std::vector<float> mst;
    unpack_params(params_host, mst);
    cudaError_t e = cudaMemcpy(s->master, mst.data(), Off::total * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s->m, 0, Off::total * 4);
    if (e == cudaSuccess) e = cudaMemset(s->v, 0, Off::total * 4);
    if (e == cudaSuccess) e = cudaMemset(s->error, 0, sizeof(int));
    if (e != cudaSuccess || weight_copies(s, 0) != SUPA_OK || cudaDeviceSynchronize() != cudaSuccess) {
        supa_surrogate_destroy(s);
        return sfail(SUPA_ERR_CUDA, "supa_surrogate_create: upload failed");
    }
    *out = s;
    return SUPA_OK;
}

int supa_surrogate_get_params(supa_surrogate *s, float *params_host) {
    if (!s || !params_host) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_get_params: null argument");
    std::vector<float> mst(Off::total);
    if (cudaMemcpy(mst.data(), s->master, Off::total * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "supa_surrogate_get_params: copy failed");
    pack_params(mst, params_host);
    return SUPA_OK;
}

int supa_surrogate_gradients(supa_surrogate *s, const float *x_dev, const float *y_dev, float *grads_host,
                             double *loss_host, void *stream) {
    if (!s || !x_dev || !y_dev || !grads_host) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_gradients: null");
    if (((uintptr_t)x_dev & 3) || ((uintptr_t)y_dev & 7))
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_gradients: x must be 4-byte and y 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    if (cudaMemsetAsync(s->loss_tmp, 0, sizeof(double), st) != cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "memset failed");
    cudaError_t e = train_pass(s, x_dev, y_dev, s->B, 1, 0, 0, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return sfail(SUPA_ERR_CUDA, std::string("gradients: ") + cudaGetErrorString(e));
    int rc = check_error_word(s);
    if (rc != SUPA_OK) return rc;
    std::vector<float> g(Off::total);
    if (cudaMemcpy(g.data(), s->grad, Off::total * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "gradient copy failed");
    pack_params(g, grads_host);
    if (loss_host && cudaMemcpy(loss_host, s->loss_tmp, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "loss copy failed");
    return SUPA_OK;
}

}  // extern "C"

namespace {
// The training pass of the minibatch (see train_pass; loss added to *loss),
// then the Adam update.
int train_minibatch(supa_surrogate *s, const float *x, const float *y, int64_t n, uint64_t a, uint64_t c, int64_t i0,
                    float lr, double *loss, cudaStream_t st, const float4 *yt = nullptr) {
    // train_pass() adds the minibatch loss to s->loss_tmp; point it at the accumulator
    double *keep = s->loss_tmp;
    s->loss_tmp = loss;
    cudaError_t e = train_pass(s, x, y, n, a, c, i0, st, yt);
    s->loss_tmp = keep;
    if (e != cudaSuccess) return sfail(SUPA_ERR_CUDA, std::string("train_step: ") + cudaGetErrorString(e));
    s->t += 1;
    const float c1 = 1.0f - std::pow(s->beta1, (float)s->t), c2 = 1.0f - std::pow(s->beta2, (float)s->t);
    const WeightCopies wc{{(int)Off::W1, (int)Off::W2, (int)Off::W3, (int)Off::W4},
                          {kHid * kInPad, kHid * kHid, kHid * kHid, kOutPad * kHid},
                          {s->W1b, s->W2b, s->W3b, s->W4b}};
    static_assert(Off::total % 4 == 0 && Off::W1 % 4 == 0 && Off::W2 % 4 == 0 && Off::W3 % 4 == 0 &&
                      Off::W4 % 4 == 0 && (kHid * kInPad) % 4 == 0 && (kOutPad * kHid) % 4 == 0,
                  "the Adam update takes four parameters a thread");
    if (launch_pdl(adam_update, dim3((unsigned)((Off::total / 4 + 255) / 256)), dim3(256), 0, st, s->master, s->m, s->v,
                   s->grad, (int)Off::total, lr, s->beta1, s->beta2, s->eps, 1.0f / c1, 1.0f / std::sqrt(c2), wc,
                   s->avg_on ? s->avg : (float *)nullptr, s->avg_on ? 1.0f / (float)(s->avg_n + 1) : 0.0f) !=
        cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "train_step launch failed");
    s->grad_zero = true;
    if (s->avg_on) ++s->avg_n;
    return SUPA_OK;
}
}  // namespace

extern "C" {

int supa_surrogate_train_step(supa_surrogate *s, const float *x_dev, const float *y_dev, float lr,
                              double *loss_acc_dev, void *stream) {
    if (!s || !x_dev || !y_dev) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_train_step: null argument");
    if (((uintptr_t)x_dev & 3) || ((uintptr_t)y_dev & 7))
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_train_step: x must be 4-byte and y 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    return train_minibatch(s, x_dev, y_dev, s->B, 1, 0, 0, lr, loss_acc_dev ? loss_acc_dev : s->loss_tmp, st);
}

int supa_surrogate_average(supa_surrogate *s, int32_t mode, void *stream) {
    if (!s) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_average: null surrogate");
    cudaStream_t st = (cudaStream_t)stream;
    if (mode == SUPA_AVERAGE_START) {
        // zeroed, so that the first step added (weight 1) gives exactly its parameters
        if (cudaMemsetAsync(s->avg, 0, Off::total * sizeof(float), st) != cudaSuccess)
            return sfail(SUPA_ERR_CUDA, "supa_surrogate_average: memset failed");
        s->avg_on = true;
        s->avg_n = 0;
    } else if (mode == SUPA_AVERAGE_STOP) {
        s->avg_on = false;
    } else if (mode == SUPA_AVERAGE_APPLY) {
        if (s->avg_n > 0 &&
            (cudaMemcpyAsync(s->master, s->avg, Off::total * sizeof(float), cudaMemcpyDeviceToDevice, st) !=
                 cudaSuccess ||
             weight_copies(s, st) != SUPA_OK))
            return sfail(SUPA_ERR_CUDA, "supa_surrogate_average: apply failed");
    } else {
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_average: mode must be 0, 1 or 2");
    }
    return SUPA_OK;
}

int supa_surrogate_train_epoch(supa_surrogate *s, const float *x_dev, const float *y_dev, int64_t n, uint64_t seed,
                               float lr, double *loss_acc_dev, void *stream) {
    if (!s || !x_dev || !y_dev || n < s->B)
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_train_epoch: need at least one full minibatch");
    if (((uintptr_t)x_dev & 3) || ((uintptr_t)y_dev & 7))
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_train_epoch: x must be 4-byte and y 8-byte aligned");
    cudaStream_t st = (cudaStream_t)stream;
    // permutation i -> (a i + c) mod n with gcd(a, n) = 1
    uint64_t a = (seed * 0x9E3779B97F4A7C15ull + 0x632BE59BD9B4E019ull) % (uint64_t)n;
    if (a == 0) a = 1;
    auto gcd = [](uint64_t u, uint64_t v) {
        while (v) {
            const uint64_t t = u % v;
            u = v;
            v = t;
        }
        return u;
    };
    while (gcd(a, (uint64_t)n) != 1) a = (a + 1) % (uint64_t)n == 0 ? 1 : a + 1;
    const uint64_t c = (seed ^ 0xD1B54A32D192ED03ull) % (uint64_t)n;
    const int64_t steps = n / s->B;
    double *loss = loss_acc_dev ? loss_acc_dev : s->loss_tmp;
    // the epoch's targets in the training pass's order, staged once (the
    // gather of random rows is then off the passes' critical path)
    const int64_t tiles = steps * (s->B / 128);
    if (tiles > s->yt_epoch_tiles) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return sfail(SUPA_ERR_CUDA, "train_epoch: stream failed");
        cudaFree(s->yt_epoch);
        s->yt_epoch = nullptr;
        s->yt_epoch_tiles = 0;
        if (cudaMalloc((void **)&s->yt_epoch, (size_t)tiles * 2048 * sizeof(float4)) != cudaSuccess)
            return sfail(SUPA_ERR_OOM, "supa_surrogate_train_epoch: out of device memory for the staged targets");
        s->yt_epoch_tiles = tiles;
    }
    if (launch_stage_targets(y_dev, n, 0, a, c, tiles, s->yt_epoch, st) != cudaSuccess)
        return sfail(SUPA_ERR_CUDA, "train_epoch: staging launch failed");
    for (int64_t k = 0; k < steps; ++k) {
        const int rc = train_minibatch(s, x_dev, y_dev, n, a, c, k * s->B, lr, loss, st,
                                       s->yt_epoch + (size_t)k * (s->B / 128) * 2048);
        if (rc != SUPA_OK) return rc;
    }
    return cudaGetLastError() == cudaSuccess ? SUPA_OK : sfail(SUPA_ERR_CUDA, "train_epoch launch failed");
}

int supa_surrogate_forward(supa_surrogate *s, const float *x_dev, int64_t n, float *out_dev, int64_t ld_out,
                           void *stream) {
    if (!s || (!x_dev && n > 0) || (!out_dev && n > 0))
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_forward: null argument");
    if (n < 0 || n > INT32_MAX) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_forward: n out of range");
    if ((uintptr_t)x_dev & 7) return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_forward: x must be 8-byte aligned");
    if (ld_out < kOut || ld_out > INT32_MAX)
        return sfail(SUPA_ERR_INVALID_ARG, "supa_surrogate_forward: ld_out must be in [90, 2^31)");
    MlpInferArgs a{};
    a.x = x_dev;
    a.rows = (int)n;
    a.b1 = s->master + Off::b1;
    a.b2 = s->master + Off::b2;
    a.b3 = s->master + Off::b3;
    a.b4 = s->master + Off::b4;
    a.out = out_dev;
    a.ld = (int)ld_out;
    // a pitch of whole 16-byte groups takes the TMA stores, which write whole
    // groups: then the padding outputs 90.. (zero) are written too, up to 96
    a.ncols = ld_out % 4 == 0 ? (int)std::min<int64_t>(ld_out, kInferLd) : kOut;
    a.error = s->error;
    const cudaError_t e = launch_sur_mlp(s->tm.w1, s->tm.w2, s->tm.w3, s->mW4i, a, (cudaStream_t)stream);
    if (e != cudaSuccess) return sfail(SUPA_ERR_CUDA, std::string("forward: ") + cudaGetErrorString(e));
    return SUPA_OK;
}

int supa_surrogate_check(supa_surrogate *s) {
    if (!s) return sfail(SUPA_ERR_INVALID_ARG, "null surrogate");
    if (cudaDeviceSynchronize() != cudaSuccess) return sfail(SUPA_ERR_CUDA, "device error");
    return check_error_word(s);
}

int supa_check_wait_expiry(int64_t limit_cycles, void *stream) {
    if (limit_cycles < 1 || limit_cycles > (1ll << 40))
        return sfail(SUPA_ERR_INVALID_ARG, "limit_cycles must be in [1, 2^40]");
    cudaStream_t st = (cudaStream_t)stream;
    int *d_status = nullptr;
    int status = -1;
    cudaError_t e = cudaMalloc(&d_status, sizeof(int));
    if (e == cudaSuccess) e = launch_wait_expiry_probe((long long)limit_cycles, d_status, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_status);
    if (e != cudaSuccess) return sfail(SUPA_ERR_CUDA, cudaGetErrorString(e));
    if (status == 1) return sfail(SUPA_ERR_TIMEOUT, "the bounded wait gave up, as it must");
    return SUPA_OK;
}

}  // extern "C"
