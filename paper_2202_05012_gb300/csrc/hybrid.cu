// hybrid.cu -- the surrogate side of the hybrid path (no counterpart in the
// SUPA paper) and the training set of the surrogate.
//
// After the step kernel has queued every particle that fell below E_s on a
// readout slice, and the network has predicted per-layer deposit
// distributions for the queue (means mu_j and log-variances s_j of the
// deposit fraction of layer start + j), these kernels
//   1. draw d_j = E max(0, mu_j + exp(s_j / 2) n_j) with standard normals n_j
//      from Philox (stream tag 1, keyed by shower, slice and lineage, so the
//      draw is replayable), truncated at the detector's back and scaled down
//      when they add up to more than E; the rest of E is booked as
//      surrogate leakage;
//   2. add the deposits to the shower's FP64 layer sums and count one hit per
//      non-empty layer;
//   3. after a scan of the counts, write the hits -- one per layer, at the
//      straight-line continuation of the particle to the layer's mid depth --
//      into a per-shower segment that follows the stepped hits.
#include <algorithm>

#include "philox.cuh"
#include "supa_internal.cuh"

namespace supa {

namespace {

// 32 standard normals (Box-Muller) for one diverted particle.
__device__ void normals32(uint32_t sid, int k, uint32_t lin_lo, uint32_t lin_hi, uint64_t seed, float *z) {
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
    for (int blk = 0; blk < 8; ++blk) {
        const uint4 r = philox4x32_10(make_uint4(sid, (uint32_t)k | (1u << 16) | ((uint32_t)blk << 20), lin_lo, lin_hi),
                                      k0, k1);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const float u1 = (float)((w[2 * p] >> 8) + 1u) * (1.0f / 16777216.0f);  // (0, 1]
            const float u2 = u24(w[2 * p + 1]);
            const float rad = sqrtf(-2.0f * logf(u1));
            float sn, cs;
            sincospif(2.0f * u2, &sn, &cs);
            z[4 * blk + 2 * p] = rad * cs;
            z[4 * blk + 2 * p + 1] = rad * sn;
        }
    }
}

}  // namespace

// Pass 1: deposits per diverted particle, layer sums, hit counts, leakage.
__global__ void sur_deposits(const SurParams p) {
    const unsigned n = min(*p.count, (unsigned)p.cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SurRec r = p.rec[i];
        const supa_primary pr = p.prim[r.shower];
        const GeomDev g = p.geoms[pr.geom & 0xFFFFu];
        float z[32];
        if (p.mode == SUPA_SURROGATE_SAMPLE)
            normals32((uint32_t)(p.shower_id_base + r.shower), r.k, r.lin_lo, r.lin_hi, p.seed, z);
        const float *o = p.out + (size_t)i * 64;
        float d[kSurLayers];
        float sum = 0.0f;
#pragma unroll
        for (int j = 0; j < kSurLayers; ++j) {
            float v = 0.0f;
            if (r.layer + j < g.n_layers) {
                const float f = p.mode == SUPA_SURROGATE_SAMPLE ? fmaf(expf(0.5f * o[kSurLayers + j]), z[j], o[j])
                                                               : o[j];
                v = r.E * fmaxf(0.0f, f);
            }
            d[j] = v;
            sum += v;
        }
        const float scale = sum > r.E ? r.E / sum : 1.0f;
        double kept = 0.0;
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < kSurLayers; ++j) {
            const float v = d[j] * scale;
            p.dep[(size_t)i * kSurLayers + j] = v;
            if (v > 0.0f) {
                ++cnt;
                kept += (double)v;
                atomicAdd(&p.lsum[(size_t)r.shower * p.lsum_stride + r.layer + j], (double)v);
            }
        }
        atomicAdd(&p.sur_leak[r.shower], (double)r.E - kept);
        if (cnt) atomicAdd(&p.scount[r.shower], (unsigned)cnt);
    }
}

// Pass 2: the hits, into each shower's segment [soff[s], soff[s] + scount[s]).
__global__ void sur_hits(const SurParams p) {
    const unsigned n = min(*p.count, (unsigned)p.cap);
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const SurRec r = p.rec[i];
        const supa_primary pr = p.prim[r.shower];
        const GeomDev g = p.geoms[pr.geom & 0xFFFFu];
        const float *d = p.dep + (size_t)i * kSurLayers;
        int cnt = 0;
        for (int j = 0; j < kSurLayers; ++j) cnt += d[j] > 0.0f;
        if (!cnt) continue;
        int64_t at = p.soff[r.shower] + (int64_t)atomicAdd(&p.scursor[r.shower], (unsigned)cnt);
        const float zk = (float)r.k * g.dz;
        for (int j = 0; j < kSurLayers; ++j) {
            if (!(d[j] > 0.0f)) continue;
            const float zm = p.zmid[g.layer_off + r.layer + j];
            const float dz = zm - zk;
            p.hits[at++] = make_float4(fmaf(dz, r.tx, r.x), fmaf(dz, r.ty, r.y), zm, d[j]);
        }
    }
}

__global__ void add_counts(const uint32_t *a, const uint32_t *b, int64_t n, uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// Training set of the surrogate from a batch of sub-showers: features of
// each sub-shower's start and its deposit fractions per layer from the start
// layer on.
__global__ void training_set(const supa_primary *prim, int64_t n, const GeomDev *geoms, const int8_t *s2l,
                             const LayerInfo *linfo, const double *lsum, int stride, float e_s, float *x, float *y,
                             int *bad) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const supa_primary pr = prim[s];
        const GeomDev g = geoms[pr.geom & 0xFFFFu];
        const int k0 = (int)(pr.geom >> 16);
        const int l0 = (k0 < g.n_slices) ? (int)s2l[g.slice_off + k0] : -1;
        if (l0 < 0) {
            atomicOr(bad, 1);
            continue;
        }
        float st, ct, sp, cp;
        sincosf(pr.theta, &st, &ct);
        sincosf(pr.phi, &sp, &cp);
        float f[kSurIn];
        surrogate_features(pr.E, st * cp, st * sp, ct, k0, l0, g.n_layers, linfo[g.layer_off + l0], e_s, f);
        for (int i = 0; i < kSurIn; ++i) x[s * kSurIn + i] = f[i];
        for (int j = 0; j < kSurLayers; ++j)
            y[s * kSurLayers + j] =
                (l0 + j < g.n_layers) ? (float)(lsum[(size_t)s * stride + l0 + j] / (double)pr.E) : 0.0f;
    }
}

cudaError_t launch_sur_deposits(const SurParams &p, cudaStream_t st) {
    sur_deposits<<<2048, 128, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sur_hits(const SurParams &p, cudaStream_t st) {
    sur_hits<<<2048, 128, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_add_counts(const uint32_t *a, const uint32_t *b, int64_t n, uint32_t *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    add_counts<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(a, b, n, out);
    return cudaGetLastError();
}

cudaError_t launch_training_set(const supa_primary *prim, int64_t n, const GeomDev *geoms, const int8_t *s2l,
                                const LayerInfo *linfo, const double *lsum, int stride, float e_s, float *x, float *y,
                                int *bad, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    training_set<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(prim, n, geoms, s2l, linfo, lsum,
                                                                                    stride, e_s, x, y, bad);
    return cudaGetLastError();
}

}  // namespace supa
