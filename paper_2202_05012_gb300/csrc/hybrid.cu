// hybrid.cu -- the surrogate side of the hybrid path (no counterpart in the
// SUPA paper) and the training set of the surrogate.
//
// After the step kernel has queued every particle that fell below E_s on a
// readout slice, and the network has predicted per-layer deposit
// distributions for the queue (means mu_j and log-variances s_j of the
// deposit fraction of layer start + j, mean lateral distances rho_j), these
// kernels
//   1. take d_j = E mu_j, mu_j = exp(o_j - 4) (MEAN; 0 below a millionth),
//      or split the MEAN total T = sum_j f_j of those fractions over their
//      layers by a Dirichlet draw whose means
//      are the MEAN shares and whose concentration c matches the predicted
//      variances exp(s_j) (SAMPLE: d_j = E T G_j / sum G, G_j ~ Gamma(c m_j)
//      by Marsaglia and Tsang's method on Philox stream tag 3, keyed by
//      shower, slice and lineage, so the draw is replayable; every layer's
//      expected deposit is its MEAN deposit), truncated at the detector's
//      back and scaled down when they add up to more than E; the rest of E
//      is booked as surrogate leakage;
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

constexpr unsigned kFull = 0xFFFFFFFFu;

// Gamma(alpha, 1) variate of layer j of a diverted particle: Marsaglia and
// Tsang, "A simple method for generating gamma variables" (ACM TOMS 26(3),
// 2000), for shape a = alpha, or a = alpha + 1 times u3^(1/alpha) when
// alpha < 1.  Attempt t (0..3) takes the Philox block with counter
// (shower id, slice | 3 << 16 | (4 j + t) << 20, lineage lo, lineage hi):
// a standard normal x from words 0 and 1 (Box-Muller), the uniform of the
// accept test from word 2, u3 from word 3.  The accept test is evaluated
// with explicitly rounded float32 operations in a fixed order (no
// contraction into fused multiply-adds), so that another implementation
// can take the same decision; four rejections in a row give the mean alpha.
__device__ float gamma_variate(float alpha, uint32_t sid, int k, uint32_t lin_lo, uint32_t lin_hi, uint64_t seed,
                               int j) {
    const bool boost = alpha < 1.0f;
    const float a = boost ? __fadd_rn(alpha, 1.0f) : alpha;
    const float d = __fsub_rn(a, 0.333333343f);  // float32(1/3)
    const float c = __fdiv_rn(1.0f, __fsqrt_rn(__fmul_rn(9.0f, d)));
    for (int t = 0; t < 4; ++t) {
        const uint4 r = philox4x32_10(
            make_uint4(sid, (uint32_t)k | (3u << 16) | ((uint32_t)(4 * j + t) << 20), lin_lo, lin_hi),
            (uint32_t)seed, (uint32_t)(seed >> 32));
        const float u1 = (float)((r.x >> 8) + 1u) * (1.0f / 16777216.0f);  // (0, 1]
        const float u2 = u24(r.y);
        const float rad = __fsqrt_rn(__fmul_rn(-2.0f, logf(u1)));
        const float x = __fmul_rn(rad, cospif(__fmul_rn(2.0f, u2)));
        const float t1 = __fadd_rn(1.0f, __fmul_rn(c, x));
        if (!(t1 > 0.0f)) continue;
        const float v = __fmul_rn(__fmul_rn(t1, t1), t1);
        const float u = (float)((r.z >> 8) + 1u) * (1.0f / 16777216.0f);
        const float rhs = __fadd_rn(__fmul_rn(0.5f, __fmul_rn(x, x)),
                                    __fmul_rn(d, __fadd_rn(__fsub_rn(1.0f, v), logf(v))));
        if (!(logf(u) < rhs)) continue;
        float g = __fmul_rn(d, v);
        if (boost) {
            const float u3 = (float)((r.w >> 8) + 1u) * (1.0f / 16777216.0f);
            g *= powf(u3, __fdiv_rn(1.0f, alpha));
        }
        return g;
    }
    return alpha;
}

// Dirichlet concentration bounds of the SAMPLE split: below kSampleCMin the
// concentration is raised to it; above kSampleCMax the spread is negligible
// and the MEAN shares are taken without a draw.
constexpr float kSampleCMin = 1.0f, kSampleCMax = 1.0e4f;

// The lateral law of the surrogate hits: the quantile function of q, a hit's
// distance from its sub-shower's axis over the mean distance rho_j, at u =
// i / 64 (i = 0..64; the last point is the quantile at u = 0.998), linear in
// between, mean 1.  Measured from plain sub-showers (energy-weighted hit
// distances about the mean distance of sub-showers alike in energy, start
// slice and layer offset, 0.05-2 GeV): an atom at 0, a core narrower and a
// tail longer than a 2-D Gaussian's.
__constant__ float c_lateral_q[65] = {
    0.00000f, 0.00000f, 0.00000f, 0.13168f, 0.19840f, 0.24732f, 0.28922f, 0.32671f,
    0.36028f, 0.39115f, 0.42114f, 0.44900f, 0.47602f, 0.50152f, 0.52699f, 0.55146f,
    0.57525f, 0.59910f, 0.62231f, 0.64475f, 0.66703f, 0.68907f, 0.71090f, 0.73253f,
    0.75422f, 0.77610f, 0.79778f, 0.81916f, 0.84060f, 0.86253f, 0.88486f, 0.90712f,
    0.92884f, 0.95082f, 0.97305f, 0.99593f, 1.01889f, 1.04247f, 1.06618f, 1.09030f,
    1.11503f, 1.14011f, 1.16589f, 1.19201f, 1.21890f, 1.24660f, 1.27561f, 1.30556f,
    1.33609f, 1.36810f, 1.40167f, 1.43705f, 1.47402f, 1.51349f, 1.55558f, 1.60084f,
    1.65098f, 1.70647f, 1.77006f, 1.84258f, 1.92934f, 2.03901f, 2.19413f, 2.48104f,
    4.43834f};

// The displacement (q cos phi, q sin phi) of all hits of a diverted particle,
// in units of each layer's rho_j: from words (w0, w1) of the Philox block with
// counter (shower id, slice | 2 << 16, lineage lo, lineage hi), same key,
// q = the law's quantile at u = (w0 >> 8) 2^-24, phi = 2 pi (w1 >> 8) 2^-24.
// A displacement needs no more than ~1e-6 relative accuracy, so the hardware
// sine and cosine serve.
__device__ float2 lateral_offset(uint32_t sid, int k, uint32_t lin_lo, uint32_t lin_hi, uint64_t seed) {
    const uint4 r = philox4x32_10(make_uint4(sid, (uint32_t)k | (2u << 16), lin_lo, lin_hi), (uint32_t)seed,
                                  (uint32_t)(seed >> 32));
    const float x = (float)(r.x >> 8) * (64.0f / 16777216.0f);  // exact: u * 64 in [0, 64)
    const int i = min(63, (int)x);
    const float q = fmaf(x - (float)i, c_lateral_q[i + 1] - c_lateral_q[i], c_lateral_q[i]);
    float sn, cs;
    __sincosf(6.28318530717958648f * u24(r.y), &sn, &cs);
    return make_float2(q * cs, q * sn);
}

// Contiguous range of queue entries of this warp: consecutive entries mostly
// belong to one shower (the step kernel queues a warp's diverted particles
// together), so runs stay whole.
__device__ __forceinline__ void warp_range(unsigned n, unsigned &i0, unsigned &i1) {
    const unsigned nw = (gridDim.x * blockDim.x) >> 5, w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned per = (n + nw - 1) / nw;
    i0 = min(n, w * per);
    i1 = min(n, i0 + per);
}

}  // namespace

constexpr int kDepWarps = 4;

// Pass 1: deposits d_j (j = 0..29, layer start + j), hit count per particle,
// and per shower the layer sums, surrogate leakage and hit count.  A warp
// walks a contiguous range of the queue 32 entries at a time.  First one
// lane per particle: it reads the particle's network outputs as float4 rows,
// forms its 30 deposits in registers, writes them and stages them in shared
// memory.  Then one particle at a time, lane L adds the staged deposits of
// absolute layers L and L + 32 to its run sums -- 64-bit fixed point (units
// of 2^-32; integer adds: the FP64 unit of this GPU is far too slow for a
// double add per deposit), summed over each run of consecutive queue
// entries of one shower (consecutive entries mostly belong to one shower)
// and converted to FP64 and added to the shower's sums once per run.
template <bool kSample>
__global__ void __launch_bounds__(kDepWarps * 32) sur_deposits(const SurParams p) {
    __shared__ float s_dep[kDepWarps][32][kSurLayers + 1];
    const unsigned n = min(*p.count, (unsigned)p.cap);
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    float(*stg)[kSurLayers + 1] = s_dep[wib];
    unsigned i0, i1;
    warp_range(n, i0, i1);
    int cur = -1;
    unsigned long long acc_lo = 0, acc_hi = 0;
    long long leak = 0;
    unsigned cnt = 0;
    auto flush = [&]() {  // warp-uniform
        if (cur < 0) return;
        double *ls = p.lsum + (size_t)cur * p.lsum_stride;
        if (acc_lo) atomicAdd(&ls[lane], from_fixed32(acc_lo));
        if (acc_hi) atomicAdd(&ls[lane + 32], from_fixed32(acc_hi));
        // the run's leakage is spread over the lanes
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) leak += __shfl_xor_sync(kFull, leak, o);
        if (lane == 0) {
            atomicAdd(&p.sur_leak[cur], (double)leak * (1.0 / 4294967296.0));
            if (cnt) atomicAdd(&p.scount[cur], cnt);
        }
        acc_lo = acc_hi = 0;
        leak = 0;
        cnt = 0;
    };
    for (unsigned g0 = i0; g0 < i1; g0 += 32) {
        const unsigned i = g0 + (unsigned)lane;
        const int m = (int)min(32u, i1 - g0);
        uint32_t sh = 0;
        int layer = 0;
        unsigned pc = 0;
        long long pleak = 0;
        if (lane < m) {
            const SurRec r = p.rec[i];
            sh = r.shower;
            layer = r.layer;
            const float E = r.E;
            const int nj = min(kSurLayers, p.geoms[p.prim[r.shower].geom & 0xFFFFu].n_layers - layer);
            float v[kSurLayers];
            const float4 *o4 = reinterpret_cast<const float4 *>(p.out + (size_t)i * p.out_ld);
#pragma unroll
            for (int q = 0; q < (kSurLayers + 3) / 4; ++q) {
                const float4 mv = __ldg(o4 + q);
                const float mq[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    if (4 * q + t < kSurLayers) v[4 * q + t] = mq[t];
            }
            // MEAN fractions of the layers inside the detector (log link;
            // none below a millionth)
            float T = 0.0f;
#pragma unroll
            for (int j = 0; j < kSurLayers; ++j) {
                const float mu = expf(v[j] - kMuShift);
                v[j] = j < nj && mu >= kFractionMin ? mu : 0.0f;
                T += v[j];
            }
            if (kSample && T > 0.0f) {
                // concentration matched to the predicted variances of the layers with a mean
                const float rT = 1.0f / T;
                float q = 0.0f, V = 0.0f;
#pragma unroll
                for (int j = 0; j < kSurLayers; ++j) {
                    if (v[j] > 0.0f) {
                        const float m = v[j] * rT;
                        q = fmaf(m, m, q);
                        V += expf(__ldg(p.out + (size_t)i * p.out_ld + kSurLayers + j)) + kVarFloor;
                    }
                }
                const float num = T * T * (1.0f - q);
                if (V > 0.0f && num <= (kSampleCMax + 1.0f) * V) {
                    const float cm = fmaxf(kSampleCMin, num / V - 1.0f) * rT;
                    // one layer at a time, the variates staged in this lane's
                    // row of shared memory (one copy of the sampler's code:
                    // unrolled over 30 layers it overflows the instruction cache)
                    float gs = 0.0f;
#pragma unroll 1
                    for (int j = 0; j < nj; ++j) {
                        const float mu = expf(__ldg(p.out + (size_t)i * p.out_ld + j) - kMuShift);
                        const float G = mu >= kFractionMin
                                            ? gamma_variate(cm * mu, (uint32_t)(p.shower_id_base + sh), r.k, r.lin_lo,
                                                            r.lin_hi, p.seed, j)
                                            : 0.0f;
                        stg[lane][j] = G;
                        gs += G;
                    }
                    if (gs > 0.0f) {
                        // drawn shares below a millionth of E get nothing; the rest normalises
                        const float tg = T / gs;
                        float gk = 0.0f;
#pragma unroll
                        for (int j = 0; j < kSurLayers; ++j) {
                            float G = j < nj ? stg[lane][j] : 0.0f;
                            if (tg * G < kFractionMin) G = 0.0f;
                            stg[lane][j] = G;
                            gk += G;
                        }
                        if (gk > 0.0f) {
                            const float sc = T / gk;
#pragma unroll
                            for (int j = 0; j < kSurLayers; ++j) v[j] = stg[lane][j] * sc;
                        }
                    }
                }
            }
            float sum = 0.0f;
#pragma unroll
            for (int j = 0; j < kSurLayers; ++j) {
                v[j] *= E;
                sum += v[j];
            }
            float scale = 1.0f;
            if (sum > E) scale = E / sum;
            float2 *d2 = reinterpret_cast<float2 *>(p.dep + (size_t)i * kSurLayers);
            pleak = (long long)fixed32(E);
#pragma unroll
            for (int j = 0; j < kSurLayers; ++j) {
                if (scale != 1.0f) v[j] *= scale;
                pc += v[j] > 0.0f;
                stg[lane][j] = v[j];
            }
#pragma unroll
            for (int j = 0; j < kSurLayers; j += 2) d2[j / 2] = make_float2(v[j], v[j + 1]);
            p.pcnt[i] = (uint8_t)pc;
        }
        __syncwarp();
        // one particle at a time: lane L takes absolute layers L and L + 32
        for (int k = 0; k < m; ++k) {
            const int sk = (int)__shfl_sync(kFull, sh, k);
            const int lk = __shfl_sync(kFull, layer, k);
            const unsigned ck = __shfl_sync(kFull, pc, k);
            if (sk != cur) {
                flush();
                cur = sk;
            }
            const int j_lo = lane - lk, j_hi = lane + 32 - lk;
            unsigned long long f_lo = 0, f_hi = 0;
            if (j_lo >= 0 && j_lo < kSurLayers) f_lo = fixed32(stg[k][j_lo]);
            if (j_hi >= 0 && j_hi < kSurLayers) f_hi = fixed32(stg[k][j_hi]);
            acc_lo += f_lo;
            acc_hi += f_hi;
            leak -= (long long)(f_lo + f_hi);
            cnt += ck;
            if (lane == k) leak += pleak;  // the particle's energy, once (in its own lane)
        }
        __syncwarp();
    }
    flush();
}

// Pass 2: the hits, into each shower's segment [soff[s], soff[s] + scount[s]).
// Per group of 32 queue entries, one cursor atomic per run of one shower
// (segmented scan of the per-particle counts), then one particle at a time
// with lane j writing the hit of layer start + j when its deposit is > 0 --
// a particle's hits are consecutive, in layer order.  The hit sits at the
// layer's mid depth, displaced from the particle's straight line by
// max(0, rho_j) (m1, m2), one lateral-law draw (m1, m2) per particle (drawn
// lane-per-particle for the group): the mean displacement of a layer's hit
// is the predicted mean distance rho_j.
__global__ void sur_hits(const SurParams p) {
    const unsigned n = min(*p.count, (unsigned)p.cap);
    const int lane = threadIdx.x & 31;
    const unsigned lt = (1u << lane) - 1u;
    unsigned i0, i1;
    warp_range(n, i0, i1);
    for (unsigned g0 = i0; g0 < i1; g0 += 32) {
        const unsigned i = g0 + lane;
        const int m = (int)min(32u, i1 - g0);
        const bool valid = lane < m;
        int sh = -1 - lane, r_loff = 0;
        unsigned c = 0;
        float r_x = 0.f, r_y = 0.f, r_tx = 0.f, r_ty = 0.f, r_zk = 0.f;
        float2 r_m = make_float2(0.f, 0.f);
        unsigned long long r_tag = 0;
        if (valid) {
            const SurRec r = p.rec[i];
            sh = (int)r.shower;
            r_tag = (1ull << 63) | ((unsigned long long)r.lin_hi << 32) | r.lin_lo;
            c = p.pcnt[i];
            if (c) r_m = lateral_offset((uint32_t)(p.shower_id_base + r.shower), r.k, r.lin_lo, r.lin_hi, p.seed);
            const GeomDev &g = p.geoms[p.prim[r.shower].geom & 0xFFFFu];
            r_loff = g.layer_off + r.layer;
            r_zk = (float)r.k * g.dz;
            r_x = r.x;
            r_y = r.y;
            r_tx = r.tx;
            r_ty = r.ty;
        }
        // runs of equal shower among the lanes
        const int prev = __shfl_up_sync(kFull, sh, 1);
        const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != sh);
        const int start = 31 - __clz(heads & (lt | (1u << lane)));
        const unsigned later = heads & ~(lt | (1u << lane));
        const int end = later ? __ffs(later) - 2 : 31;
        // inclusive prefix of c over the warp
        unsigned inc = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned t = __shfl_up_sync(kFull, inc, o);
            if (lane >= o) inc += t;
        }
        const unsigned exc = inc - c;
        const unsigned run_exc = exc - __shfl_sync(kFull, exc, start);
        const unsigned run_tot = __shfl_sync(kFull, inc, end) - __shfl_sync(kFull, exc, start);
        unsigned base = 0;
        if (lane == end && valid && run_tot) base = atomicAdd(&p.scursor[sh], run_tot);
        base = __shfl_sync(kFull, base, end);
        const int64_t at_lane = valid ? p.soff[sh] + (int64_t)(base + run_exc) : 0;
        for (int k0 = 0; k0 < m; k0 += 8) {
            float d[8], rho[8], zmid[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const bool ld = k0 + u < m && lane < kSurLayers;
                d[u] = ld ? p.dep[(size_t)(g0 + k0 + u) * kSurLayers + lane] : 0.0f;
                rho[u] = ld ? p.out[(size_t)(g0 + k0 + u) * p.out_ld + 2 * kSurLayers + lane] : 0.0f;
            }
            // mid depths of the layers that get a hit (a deposit > 0 lies inside the detector)
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int loff = __shfl_sync(kFull, r_loff, (k0 + u) & 31);
                zmid[u] = d[u] > 0.0f ? p.zmid[loff + lane] : 0.0f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = k0 + u;
                if (k >= m) break;
                const int64_t at = __shfl_sync(kFull, at_lane, k);
                const float zk = __shfl_sync(kFull, r_zk, k), x = __shfl_sync(kFull, r_x, k),
                            y = __shfl_sync(kFull, r_y, k), tx = __shfl_sync(kFull, r_tx, k),
                            ty = __shfl_sync(kFull, r_ty, k), m1 = __shfl_sync(kFull, r_m.x, k),
                            m2 = __shfl_sync(kFull, r_m.y, k);
                const unsigned nz = __ballot_sync(kFull, d[u] > 0.0f);
                const unsigned long long tag = p.tags ? __shfl_sync(kFull, r_tag, k) : 0ull;
                if (d[u] > 0.0f) {
                    const float zm = zmid[u];
                    const float dz = zm - zk;
                    const float sig = fmaxf(0.0f, rho[u]);
                    p.hits[at + __popc(nz & lt)] =
                        make_float4(fmaf(sig, m1, fmaf(dz, tx, x)), fmaf(sig, m2, fmaf(dz, ty, y)), zm, d[u]);
                    if (p.tags) p.tags[at + __popc(nz & lt)] = tag;
                }
            }
        }
    }
}

__global__ void add_counts(const uint32_t *a, const uint32_t *b, int64_t n, uint32_t *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = a[i] + b[i];
}

// Training set of the surrogate from a batch of sub-showers: features of
// each sub-shower's start and its deposit fractions per layer from the start
// layer on (columns 0..29 of y [n][60]; the mean distances, columns 30..59,
// come from launch_lateral_targets).
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
            y[s * 2 * kSurLayers + j] =
                (l0 + j < g.n_layers) ? (float)(lsum[(size_t)s * stride + l0 + j] / (double)pr.E) : 0.0f;
    }
}

// The diverted particles of the last hybrid run as sub-shower primaries: each
// enters on its slice of diversion with its energy, position and direction
// (polar angle and azimuth from the slopes), in the geometry of its shower.
__global__ void export_diverted(const SurRec *rec, int64_t n, const supa_primary *prim, supa_primary *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const SurRec r = rec[i];
        supa_primary q;
        q.E = r.E;
        q.x0 = r.x;
        q.y0 = r.y;
        q.theta = atanf(sqrtf(r.tx * r.tx + r.ty * r.ty));
        q.phi = atan2f(r.ty, r.tx);
        q.geom = (prim[r.shower].geom & 0xFFFFu) | ((uint32_t)r.k << 16);
        out[i] = q;
    }
}

// Per diverted particle: its queue record, network outputs, deposits and
// hit count as one supa_diverted_record.
__global__ void export_surrogate(const SurParams p, int64_t n, supa_diverted_record *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const SurRec r = p.rec[i];
        supa_diverted_record &o = out[i];
        o.shower = r.shower;
        o.slice = r.k;
        o.layer = r.layer;
        o.x = r.x;
        o.y = r.y;
        o.tx = r.tx;
        o.ty = r.ty;
        o.E = r.E;
        o.lineage = ((uint64_t)r.lin_hi << 32) | r.lin_lo;
        const float *row = p.out + (size_t)i * p.out_ld;
        for (int j = 0; j < kSurLayers; ++j) {
            o.lmu[j] = row[j];
            o.s[j] = row[kSurLayers + j];
            o.rho[j] = row[2 * kSurLayers + j];
            o.dep[j] = p.dep[(size_t)i * kSurLayers + j];
        }
        o.n_hits = p.pcnt[i];
        o.reserved = 0;
    }
}

cudaError_t launch_export_surrogate(const SurParams &p, int64_t n, supa_diverted_record *out, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    export_surrogate<<<(unsigned)std::min<int64_t>((n + 127) / 128, 8192), 128, 0, st>>>(p, n, out);
    return cudaGetLastError();
}

cudaError_t launch_export_diverted(const SurRec *rec, int64_t n, const supa_primary *prim, supa_primary *out,
                                   cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    export_diverted<<<(unsigned)std::min<int64_t>((n + 255) / 256, 8192), 256, 0, st>>>(rec, n, prim, out);
    return cudaGetLastError();
}

cudaError_t launch_sur_deposits(const SurParams &p, cudaStream_t st) {
    if (p.mode == SUPA_SURROGATE_SAMPLE)
        sur_deposits<true><<<4096, kDepWarps * 32, 0, st>>>(p);
    else
        sur_deposits<false><<<4096, kDepWarps * 32, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_sur_hits(const SurParams &p, cudaStream_t st) {
    sur_hits<<<4096, 128, 0, st>>>(p);
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
