// aux_kernels.cu -- hit fetch, shower profiles and shape variables, offset
// scan and the energy-ordered work queue of the SUPA library.
#include <algorithm>

#include "hits.cuh"
#include "supa_internal.cuh"

namespace supa {

namespace {
constexpr unsigned kFull = 0xFFFFFFFFu;
}  // namespace

// ---------------------------------------------------------------- fetch ---
// Copy canonical hits [first, first+count) (shower order) to dst.  Every warp
// finds the first shower overlapping the range by binary search over the
// offsets, then warps stride over the overlapping showers.
__global__ void supa_fetch_kernel(const FetchParams p, const int64_t *canon) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t lo_hit = p.first, hi_hit = p.first + p.count;
    // first shower s with canon[s+1] > lo_hit
    int64_t a = 0, b = p.n_showers;  // answer in [a, b)
    while (a < b) {
        const int64_t m = (a + b) >> 1;
        if (canon[m + 1] > lo_hit) b = m; else a = m + 1;
    }
    for (int64_t s = a + warp; s < p.n_showers; s += n_warps) {
        const int64_t s0 = canon[s];
        if (s0 >= hi_hit) break;
        ShowerHits it;
        it.init(p.src, s);
        int64_t i0 = 0;  // index within the shower of the segment start
        if (it.remaining <= 0) continue;
        do {
            for (int j = lane; j < it.seg_len; j += 32) {
                const int64_t gidx = s0 + i0 + j;
                if (gidx < lo_hit || gidx >= hi_hit) continue;
                if (p.dst_tags)
                    p.dst_tags[gidx - lo_hit] =
                        it.phase == 0 ? p.tag_pool[(size_t)(it.seg_ptr - p.src.pool) + j]
                                      : (p.sur_tags ? p.sur_tags[(size_t)(it.seg_ptr - p.src.sur_hits) + j] : 0ull);
                else
                    p.dst[gidx - lo_hit] = it.seg_ptr[j];
            }
            i0 += it.seg_len;
        } while (it.next());
    }
}

cudaError_t launch_fetch(const FetchParams &p, cudaStream_t st) {
    if (p.count <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    supa_fetch_kernel<<<sms * 8, 256, 0, st>>>(p, p.src.offsets);
    return cudaGetLastError();
}

// ------------------------------------------------------------ profiles ---
// Shower-shape profiles summed over a range of showers (Sec. 5.1 "layer
// energy"; lateral spread around the shower axis):
//   longi[l] += layer_sum[s][l] / E0_s
//   lat[b]   += E_hit / E0_s for hits whose transverse distance r from the
//               incidence axis through the impact point (at the hit's depth)
//               falls in bin b = floor(r / r_max * nbins) (last bin: overflow).
// One CTA per shower; FP32 shared-memory bins, FP64 global sums.
__global__ void __launch_bounds__(256) supa_profile_kernel(const ProfileParams p) {
    extern __shared__ float pbins[];
    const int64_t srel = blockIdx.x;
    const int64_t s = p.s_begin + srel;
    for (int i = threadIdx.x; i < p.nbins; i += blockDim.x) pbins[i] = 0.0f;
    __syncthreads();
    const supa_primary pr = p.prim[s];
    const double inv = 1.0 / (double)pr.E;
    for (int l = threadIdx.x; l < p.L; l += blockDim.x)
        atomicAdd(&p.longi[l], p.lsum[(size_t)s * p.L + l] * inv);
    const float t = tanf(pr.theta);
    const float tx = t * cosf(pr.phi), ty = t * sinf(pr.phi);
    const float scale = (float)p.nbins / p.r_max;
    ShowerHits it;
    it.init(p.src, s);
    if (it.remaining > 0) {
        do {
            for (int j = threadIdx.x; j < it.seg_len; j += blockDim.x) {
                const float4 h = __ldg(it.seg_ptr + j);
                const float r = hypotf(h.x - fmaf(h.z, tx, pr.x0), h.y - fmaf(h.z, ty, pr.y0));
                const int b = min((int)(r * scale), p.nbins - 1);
                atomicAdd(&pbins[b], h.w);
            }
        } while (it.next());
    }
    __syncthreads();
    for (int i = threadIdx.x; i < p.nbins; i += blockDim.x)
        if (pbins[i] != 0.0f) atomicAdd(&p.lat[i], (double)pbins[i] * inv);
}

// ------------------------------------------------------- shower shapes ---
// Shower shape variables of Sec. 5.1 and App. A.1 for one shower per CTA.
// Lateral coordinates of a point: (eta, phi) = (x, y) minus the incidence
// axis through the impact point at the point's depth, r = |(eta, phi)|.
// Pass 1 over the shower's hits: per layer the point count, sums of eta,
// phi, r, E, E eta, E phi, E r, and the largest point energy; pass 2: the
// second moments about the pass-1 means (no cancellation), and the second
// largest point energy.  A shower of up to kShapeCap hits is first sorted by
// layer in shared memory (counting sort), then each layer's run is reduced
// by one warp; larger showers are summed per 32 hits and layer across the
// warp and added with shared-memory atomics.  FP32 sums; layer energies, the
// total and the depth variables come from the FP64 layer sums.  Per layer:
//   n, Ebar, f, <eta>, <phi>, <r>, <E>, sd(eta), sd(phi), sd(r), sd(E),
//   <eta>_E, <phi>_E, <r>_E, sdE(eta), sdE(phi), sdE(r), E_ratio
// per shower: E_tot, depth d (-1: none), l_d, s_d, sigma_sd.
namespace {
enum { kSn, kSeta, kSphi, kSr, kSE, kSEeta, kSEphi, kSEr, kQeta, kQphi, kQr, kQE, kWeta, kWphi, kWr, kNSums };
}

// Sum of v over the lanes of the warp (every lane gets it).
__device__ __forceinline__ float warp_allsum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

constexpr int kShapeThreads = 256;
constexpr int kShapeCap = 1536;  // hits of one shower sorted by layer in shared memory (24 KB)

__global__ void __launch_bounds__(kShapeThreads) supa_shape_kernel(const ShapeParams p) {
    __shared__ float acc[SUPA_MAX_LAYERS][kNSums];
    __shared__ float mean[SUPA_MAX_LAYERS][7];  // <eta>, <phi>, <r>, <E>, <eta>_E, <phi>_E, <r>_E
    __shared__ unsigned top1[SUPA_MAX_LAYERS], top2[SUPA_MAX_LAYERS], ntop[SUPA_MAX_LAYERS];
    __shared__ float4 sorted[kShapeCap];
    __shared__ unsigned lstart[SUPA_MAX_LAYERS + 1], lcur[SUPA_MAX_LAYERS];
    __shared__ double sh_tot[3];  // E_tot, l_d, sum of i^2 Ebar_i
    __shared__ int sh_depth;
    const int64_t srel = blockIdx.x;
    const int64_t s = p.s_begin + srel;
    const int L = p.L;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const double *ls = p.lsum + (size_t)s * L;
    for (int i = threadIdx.x; i < L * kNSums; i += blockDim.x) acc[i / kNSums][i % kNSums] = 0.0f;
    for (int i = threadIdx.x; i < L; i += blockDim.x) top1[i] = top2[i] = ntop[i] = lcur[i] = 0u;
    if (wid == 0) {
        // the depth variables from the FP64 layer sums
        double e = 0.0, a = 0.0, a2 = 0.0;
        unsigned d = 0u;  // deepest layer with energy, + 1
        for (int l = lane; l < L; l += 32) {
            const double v = ls[l];
            e += v;
            a += (double)l * v;
            a2 += (double)l * (double)l * v;
            if (v > 0.0) d = (unsigned)l + 1u;
        }
        for (int o = 16; o > 0; o >>= 1) {
            e += __shfl_xor_sync(kFull, e, o);
            a += __shfl_xor_sync(kFull, a, o);
            a2 += __shfl_xor_sync(kFull, a2, o);
        }
        d = __reduce_max_sync(kFull, d);
        if (lane == 0) {
            sh_tot[0] = e;
            sh_tot[1] = a;
            sh_tot[2] = a2;
            sh_depth = (int)d - 1;
        }
    }
    __syncthreads();
    const supa_primary pr = p.prim[s];
    const GeomDev &g = p.geoms[pr.geom & 0xFFFFu];
    const float t = tanf(pr.theta);
    const float tx = t * cosf(pr.phi), ty = t * sinf(pr.phi);
    const float inv_dz = 1.0f / g.dz;
    ShowerHits it0;
    it0.init(p.src, s);
    if (it0.remaining <= kShapeCap) {
        // Counting sort of the shower's hits by layer, then one warp per layer
        // reduces its contiguous run: no atomics on the sums.
        for (int pass = 0; pass < 2; ++pass) {
            ShowerHits it;
            it.init(p.src, s);
            if (it.remaining > 0) {
                do {
                    for (int j = threadIdx.x; j < it.seg_len; j += blockDim.x) {
                        const float4 h = __ldg(it.seg_ptr + j);
                        const int l = p.s2l[g.slice_off + (int)rintf(h.z * inv_dz)];  // readout layers only
                        if (l < 0) continue;
                        if (pass == 0)
                            atomicAdd(&lcur[l], 1u);
                        else
                            sorted[atomicAdd(&lcur[l], 1u)] = h;
                    }
                } while (it.next());
            }
            __syncthreads();
            if (pass == 0) {
                if (wid == 0) {  // exclusive scan of the counts (L <= 64: two per lane)
                    const unsigned c0 = lane < L ? lcur[lane] : 0u, c1 = lane + 32 < L ? lcur[lane + 32] : 0u;
                    unsigned s0 = c0, s1 = c1;
                    for (int o = 1; o < 32; o <<= 1) {
                        const unsigned u0 = __shfl_up_sync(kFull, s0, o), u1 = __shfl_up_sync(kFull, s1, o);
                        if (lane >= o) {
                            s0 += u0;
                            s1 += u1;
                        }
                    }
                    const unsigned t0 = __shfl_sync(kFull, s0, 31), t1 = __shfl_sync(kFull, s1, 31);
                    if (lane < L) lstart[lane] = lcur[lane] = s0 - c0;
                    if (lane + 32 < L) lstart[lane + 32] = lcur[lane + 32] = t0 + s1 - c1;
                    if (lane == 0) lstart[L] = t0 + t1;
                }
                __syncthreads();
            }
        }
        for (int l = wid; l < L; l += kShapeThreads / 32) {
            const int a = (int)lstart[l], b = (int)lstart[l + 1];
            if (a == b) continue;
            float v[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            unsigned mx = 0u;
            for (int j = a + lane; j < b; j += 32) {
                const float4 h = sorted[j];
                const float eta = h.x - fmaf(h.z, tx, pr.x0), phi = h.y - fmaf(h.z, ty, pr.y0);
                const float r = sqrtf(fmaf(eta, eta, phi * phi));
                v[0] += eta; v[1] += phi; v[2] += r; v[3] += h.w;
                v[4] += h.w * eta; v[5] += h.w * phi; v[6] += h.w * r;
                mx = max(mx, __float_as_uint(h.w));  // positive floats order as integers
            }
#pragma unroll
            for (int c = 0; c < 7; ++c) v[c] = warp_allsum(v[c]);
            mx = __reduce_max_sync(kFull, mx);
            const float n = (float)(b - a), in = 1.0f / n, iE = v[3] > 0.0f ? 1.0f / v[3] : 0.0f;
            const float mu[7] = {v[0] * in, v[1] * in, v[2] * in, v[3] * in, v[4] * iE, v[5] * iE, v[6] * iE};
            float q[7] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            unsigned nt = 0u, mx2 = 0u;
            for (int j = a + lane; j < b; j += 32) {
                const float4 h = sorted[j];
                const float eta = h.x - fmaf(h.z, tx, pr.x0), phi = h.y - fmaf(h.z, ty, pr.y0);
                const float r = sqrtf(fmaf(eta, eta, phi * phi));
                const float de = eta - mu[0], dp = phi - mu[1], dr = r - mu[2], dE = h.w - mu[3];
                const float we = eta - mu[4], wp = phi - mu[5], wr = r - mu[6];
                q[0] += de * de; q[1] += dp * dp; q[2] += dr * dr; q[3] += dE * dE;
                q[4] += h.w * we * we; q[5] += h.w * wp * wp; q[6] += h.w * wr * wr;
                const unsigned bits = __float_as_uint(h.w);
                if (bits == mx)
                    ++nt;
                else
                    mx2 = max(mx2, bits);
            }
#pragma unroll
            for (int c = 0; c < 7; ++c) q[c] = warp_allsum(q[c]);
            nt = __reduce_add_sync(kFull, nt);
            mx2 = __reduce_max_sync(kFull, mx2);
            if (lane == 0) {
                acc[l][kSn] = n;
#pragma unroll
                for (int c = 0; c < 7; ++c) {
                    acc[l][kSeta + c] = v[c];
                    acc[l][kQeta + c] = q[c];
                    mean[l][c] = mu[c];
                }
                top1[l] = mx;
                top2[l] = mx2;
                ntop[l] = nt;
            }
        }
        __syncthreads();
    }
    // Larger showers: each warp takes 32 consecutive hits at a time; the hits
    // of one layer among them are summed across lanes first and one lane adds
    // the sums to the shared accumulators.
    for (int pass = 0; pass < 2 && it0.remaining > kShapeCap; ++pass) {
        ShowerHits it;
        it.init(p.src, s);
        if (it.remaining > 0) {
            do {
                for (int j0 = wid * 32; j0 < it.seg_len; j0 += kShapeThreads) {
                    const int j = j0 + lane;
                    int l = -1;
                    float eta = 0.0f, phi = 0.0f, r = 0.0f, E = 0.0f;
                    if (j < it.seg_len) {
                        const float4 h = __ldg(it.seg_ptr + j);
                        l = p.s2l[g.slice_off + (int)rintf(h.z * inv_dz)];  // hits lie in readout layers
                        eta = h.x - fmaf(h.z, tx, pr.x0);
                        phi = h.y - fmaf(h.z, ty, pr.y0);
                        r = sqrtf(fmaf(eta, eta, phi * phi));
                        E = h.w;
                    }
                    unsigned todo = __ballot_sync(kFull, l >= 0);
                    while (todo) {
                        const int l0 = __shfl_sync(kFull, l, __ffs(todo) - 1);
                        const bool in = l == l0;
                        const unsigned m = __ballot_sync(kFull, in);
                        const unsigned bits = __float_as_uint(E);
                        float v[7];
                        if (pass == 0) {
                            v[0] = eta; v[1] = phi; v[2] = r; v[3] = E;
                            v[4] = E * eta; v[5] = E * phi; v[6] = E * r;
                        } else {
                            const float *mu = mean[l0];
                            const float de = eta - mu[0], dp = phi - mu[1], dr = r - mu[2], dE = E - mu[3];
                            const float we = eta - mu[4], wp = phi - mu[5], wr = r - mu[6];
                            v[0] = de * de; v[1] = dp * dp; v[2] = dr * dr; v[3] = dE * dE;
                            v[4] = E * we * we; v[5] = E * wp * wp; v[6] = E * wr * wr;
                        }
#pragma unroll
                        for (int c = 0; c < 7; ++c) v[c] = warp_allsum(in ? v[c] : 0.0f);
                        float *a = acc[l0];
                        if (pass == 0) {
                            const unsigned mx = __reduce_max_sync(kFull, in ? bits : 0u);
                            if (lane == 0) {
                                atomicAdd(&a[kSn], (float)__popc(m));
#pragma unroll
                                for (int c = 0; c < 7; ++c) atomicAdd(&a[kSeta + c], v[c]);
                                atomicMax(&top1[l0], mx);  // positive floats order as integers
                            }
                        } else {
                            const unsigned t1 = top1[l0];
                            const unsigned nt = __popc(__ballot_sync(kFull, in && bits == t1));
                            const unsigned mx2 = __reduce_max_sync(kFull, (in && bits != t1) ? bits : 0u);
                            if (lane == 0) {
#pragma unroll
                                for (int c = 0; c < 7; ++c) atomicAdd(&a[kQeta + c], v[c]);
                                if (nt) atomicAdd(&ntop[l0], nt);
                                atomicMax(&top2[l0], mx2);
                            }
                        }
                        todo &= ~m;
                    }
                }
            } while (it.next());
        }
        __syncthreads();
        if (pass == 0) {
            for (int l = threadIdx.x; l < L; l += blockDim.x) {
                const float n = acc[l][kSn], E = acc[l][kSE];
                const float in = n > 0.0f ? 1.0f / n : 0.0f, iE = E > 0.0f ? 1.0f / E : 0.0f;
                mean[l][0] = acc[l][kSeta] * in;
                mean[l][1] = acc[l][kSphi] * in;
                mean[l][2] = acc[l][kSr] * in;
                mean[l][3] = E * in;
                mean[l][4] = acc[l][kSEeta] * iE;
                mean[l][5] = acc[l][kSEphi] * iE;
                mean[l][6] = acc[l][kSEr] * iE;
            }
            __syncthreads();
        }
    }
    const double Etot = sh_tot[0];
    const float iEtot = Etot > 0.0 ? (float)(1.0 / Etot) : 0.0f;
    float *lf = p.layer_feats + (size_t)srel * L * kShapeLayerFeats;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        const float n = acc[l][kSn], E = acc[l][kSE];
        const float Eb = (float)ls[l];
        float *o = lf + (size_t)l * kShapeLayerFeats;
        o[0] = n;
        o[1] = Eb;
        o[2] = Eb * iEtot;
        if (n > 0.0f) {
            const float in = 1.0f / n, iE = 1.0f / E;
            o[3] = mean[l][0]; o[4] = mean[l][1]; o[5] = mean[l][2];
            o[6] = Eb * in;
            o[7] = sqrtf(acc[l][kQeta] * in); o[8] = sqrtf(acc[l][kQphi] * in);
            o[9] = sqrtf(acc[l][kQr] * in); o[10] = sqrtf(acc[l][kQE] * in);
            o[11] = mean[l][4]; o[12] = mean[l][5]; o[13] = mean[l][6];
            o[14] = sqrtf(acc[l][kWeta] * iE); o[15] = sqrtf(acc[l][kWphi] * iE); o[16] = sqrtf(acc[l][kWr] * iE);
            const float e1 = __uint_as_float(top1[l]);
            const float e2 = ntop[l] >= 2u ? e1 : __uint_as_float(top2[l]);
            o[17] = (e1 - e2) / (e1 + e2);
        } else {
            for (int c = 3; c < kShapeLayerFeats; ++c) o[c] = 0.0f;
        }
    }
    if (threadIdx.x == 0) {
        float *o = p.shower_feats + (size_t)srel * kShapeShowerFeats;
        o[0] = (float)Etot;
        o[1] = (float)sh_depth;
        o[2] = (float)sh_tot[1];
        const double sd = Etot > 0.0 ? sh_tot[1] / Etot : 0.0;
        o[3] = (float)sd;
        o[4] = Etot > 0.0 ? (float)sqrt(fmax(0.0, sh_tot[2] / Etot - sd * sd)) : 0.0f;
    }
}

cudaError_t launch_shower_shapes(const ShapeParams &p, cudaStream_t st) {
    if (p.n_showers <= 0) return cudaSuccess;
    supa_shape_kernel<<<(unsigned)p.n_showers, kShapeThreads, 0, st>>>(p);
    return cudaGetLastError();
}

// Training targets of the surrogate's lateral outputs: for a sub-shower
// entering on slice k0 at (x0, y0) with direction (theta, phi), each hit
// (x, y, z, E) of layer l0 + j (j = 0..29) lies at distance
//   r = |(x, y) - (x0, y0) - (z - k0 dz) (tan theta cos phi, tan theta sin phi)|
// from the sub-shower's axis; R_j = sum E r / sum E over the layer's hits,
// 0 for an empty layer.  One warp per sub-shower, FP32 sums in shared memory.
__global__ void __launch_bounds__(256) lateral_targets_kernel(const LateralParams p) {
    __shared__ float er[8][32], es[8][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int64_t s = (int64_t)blockIdx.x * 8 + w; s < p.n; s += (int64_t)gridDim.x * 8) {
        er[w][lane] = 0.0f;
        es[w][lane] = 0.0f;
        __syncwarp();
        const supa_primary pr = p.prim[s];
        const GeomDev &g = p.geoms[pr.geom & 0xFFFFu];
        const int k0 = (int)(pr.geom >> 16);
        const int l0 = k0 < g.n_slices ? (int)p.s2l[g.slice_off + k0] : -1;
        if (l0 >= 0) {
            const float t = tanf(pr.theta);
            const float tx = t * cosf(pr.phi), ty = t * sinf(pr.phi);
            const float z0 = (float)k0 * g.dz;
            ShowerHits it;
            it.init(p.src, s);
            if (it.remaining > 0) {
                do {
                    for (int j = lane; j < it.seg_len; j += 32) {
                        const float4 h = __ldg(it.seg_ptr + j);
                        const int k = (int)rintf(h.z / g.dz);
                        const int jj = (k >= 0 && k < g.n_slices) ? (int)p.s2l[g.slice_off + k] - l0 : -1;
                        if (jj >= 0 && jj < kSurLayers) {
                            const float dz = h.z - z0;
                            const float r = hypotf(h.x - fmaf(dz, tx, pr.x0), h.y - fmaf(dz, ty, pr.y0));
                            atomicAdd(&er[w][jj], h.w * r);
                            atomicAdd(&es[w][jj], h.w);
                        }
                    }
                } while (it.next());
            }
        }
        __syncwarp();
        if (lane < kSurLayers)
            p.y[s * 2 * kSurLayers + kSurLayers + lane] = es[w][lane] > 0.0f ? er[w][lane] / es[w][lane] : 0.0f;
        __syncwarp();
    }
}

cudaError_t launch_lateral_targets(const LateralParams &p, cudaStream_t st) {
    if (p.n <= 0) return cudaSuccess;
    lateral_targets_kernel<<<(unsigned)std::min<int64_t>((p.n + 7) / 8, 16384), 256, 0, st>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_profiles(const ProfileParams &p, cudaStream_t st) {
    if (p.n_showers <= 0) return cudaSuccess;
    supa_profile_kernel<<<(unsigned)p.n_showers, 256, p.nbins * sizeof(float), st>>>(p);
    return cudaGetLastError();
}

// ----------------------------------------------------------------- scan ---
// Exclusive scan of per-shower hit counts into int64 offsets [n+1]:
// per-block totals, a single-block scan of the totals, then the final pass.
namespace {
__device__ __forceinline__ long long block_exclusive_scan(long long v, long long *warp_tot, long long &total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    long long inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(kFull, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long x = (lane < (int)(blockDim.x >> 5)) ? warp_tot[lane] : 0;
        long long xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const long long t = __shfl_up_sync(kFull, xi, o);
            if (lane >= o) xi += t;
        }
        warp_tot[lane] = xi - x;  // exclusive per-warp offsets
        if (lane == 31) warp_tot[32] = xi;
    }
    __syncthreads();
    const long long res = warp_tot[wid] + inc - v;
    total = warp_tot[32];
    __syncthreads();
    return res;
}
}  // namespace

__global__ void __launch_bounds__(kScanThreads) scan_block_totals(const uint32_t *c, int64_t n, unsigned long long *bt) {
    __shared__ long long wt[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v = 0;
    for (int i = 0; i < kScanItems; ++i)
        if (base + i < n) v += c[base + i];
    long long total;
    block_exclusive_scan(v, wt, total);
    if (threadIdx.x == 0) bt[blockIdx.x] = (unsigned long long)total;
}

__global__ void __launch_bounds__(kScanThreads) scan_totals(unsigned long long *bt, int64_t nb) {
    __shared__ long long wt[33];
    long long carry = 0;
    for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int64_t i = b0 + threadIdx.x;
        const long long v = i < nb ? (long long)bt[i] : 0;
        long long total;
        const long long ex = block_exclusive_scan(v, wt, total);
        if (i < nb) bt[i] = (unsigned long long)(carry + ex);
        carry += total;
    }
    if (threadIdx.x == 0) bt[nb] = (unsigned long long)carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_final(const uint32_t *c, int64_t n, const unsigned long long *bt,
                                                           int64_t nb, int64_t *off) {
    __shared__ long long wt[33];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    long long v[kScanItems];
    long long sum = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? (long long)c[base + i] : 0;
        sum += v[i];
    }
    long long total;
    long long ex = block_exclusive_scan(sum, wt, total) + (long long)bt[blockIdx.x];
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) off[base + i] = ex;
        ex += v[i];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[n] = (int64_t)bt[nb];
}

size_t scan_tmp_elems(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile) + 1; }

cudaError_t launch_scan_counts(const uint32_t *counts, int64_t n, int64_t *offsets, unsigned long long *block_tmp,
                               cudaStream_t st) {
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb > 0) scan_block_totals<<<(unsigned)nb, kScanThreads, 0, st>>>(counts, n, block_tmp);
    scan_totals<<<1, kScanThreads, 0, st>>>(block_tmp, nb);
    scan_final<<<(unsigned)(nb > 0 ? nb : 1), kScanThreads, 0, st>>>(counts, n, block_tmp, nb, offsets);
    return cudaGetLastError();
}

// ---------------------------------------------------------- LPT queue ---
// Hand showers out by decreasing primary energy (longest work first): a
// counting sort of the showers into 256 buckets of log2(E) at 1/4 octave.
namespace {
constexpr int kBuckets = 256;
__device__ __forceinline__ int energy_bucket(float E) {
    const int b = (int)floorf(log2f(fmaxf(E, 1e-30f)) * 4.0f) + 64;
    return kBuckets - 1 - min(max(b, 0), kBuckets - 1);  // high energy first
}
}  // namespace

__global__ void lpt_histogram(const supa_primary *prim, int64_t n, uint32_t *cnt) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&cnt[energy_bucket(prim[i].E)], 1u);
}

__global__ void lpt_scan(uint32_t *cnt) {
    __shared__ long long wt[33];
    const long long v = threadIdx.x < kBuckets ? cnt[threadIdx.x] : 0;
    long long total;
    const long long ex = block_exclusive_scan(v, wt, total);
    if (threadIdx.x < kBuckets) cnt[threadIdx.x] = (uint32_t)ex;
}

__global__ void lpt_scatter(const supa_primary *prim, int64_t n, uint32_t *cursor, uint32_t *queue) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pos = atomicAdd(&cursor[energy_bucket(prim[i].E)], 1u);
        queue[pos] = (uint32_t)i;
    }
}

cudaError_t launch_lpt_queue(const supa_primary *prim, int64_t n, uint32_t *queue, uint32_t *bucket_cnt,
                             cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bucket_cnt, 0, kBuckets * sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    const int blocks = (int)imin64((n + 255) / 256, 4096);
    if (blocks == 0) return cudaSuccess;
    lpt_histogram<<<blocks, 256, 0, st>>>(prim, n, bucket_cnt);
    lpt_scan<<<1, kBuckets, 0, st>>>(bucket_cnt);
    lpt_scatter<<<blocks, 256, 0, st>>>(prim, n, bucket_cnt, queue);
    return cudaGetLastError();
}

}  // namespace supa
