// aux_kernels.cu -- downsampling (App. A.5), hit fetch, offset scan and the
// energy-ordered work queue of the SUPA library.
#include <algorithm>

#include "supa_internal.cuh"

namespace supa {

namespace {
constexpr unsigned kFull = 0xFFFFFFFFu;

__host__ __device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

// Walks the hits of one shower as contiguous segments.  In pages mode the
// stepped hits of shower s start at hit_start[s] in the pool and continue
// along page_next; in contiguous mode they are hits[offsets[s] ...).  On the
// hybrid path the shower's surrogate hits follow as one more segment.
struct ShowerHits {
    const float4 *seg_ptr;  // current contiguous segment
    int seg_len;
    int64_t remaining;      // hits from the current segment on (both phases)
    int64_t rem_main;       // stepped hits from the current segment on
    int page;
    int phase;              // 0: stepped hits, 1: surrogate hits
    int64_t s;
    const HitSource *src;

    __device__ void init(const HitSource &hs, int64_t s_) {
        src = &hs;
        s = s_;
        phase = 0;
        const int64_t sur = hs.sur_count ? (int64_t)hs.sur_count[s] : 0;
        if (hs.pool) {
            const unsigned long long st = hs.hit_start[s];
            rem_main = hs.hit_count[s];
            page = (int)(st / kPageHits);
            const int off = (int)(st % kPageHits);
            seg_ptr = hs.pool + st;
            seg_len = (int)imin64(rem_main, kPageHits - off);
        } else {
            const int64_t a = hs.offsets[s], b = hs.offsets[s + 1];
            rem_main = b - a;
            page = -1;
            seg_ptr = hs.hits + a;
            seg_len = (int)imin64(rem_main, (int64_t)1 << 30);
        }
        remaining = rem_main + sur;
        if (rem_main == 0 && sur > 0) enter_surrogate();
    }
    __device__ void enter_surrogate() {
        phase = 1;
        seg_ptr = src->sur_hits + src->sur_off[s];
        seg_len = (int)src->sur_count[s];
    }
    // Advance past the current segment; false when the shower is exhausted.
    __device__ bool next() {
        remaining -= seg_len;
        if (remaining <= 0) return false;
        if (phase == 1) return false;
        rem_main -= seg_len;
        if (rem_main <= 0) {
            enter_surrogate();
        } else if (src->pool) {
            page = src->page_next[page];
            seg_ptr = src->pool + (size_t)page * kPageHits;
            seg_len = (int)imin64(rem_main, kPageHits);
        } else {
            seg_ptr += seg_len;
            seg_len = (int)imin64(rem_main, (int64_t)1 << 30);
        }
        return true;
    }
};

__device__ __forceinline__ double block_sum_double(double v, double *red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) red[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    return t;  // valid in thread 0
}

}  // namespace

// Persistent downsampling kernel (App. A.5: per layer, a region of nx x ny
// cells; each cell sums the energy of the points inside it).  Each CTA takes
// whole showers in turn:
//  1. one pass over the shower's hits computes each hit's layer and cell
//     (float32, half-open cells) into a list in shared memory;
//  2. for each group of G consecutive layers: zero an image buffer in shared
//     memory, add the listed energies with shared-memory atomics, then copy
//     the finished images to HBM with one bulk asynchronous copy
//     (cp.async.bulk, TMA engine).  Two buffers alternate, so binning of one
//     group overlaps the store of the previous one.
// The images of consecutive layers of a shower are contiguous in the
// [shower][layer][ny][nx] layout, so a group is one contiguous store.
// Showers with more hits than the list holds re-read their hits per group.
namespace {
constexpr unsigned kNoCell = 0xFFFFFFFFu;
constexpr int kTouchCap = 2048;  // touched cells remembered per image buffer

// Add E to an image cell; the first deposit into a cell records it so that
// the buffer can be reset cell by cell after its store.
__device__ __forceinline__ void deposit(float *tile, uint32_t *touched, int *n_touched, int cell, float E) {
    const float old = atomicAdd(&tile[cell], E);
    if (old == 0.0f) {
        const int i = atomicAdd(n_touched, 1);
        if (i < kTouchCap) touched[i] = (uint32_t)cell;
    }
}

__device__ __forceinline__ void bulk_store(float *dst, const float *src, unsigned bytes) {
    const unsigned saddr = (unsigned)__cvta_generic_to_shared(src);
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;\n" ::"l"(dst), "r"(saddr), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;\n" ::: "memory");
}

// cell key of a hit: layer << 24 | cell, or kNoCell outside every region
__device__ __forceinline__ unsigned hit_key(const float4 &h, const GeomDev &g, const int8_t *s2l, const float *rx,
                                            const float *ry, const VoxParams &p, bool &dead) {
    const int k = (int)rintf(__fdiv_rn(h.z, g.dz));
    const int layer = (k >= 0 && k < g.n_slices) ? (int)__ldg(s2l + g.slice_off + k) : -1;
    dead = layer < 0;
    if (layer < 0) return kNoCell;
    const float fx = floorf(__fdiv_rn(__fsub_rn(h.x, rx[layer]), p.wx));
    const float fy = floorf(__fdiv_rn(__fsub_rn(h.y, ry[layer]), p.wy));
    if (fx >= 0.0f && fx < (float)p.nx && fy >= 0.0f && fy < (float)p.ny)
        return ((unsigned)layer << 24) | (unsigned)((int)fy * p.nx + (int)fx);
    return kNoCell;
}
}  // namespace

__global__ void __launch_bounds__(512) supa_voxel_kernel(const VoxParams p) {
    extern __shared__ __align__(128) unsigned char vsm[];
    __shared__ float roi_x[SUPA_MAX_LAYERS], roi_y[SUPA_MAX_LAYERS];
    __shared__ double red[32];
    __shared__ int touched_n[2];
    const int cells = p.nx * p.ny;
    const int tile_floats = p.G * cells;
    float *const tile0 = reinterpret_cast<float *>(vsm);
    float *const tile1 = tile0 + tile_floats;
    uint32_t *const touched0 = reinterpret_cast<uint32_t *>(tile1 + tile_floats);
    uint32_t *const touched1 = touched0 + kTouchCap;
    uint2 *list = reinterpret_cast<uint2 *>(touched1 + kTouchCap);
    const float half_x = (float)p.nx * p.wx * 0.5f;
    const float half_y = (float)p.ny * p.wy * 0.5f;
    int phase = 0;
    // Both image buffers start zero and are kept zero between uses: after a
    // buffer's bulk store has been read, only the cells it touched (listed in
    // touched0/1; a full clear if that list overflowed) are reset.
    {
        float4 *t4 = reinterpret_cast<float4 *>(tile0);
        for (int i = threadIdx.x; i < 2 * tile_floats / 4; i += blockDim.x) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (threadIdx.x < 2) touched_n[threadIdx.x] = 0;
    }

    for (int64_t item = blockIdx.x; item < p.n_showers; item += gridDim.x) {
        const int64_t s = p.s_begin + item;
        const GeomDev g = p.geoms[p.single_geom ? 0 : (p.prim[s].geom & 0xFFFFu)];
        for (int l = threadIdx.x; l < p.L; l += blockDim.x) {
            float rx = -half_x, ry = -half_y;
            if (p.roi_x0) {
                if (l < g.n_layers) {
                    rx = p.roi_x0[s * g.n_layers + l];
                    ry = p.roi_y0[s * g.n_layers + l];
                }
            } else if (g.roi_axis && l < g.n_layers) {
                // centred on the incidence axis at the layer's mid depth
                const supa_primary pr = p.prim[s];
                const float t = tanf(pr.theta);
                const float tx = __fmul_rn(t, cosf(pr.phi));
                const float ty = __fmul_rn(t, sinf(pr.phi));
                const float zm = p.zmid[g.layer_off + l];
                rx = __fsub_rn(__fmul_rn(zm, tx), half_x);
                ry = __fsub_rn(__fmul_rn(zm, ty), half_y);
            }
            roi_x[l] = rx;
            roi_y[l] = ry;
        }
        __syncthreads();

        // 1. classify every hit once
        double oor = 0.0;
        ShowerHits it;
        it.init(p.src, s);
        const int64_t count = it.remaining;
        const bool listed = count <= p.list_cap;
        if (count > 0) {
            int64_t base = 0;
            do {
                for (int j = threadIdx.x; j < it.seg_len; j += blockDim.x) {
                    const float4 h = __ldg(it.seg_ptr + j);
                    bool dead;
                    const unsigned key = hit_key(h, g, p.s2l, roi_x, roi_y, p, dead);
                    if (key == kNoCell) oor += (double)h.w;
                    if (listed) list[base + j] = make_uint2(key, __float_as_uint(h.w));
                }
                base += it.seg_len;
            } while (it.next());
        }
        const double tot = block_sum_double(oor, red);
        if (threadIdx.x == 0 && p.oor) p.oor[item] = tot;

        // 2. one image group at a time, double-buffered bulk stores
        for (int grp = 0; grp < p.n_groups; ++grp) {
            const int l0 = grp * p.G;
            const int G = min(p.G, p.L - l0);
            float *tile = phase ? tile1 : tile0;
            uint32_t *touched = phase ? touched1 : touched0;
            // the store issued from this buffer two groups ago must have read it
            if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
            __syncthreads();
            const int nt = touched_n[phase];
            __syncthreads();
            if (threadIdx.x == 0) touched_n[phase] = 0;
            if (nt > kTouchCap) {
                float4 *t4 = reinterpret_cast<float4 *>(tile);
                for (int i = threadIdx.x; i < tile_floats / 4; i += blockDim.x) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            } else {
                for (int i = threadIdx.x; i < nt; i += blockDim.x) tile[touched[i]] = 0.0f;
            }
            __syncthreads();
            if (listed) {
                for (int j = threadIdx.x; j < count; j += blockDim.x) {
                    const uint2 e = list[j];
                    const int li = (int)(e.x >> 24) - l0;
                    if (e.x != kNoCell && li >= 0 && li < G)
                        deposit(tile, touched, &touched_n[phase], li * cells + (int)(e.x & 0xFFFFFFu),
                                __uint_as_float(e.y));
                }
            } else if (count > 0) {
                ShowerHits it2;
                it2.init(p.src, s);
                do {
                    for (int j = threadIdx.x; j < it2.seg_len; j += blockDim.x) {
                        const float4 h = __ldg(it2.seg_ptr + j);
                        bool dead;
                        const unsigned key = hit_key(h, g, p.s2l, roi_x, roi_y, p, dead);
                        const int li = (int)(key >> 24) - l0;
                        if (key != kNoCell && li >= 0 && li < G)
                            deposit(tile, touched, &touched_n[phase], li * cells + (int)(key & 0xFFFFFFu), h.w);
                    }
                } while (it2.next());
            }
            __syncthreads();
            if (threadIdx.x == 0)
                bulk_store(p.grid + ((size_t)item * p.L + l0) * cells, tile, (unsigned)(G * cells) * 4u);
            phase ^= 1;
        }
    }
    // all bulk stores complete (written) before the CTA retires
    if (threadIdx.x == 0) asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory");
}

size_t vox_smem_bytes(int G, int nx, int ny, int list_cap) {
    return (size_t)2 * G * nx * ny * sizeof(float) + (size_t)2 * kTouchCap * sizeof(uint32_t) +
           (size_t)list_cap * 8;
}

void vox_plan(int L, int nx, int ny, int *G, int *n_groups, int *list_cap) {
    const size_t layer_bytes = (size_t)nx * ny * 4;
    int ng = (int)((L * layer_bytes + 32768 - 1) / 32768);
    ng = std::max(1, std::min(ng, L));
    *G = (L + ng - 1) / ng;
    *n_groups = (L + *G - 1) / *G;
    const size_t fixed = 2 * (size_t)(*G) * layer_bytes + 2 * kTouchCap * sizeof(uint32_t);
    const size_t budget = fixed <= 96 * 1024 ? 108 * 1024 : 220 * 1024;
    *list_cap = fixed < budget ? (int)((budget - fixed) / 8) : 0;
}

cudaError_t launch_voxelize(const VoxParams &p, cudaStream_t st) {
    if (p.n_showers == 0) return cudaSuccess;
    const size_t smem = vox_smem_bytes(p.G, p.nx, p.ny, p.list_cap);
    cudaError_t e = cudaFuncSetAttribute(supa_voxel_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(supa_voxel_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, supa_voxel_kernel, 512, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (p.ctas_per_sm > 0) per_sm = std::min(per_sm, p.ctas_per_sm);
    const int64_t grid = std::min<int64_t>((int64_t)sms * per_sm, p.n_showers);
    supa_voxel_kernel<<<(unsigned)grid, 512, smem, st>>>(p);
    return cudaGetLastError();
}

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
                if (p.dst_tags)  // surrogate hits carry no lineage: tag 0
                    p.dst_tags[gidx - lo_hit] =
                        it.phase == 0 ? p.tag_pool[(size_t)(it.seg_ptr - p.src.pool) + j] : 0ull;
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
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

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
