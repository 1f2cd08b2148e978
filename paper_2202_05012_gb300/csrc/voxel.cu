// voxel.cu -- downsampling of the point clouds onto the uniform per-layer
// grid (App. A.5 "Downsampling"), optionally writing the point clouds out in
// shower order in the same pass over the hits.
#include <algorithm>

#include "hits.cuh"
#include "supa_internal.cuh"

namespace supa {

namespace {
constexpr unsigned kFull = 0xFFFFFFFFu;

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
//     (float32, half-open cells), sums the out-of-region energy and counts
//     the hits per layer (the bucket sizes of a counting sort by layer);
//  2. the layers are taken in windows of image groups whose hits fit a list
//     in shared memory: a second read of the hits (L2-resident by now)
//     scatters the window's (cell, energy) pairs into the list by layer --
//     except for images of at most kScanGroups groups whose shower fits the
//     list, where pass 1 writes the list unsorted and every group scans it;
//  3. for each group of G consecutive layers: zero an image buffer in shared
//     memory, add its own bucket of energies with shared-memory atomics,
//     then copy the finished images to HBM with one bulk asynchronous copy
//     (cp.async.bulk, TMA engine).  Two buffers alternate, so binning of one
//     group overlaps the store of the previous one.
// The images of consecutive layers of a shower are contiguous in the
// [shower][layer][ny][nx] layout, so a group is one contiguous store.  A
// single group with more hits than the list holds bins straight from the
// hits.
namespace {
constexpr unsigned kNoCell = 0xFFFFFFFFu;
constexpr int kTouchCap = 2048;  // touched cells remembered per image buffer
constexpr int kScanGroups = 16;  // up to this many image groups a group scans the whole hit list

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
    // touched-cell counts per image buffer, two per buffer alternating by use:
    // a use adds to one while the next use still reads the other
    __shared__ int touched_n[2][2];
    __shared__ int lcount[SUPA_MAX_LAYERS], lstart[SUPA_MAX_LAYERS + 1], cursor[SUPA_MAX_LAYERS];
    const int cells = p.nx * p.ny;
    const int tile_floats = p.G * cells;
    float *const tile0 = reinterpret_cast<float *>(vsm);
    float *const tile1 = tile0 + tile_floats;
    uint32_t *const touched0 = reinterpret_cast<uint32_t *>(tile1 + tile_floats);
    uint32_t *const touched1 = touched0 + kTouchCap;
    uint2 *list = reinterpret_cast<uint2 *>(touched1 + kTouchCap);
    const float half_x = (float)p.nx * p.wx * 0.5f;
    const float half_y = (float)p.ny * p.wy * 0.5f;
    int phase = 0;  // image buffer of the next group
    int n_use = 0;  // groups binned so far (buffer uses: n_use >> 1 per buffer)
    // Both image buffers start zero and are kept zero between uses: after a
    // buffer's bulk store has been read, only the cells it touched (listed in
    // touched0/1; a full clear if that list overflowed) are reset.
    {
        float4 *t4 = reinterpret_cast<float4 *>(tile0);
        for (int i = threadIdx.x; i < 2 * tile_floats / 4; i += blockDim.x) t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (threadIdx.x < 4) touched_n[threadIdx.x >> 1][threadIdx.x & 1] = 0;
        for (int l = threadIdx.x; l < SUPA_MAX_LAYERS; l += blockDim.x) lcount[l] = 0;
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

        // 1. classify every hit once: out-of-region energy, per-layer counts
        //    (and, in supa_voxelize_fetch, the point cloud)
        double oor = 0.0;
        ShowerHits it;
        it.init(p.src, s);
        const int64_t count = it.remaining;
        // few image groups and a list that holds every hit: each group scans
        // the whole (unsorted) list; otherwise the counting sort by layer
        const bool scan_all = count <= p.list_cap && p.n_groups <= kScanGroups;
        if (count > 0) {
            int64_t base = 0;
            float4 *const out = p.hits_out ? p.hits_out + (p.offsets[s] - p.hits_base) : nullptr;
            do {
                for (int j = threadIdx.x; j < it.seg_len; j += blockDim.x) {
                    const float4 h = __ldg(it.seg_ptr + j);
                    if (out) out[base + j] = h;  // the point cloud, in shower order
                    bool dead;
                    const unsigned key = hit_key(h, g, p.s2l, roi_x, roi_y, p, dead);
                    if (key == kNoCell)
                        oor += (double)h.w;
                    if (scan_all)
                        list[base + j] = make_uint2(key, __float_as_uint(h.w));
                    else if (key != kNoCell)
                        atomicAdd(&lcount[key >> 24], 1);
                }
                base += it.seg_len;
            } while (it.next());
        }
        const double tot = block_sum_double(oor, red);
        if (threadIdx.x == 0 && p.oor) p.oor[item] = tot;
        if (!scan_all && threadIdx.x == 0) {
            // bucket starts of the counting sort by layer
            int a = 0;
            for (int l = 0; l < p.L; ++l) {
                lstart[l] = a;
                cursor[l] = a;
                a += lcount[l];
                lcount[l] = 0;
            }
            lstart[p.L] = a;
        }
        __syncthreads();

        // 2. windows of consecutive image groups whose hits fit the list:
        //    the window's hits are sorted into it by layer (a second read of
        //    the shower's hits, from L2), then each group deposits only its
        //    own bucket -- one image group at a time, double-buffered bulk
        //    stores.  A single group with more hits than the list holds
        //    deposits straight from the hits.
        for (int gb = 0; gb < p.n_groups;) {
            const int lb = gb * p.G;
            int ge = scan_all ? p.n_groups : gb + 1;
            while (ge < p.n_groups && lstart[min(p.L, (ge + 1) * p.G)] - lstart[lb] <= p.list_cap) ++ge;
            const bool fits = scan_all || lstart[min(p.L, ge * p.G)] - lstart[lb] <= p.list_cap;
            const int le = min(p.L, ge * p.G);
            if (!scan_all && fits && lstart[le] > lstart[lb]) {
                ShowerHits it1;
                it1.init(p.src, s);
                do {
                    for (int j = threadIdx.x; j < it1.seg_len; j += blockDim.x) {
                        const float4 h = __ldg(it1.seg_ptr + j);
                        bool dead;
                        const unsigned key = hit_key(h, g, p.s2l, roi_x, roi_y, p, dead);
                        const int l = (int)(key >> 24);
                        if (key != kNoCell && l >= lb && l < le)
                            list[atomicAdd(&cursor[l], 1) - lstart[lb]] = make_uint2(key, __float_as_uint(h.w));
                    }
                } while (it1.next());
                __syncthreads();
            }
            for (int grp = gb; grp < ge; ++grp) {
                const int l0 = grp * p.G;
                const int G = min(p.G, p.L - l0);
                float *tile = phase ? tile1 : tile0;
                uint32_t *touched = phase ? touched1 : touched0;
                // this buffer's use number u = n_use >> 1: its deposits count
                // in touched_n[phase][u & 1]; use u - 1 counted in the other
                const int cu = (n_use >> 1) & 1;
                int *const tn = &touched_n[phase][cu];
                // the store issued from this buffer two groups ago must have
                // read it; the counter of use u - 2 was read by use u - 1
                if (threadIdx.x == 0) {
                    asm volatile("cp.async.bulk.wait_group.read 1;\n" ::: "memory");
                    *tn = 0;
                }
                __syncthreads();
                const int nt = touched_n[phase][cu ^ 1];
                if (nt > kTouchCap) {
                    float4 *t4 = reinterpret_cast<float4 *>(tile);
                    for (int i = threadIdx.x; i < tile_floats / 4; i += blockDim.x)
                        t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                } else {
                    for (int i = threadIdx.x; i < nt; i += blockDim.x) tile[touched[i]] = 0.0f;
                }
                __syncthreads();
                if (scan_all) {
                    for (int j = threadIdx.x; j < count; j += blockDim.x) {
                        const uint2 e = list[j];
                        const int li = (int)(e.x >> 24) - l0;
                        if (e.x != kNoCell && li >= 0 && li < G)
                            deposit(tile, touched, tn, li * cells + (int)(e.x & 0xFFFFFFu),
                                    __uint_as_float(e.y));
                    }
                } else if (fits) {
                    const int j1 = lstart[l0 + G] - lstart[lb];
                    for (int j = lstart[l0] - lstart[lb] + threadIdx.x; j < j1; j += blockDim.x) {
                        const uint2 e = list[j];
                        deposit(tile, touched, tn, ((int)(e.x >> 24) - l0) * cells + (int)(e.x & 0xFFFFFFu),
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
                                deposit(tile, touched, tn, li * cells + (int)(key & 0xFFFFFFu), h.w);
                        }
                    } while (it2.next());
                }
                // each thread orders its own shared-memory writes of the tile
                // before the async-proxy read of the bulk copy
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                __syncthreads();
                if (threadIdx.x == 0)
                    bulk_store(p.grid + ((size_t)item * p.L + l0) * cells, tile, (unsigned)(G * cells) * 4u);
                phase ^= 1;
                ++n_use;
            }
            gb = ge;
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

}  // namespace supa
