// grids.cu -- downsampling onto per-layer grids at several resolutions from
// one pass over the hits (App. A.5 "Downsampling" and the grid experiments:
// a CaloGAN-like detector with 3 x 96, 12 x 12 and 12 x 6 cells, at "1x",
// "2x" and "3x").
//
// Layer l has nx_l x ny_l cells of wx_l x wy_l over a region placed like the
// uniform grid's (centred on the z axis, or on the incidence axis at the
// layer's mid depth); at factor f its cells are w / f wide (float32), f times
// as many in each direction.  Cell index floor((x - lo) / w') in float32;
// points outside the region (or in no readout layer) add to that factor's
// out-of-region energy.  One CTA holds all (factor, layer) images of a shower
// in shared memory, adds its hits with shared-memory atomics and writes the
// images out coalesced.
#include <algorithm>

#include "hits.cuh"
#include "supa_internal.cuh"

namespace supa {

namespace {

constexpr int kGridThreads = 256;

__global__ void __launch_bounds__(kGridThreads) supa_grid_kernel(const __grid_constant__ GridParams p) {
    extern __shared__ __align__(16) float img[];
    __shared__ float lo_x[SUPA_MAX_LAYERS], lo_y[SUPA_MAX_LAYERS];
    __shared__ double red[kGridThreads / 32][kMaxGridFactors];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int64_t item = blockIdx.x; item < p.n_showers; item += gridDim.x) {
        const int64_t s = p.s_begin + item;
        const supa_primary pr = p.prim[s];
        const GeomDev g = p.geoms[p.single_geom ? 0 : (pr.geom & 0xFFFFu)];
        for (int i = threadIdx.x; i < p.cells; i += blockDim.x) img[i] = 0.0f;
        for (int l = threadIdx.x; l < p.n_layers; l += blockDim.x) {
            const LayerGridDev gr = p.grid[l];
            const float half_x = __fmul_rn(__fmul_rn((float)gr.nx, gr.wx), 0.5f);
            const float half_y = __fmul_rn(__fmul_rn((float)gr.ny, gr.wy), 0.5f);
            float rx = -half_x, ry = -half_y;
            if (g.roi_axis && l < g.n_layers) {
                const float t = tanf(pr.theta);
                const float tx = __fmul_rn(t, cosf(pr.phi));
                const float ty = __fmul_rn(t, sinf(pr.phi));
                const float zm = p.zmid[g.layer_off + l];
                rx = __fsub_rn(__fmul_rn(zm, tx), half_x);
                ry = __fsub_rn(__fmul_rn(zm, ty), half_y);
            }
            lo_x[l] = rx;
            lo_y[l] = ry;
        }
        __syncthreads();
        float out[kMaxGridFactors];
#pragma unroll
        for (int r = 0; r < kMaxGridFactors; ++r) out[r] = 0.0f;
        ShowerHits it;
        it.init(p.src, s);
        if (it.remaining > 0) {
            do {
                for (int j = threadIdx.x; j < it.seg_len; j += blockDim.x) {
                    const float4 h = __ldg(it.seg_ptr + j);
                    const int k = (int)rintf(__fdiv_rn(h.z, g.dz));
                    const int l = (k >= 0 && k < g.n_slices) ? (int)__ldg(p.s2l + g.slice_off + k) : -1;
                    if (l < 0 || l >= p.n_layers) {
#pragma unroll
                        for (int r = 0; r < kMaxGridFactors; ++r)
                            if (r < p.n_res) out[r] += h.w;
                        continue;
                    }
                    const LayerGridDev gr = p.grid[l];
                    const float dx = __fsub_rn(h.x, lo_x[l]), dy = __fsub_rn(h.y, lo_y[l]);
#pragma unroll
                    for (int r = 0; r < kMaxGridFactors; ++r) {
                        if (r >= p.n_res) break;
                        const int f = p.factor[r];
                        const float fx = floorf(__fdiv_rn(dx, __fdiv_rn(gr.wx, (float)f)));
                        const float fy = floorf(__fdiv_rn(dy, __fdiv_rn(gr.wy, (float)f)));
                        const int nxf = gr.nx * f, nyf = gr.ny * f;
                        if (fx >= 0.0f && fx < (float)nxf && fy >= 0.0f && fy < (float)nyf)
                            atomicAdd(&img[p.base[r][l] + (int)fy * nxf + (int)fx], h.w);
                        else
                            out[r] += h.w;
                    }
                }
            } while (it.next());
        }
        __syncthreads();
        float *dst = p.images + (size_t)item * p.cells;
        if ((p.cells & 3) == 0) {
            const float4 *src4 = reinterpret_cast<const float4 *>(img);
            float4 *dst4 = reinterpret_cast<float4 *>(dst);
            for (int i = threadIdx.x; i < p.cells / 4; i += blockDim.x) dst4[i] = src4[i];
        } else {
            for (int i = threadIdx.x; i < p.cells; i += blockDim.x) dst[i] = img[i];
        }
        if (p.oor) {
#pragma unroll
            for (int r = 0; r < kMaxGridFactors; ++r) {
                double v = (double)out[r];
                for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
                if (lane == 0) red[wid][r] = v;
            }
        }
        __syncthreads();
        if (p.oor && threadIdx.x < p.n_res) {
            double v = 0.0;
            for (int w = 0; w < kGridThreads / 32; ++w) v += red[w][threadIdx.x];
            p.oor[item * p.n_res + threadIdx.x] = v;
        }
    }
}

}  // namespace

size_t grid_smem_bytes(int cells) { return (size_t)cells * sizeof(float); }

cudaError_t launch_voxelize_layers(const GridParams &p, cudaStream_t st) {
    if (p.n_showers <= 0) return cudaSuccess;
    const size_t smem = grid_smem_bytes(p.cells);
    cudaError_t e = cudaFuncSetAttribute(supa_grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, supa_grid_kernel, kGridThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t grid = std::min<int64_t>(p.n_showers, (int64_t)sms * std::max(1, per_sm));
    supa_grid_kernel<<<(unsigned)grid, kGridThreads, smem, st>>>(p);
    return cudaGetLastError();
}

}  // namespace supa
