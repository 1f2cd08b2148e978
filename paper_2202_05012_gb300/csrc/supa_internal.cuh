// supa_internal.cuh -- device-side records shared by the SUPA kernels and the
// host code of the C ABI.  Nothing here is visible through include/supa.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/supa.h"

namespace supa {

// Hits live in a pool of fixed-size pages.  A warp writes the hits of the
// shower it is developing at the end of its current page and takes a fresh
// page (linked from the old one through page_next) when the page is full,
// so the hits of one shower form one contiguous run of the warp's page chain.
constexpr int kPageHits = 4096;  // 64 KiB of float4 hits per page

// Per-geometry constants, one record per geometry of a launch.
struct GeomDev {
    int n_slices, n_layers;
    int slice_off;   // first entry of this geometry in the slice tables
    int layer_off;   // first entry of this geometry in the per-layer tables
    float dz, e_min, uz_min;
    float theta_lo, theta_span;  // theta = theta_lo + theta_span * U
    float eps_frac;              // eps = eps_frac * theta * (2U - 1); 0 for SUPA_EPS_ZERO
    int split_literal;           // 1: both daughters deflected by theta/2 + eps
    int nx, ny;
    float wx, wy;
    int roi_axis;
    float e0_max;  // largest primary energy whose lineage ids fit 64 bits
    int thr_off;     // first entry of this geometry in the threshold tables
    int n_regions;   // lateral regions (<= 1: none); region i thresholds at thr_off + i * n_slices
    int region_off;  // first entry of this geometry in the region table
};

// One lateral region (Sec. 4.2): x = squared outer radius (float32, +inf for
// the outermost), y = theta_lo, z = theta_span, w = eps_frac.
using RegionDev = float4;

// ---- hybrid path: particles below E_s handed to the surrogate network ----
constexpr int kSurIn = 6;       // features
constexpr int kSurLayers = 30;  // predicted layers (start layer + 0..29)

// Energy in 64-bit fixed point, units of 2^-32: E = m * 2^(e-23) with a 24-bit
// significand m becomes m << (e + 9), exact for E >= 2^-9 and rounded to the
// nearest unit below (ties up).  Integer shifts only: a float -> int64
// conversion would run on the FP64 unit.  Energies are positive and below
// 2^30 (checked per primary), so the sums cannot overflow.
__device__ __forceinline__ unsigned long long fixed32(float E) {
    const uint32_t bits = __float_as_uint(E);
    const int e = (int)((bits >> 23) & 0xFFu);
    if (e == 0) return 0ull;  // zero (energies are never subnormal here)
    const unsigned long long m = (unsigned long long)((bits & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 127 + 9;
    if (sh >= 0) return m << sh;
    if (sh < -24) return 0ull;
    return (m + (1ull << (-sh - 1))) >> (-sh);
}
__device__ __forceinline__ double from_fixed32(unsigned long long v) {
    return (double)(long long)v * (1.0 / 4294967296.0);
}

// A diverted particle: where it is and what it carries.
// Surrogate network outputs per layer j: o_j (log link: deposit-fraction
// mean mu_j = exp(o_j - kMuShift)), s_j (log-variance), rho_j (mean lateral
// distance); a layer whose mean or drawn fraction is below kFractionMin of the
// particle's energy gets no deposit.
constexpr float kMuShift = 4.0f;
// Floor of the predicted variance of a deposit fraction, e^s_j + kVarFloor.
constexpr float kVarFloor = 1.0e-8f;
constexpr float kFractionMin = 1.0e-6f;

struct SurRec {
    uint32_t shower;  // index in the batch
    int16_t k;        // slice of diversion
    int16_t layer;    // its readout layer
    float x, y;       // position on slice k
    float tx, ty;     // slopes u_x/u_z, u_y/u_z
    float E;
    uint32_t lin_lo, lin_hi;
};

// Per-layer tables used by the features (first slice and slice count).
struct LayerInfo {
    int16_t k_first, n_slices;
};

// The 6 inputs of the surrogate for a particle of energy E on slice k of
// layer l: log(E / E_s), the direction cosines, the position of the slice
// within its layer, and the layers left from l to the back (over 30).
__host__ __device__ inline void surrogate_features(float E, float ux, float uy, float uz, int k, int l, int n_layers,
                                                   LayerInfo li, float e_s, float *f) {
    f[0] = logf(E / e_s);
    f[1] = ux;
    f[2] = uy;
    f[3] = uz;
    f[4] = (float)(k - li.k_first) / (float)li.n_slices;
    const float rem = (float)(n_layers - l) / (float)kSurLayers;
    f[5] = rem < 1.0f ? rem : 1.0f;
}

// Inference buffers for a queue of up to `cap` diverted particles (owned by
// a batch): the network's outputs (f32).
struct SurInfer {
    int cap = 0;
    int ld = 0;            // row stride of OUT
    float *OUT = nullptr;  // network outputs [cap][ld]: o 0..29, s 30..59, rho 60..89
};
int surrogate_infer_init(supa_surrogate *s, int cap, SurInfer *inf);
void surrogate_infer_free(SurInfer *inf);
// Outputs of the first min(*count_dev, cap) rows of feat [cap][6] into inf->OUT.
cudaError_t surrogate_infer_run(supa_surrogate *s, SurInfer *inf, const float *feat, const unsigned *count_dev,
                                cudaStream_t st);

struct SurParams {
    int mode;  // SUPA_SURROGATE_SAMPLE or SUPA_SURROGATE_MEAN
    const SurRec *rec;
    const unsigned *count;  // queue length (device)
    int cap;
    const float *out;       // network outputs [cap][out_ld]: o, s, rho (30 each)
    int out_ld;
    const supa_primary *prim;
    const GeomDev *geoms;
    const float *zmid;
    uint64_t seed, shower_id_base;
    float *dep;             // [cap][30] drawn deposits
    uint8_t *pcnt;          // [cap] hits per diverted particle
    double *lsum;
    int lsum_stride;
    double *sur_leak;       // [n]
    uint32_t *scount;       // [n] surrogate hits per shower
    const int64_t *soff;    // [n+1] exclusive scan of scount
    uint32_t *scursor;      // [n]
    float4 *hits;           // surrogate hit segments
    unsigned long long *tags;  // their lineage tags (bit 63 set), or null
};
cudaError_t launch_sur_deposits(const SurParams &p, cudaStream_t st);
cudaError_t launch_sur_hits(const SurParams &p, cudaStream_t st);
cudaError_t launch_export_diverted(const SurRec *rec, int64_t n, const supa_primary *prim, supa_primary *out,
                                   cudaStream_t st);
cudaError_t launch_export_surrogate(const SurParams &p, int64_t n, supa_diverted_record *out, cudaStream_t st);
cudaError_t launch_add_counts(const uint32_t *a, const uint32_t *b, int64_t n, uint32_t *out, cudaStream_t st);
cudaError_t launch_training_set(const supa_primary *prim, int64_t n, const GeomDev *geoms, const int8_t *s2l,
                                const LayerInfo *linfo, const double *lsum, int stride, float e_s, float *x, float *y,
                                int *bad, cudaStream_t st);

// Particle record of the per-warp global spill stack (36 bytes).
struct SpillRec {
    float x, y, ux, uy, uz, E;
    uint32_t lin_lo, lin_hi;
    int32_t k;
};

struct StepParams {
    // inputs
    const supa_primary *prim;
    const uint32_t *queue;  // order in which showers are handed out (nullptr = identity)
    int64_t n;
    int n_geoms;
    uint64_t seed;
    uint64_t shower_id_base;
    const GeomDev *geoms;
    const unsigned long long *t_stop;  // [slices] stop iff r0 < t_stop
    const unsigned long long *t_ss;    // [slices] split iff t_stop <= r0 < t_ss
    const RegionDev *regions;          // lateral regions of all geometries
    const int8_t *s2l;                 // [slices] layer or -1
    // hit pool
    float4 *pool;
    unsigned long long *tag_pool;  // nullable
    int *page_next;
    int n_pages;
    int *page_counter;
    // per-shower results
    unsigned long long *hit_start;
    uint32_t *hit_count;
    uint32_t *steps;
    double *lsum;
    int lsum_stride;
    double *dead, *leak, *escape;
    // control and totals
    int *queue_head;
    int *error;
    unsigned long long *totals;  // [0] particle-steps, [1] hits
    // scratch
    SpillRec *spill;
    int spill_cap;        // records per warp
    int stack_cap;        // particles per warp in shared memory
    int stage_cap;        // staged hits per warp (flush_thr + 32; 0: hits written directly)
    int flush_thr;        // staged hits that trigger a flush
    int warp_smem_bytes;  // shared memory per warp
    unsigned long long *warp_times;  // [warps][2] start / end global time (ns), or null
    // hybrid path (e_s = 0: off)
    float e_s;
    const LayerInfo *linfo;  // per geometry layer (layer_off + l)
    SurRec *sq_rec;
    float *sq_feat;          // [sq_cap][6]
    unsigned *sq_count;
    int sq_cap;
};

// Record the message returned by supa_last_error() and return `code`.
int set_last_error(int code, const char *msg);

// Device error word bits.
constexpr int kErrPoolOverflow = 1;
constexpr int kErrSpillOverflow = 2;
constexpr int kErrBadPrimary = 4;
constexpr int kErrQueueOverflow = 16;

size_t warp_smem_bytes(int stack_cap, int stage_cap, bool tags);

// Kernel launchers (defined in the .cu files, called by the C ABI).
// minb selects the register budget of the step kernel (3 or 4 resident
// 256-thread blocks per SM: 80 or 64 registers).
cudaError_t launch_step(int minb, bool regions, bool staged, const StepParams &p, int grid, int block, size_t smem,
                        cudaStream_t st);
cudaError_t step_kernel_attributes(int minb, bool regions, bool staged, int block, size_t smem, int *blocks_per_sm);
// Exclusive scan of per-shower counts: kScanTile showers per block of the
// first and last pass; scratch of scan_tmp_elems(n) = ceil(n / kScanTile) + 1
// per-block totals.
// Programmatic dependent launch: a kernel launched with launch_pdl may start
// while the kernel before it in the stream is still running; it runs its
// set-up (barriers, tensor memory) and then pdl_wait()s, which returns once
// every earlier kernel of the stream has completed and its writes are
// visible, before it touches their results or overwrites what they read.
// pdl_trigger() lets the next such kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                       Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
cudaError_t launch_scan_counts(const uint32_t *counts, int64_t n, int64_t *offsets, unsigned long long *block_tmp,
                               cudaStream_t st);
size_t scan_tmp_elems(int64_t n);
cudaError_t launch_lpt_queue(const supa_primary *prim, int64_t n, uint32_t *queue, uint32_t *bucket_cnt,
                             cudaStream_t st);

struct HitSource {
    // pages mode (pool != nullptr) or contiguous mode (hits != nullptr)
    const float4 *pool;
    const int *page_next;
    const unsigned long long *hit_start;
    const uint32_t *hit_count;
    const float4 *hits;
    const int64_t *offsets;
    // hybrid path: surrogate hits follow the stepped ones (null otherwise)
    const float4 *sur_hits;
    const int64_t *sur_off;
    const uint32_t *sur_count;
};

struct VoxParams {
    HitSource src;
    int64_t s_begin, n_showers;
    int L;         // layer stride of the grid
    int G;         // layers per image group (one bulk store)
    int n_groups;  // ceil(L / G)
    int list_cap;  // hits whose cells fit the shared-memory list
    int ctas_per_sm;  // persistent grid size per SM (0: as many as fit)
    int nx, ny;
    float wx, wy;
    // batch mode: ROI from the primaries; explicit mode: roi_x0/roi_y0
    const supa_primary *prim;
    const GeomDev *geoms;
    int single_geom;  // explicit mode: geometry 0 for every shower
    const int8_t *s2l;
    const float *zmid;  // per geometry-layer mid depth (layer_off + l)
    const float *roi_x0, *roi_y0;
    float *grid;
    double *oor;
    // optional: the point cloud of the showers, hit i of shower s at
    // hits_out[offsets[s] + i - hits_base], written in the same pass
    float4 *hits_out;
    const int64_t *offsets;
    int64_t hits_base;
};

cudaError_t launch_voxelize(const VoxParams &p, cudaStream_t st);
size_t vox_smem_bytes(int G, int nx, int ny, int list_cap);
// Layers per group, group count and hit-list capacity for an L x ny x nx image.
void vox_plan(int L, int nx, int ny, int *G, int *n_groups, int *list_cap);

struct ProfileParams {
    HitSource src;
    const supa_primary *prim;
    const double *lsum;  // [n][L]
    int64_t s_begin, n_showers;
    int L, nbins;
    float r_max;
    double *longi, *lat;
};
cudaError_t launch_profiles(const ProfileParams &p, cudaStream_t st);

// Per-layer grids at several resolutions (grids.cu).
constexpr int kMaxGridFactors = 8;
struct LayerGridDev {
    int nx, ny;
    float wx, wy;
};
struct GridParams {
    HitSource src;
    const supa_primary *prim;
    const GeomDev *geoms;
    const int8_t *s2l;
    const float *zmid;
    int64_t s_begin, n_showers;
    int single_geom;
    int n_layers;  // grids given (layers at or past it: out of region)
    LayerGridDev grid[SUPA_MAX_LAYERS];
    int n_res;
    int factor[kMaxGridFactors];
    int base[kMaxGridFactors][SUPA_MAX_LAYERS];  // first cell of (factor, layer) in a shower's images
    int cells;                                   // cells per shower
    float *images;                               // [n_showers][cells]
    double *oor;                                 // [n_showers][n_res], nullable
};
size_t grid_smem_bytes(int cells);
cudaError_t launch_voxelize_layers(const GridParams &p, cudaStream_t st);

// Shower shape variables (Sec. 5.1, App. A.1) of a range of showers.
constexpr int kShapeLayerFeats = 18, kShapeShowerFeats = 5;
struct ShapeParams {
    HitSource src;
    const supa_primary *prim;
    const GeomDev *geoms;
    const int8_t *s2l;
    const double *lsum;  // [n][L]
    int64_t s_begin, n_showers;
    int L;
    float *layer_feats;   // [n_showers][L][18]
    float *shower_feats;  // [n_showers][5]
};
cudaError_t launch_shower_shapes(const ShapeParams &p, cudaStream_t st);

// Training targets R_j (mean lateral distances) of a batch of sub-showers.
struct LateralParams {
    HitSource src;
    const supa_primary *prim;
    const GeomDev *geoms;
    const int8_t *s2l;
    int64_t n;
    float *y;  // [n][60]: columns 30..59 written
};
cudaError_t launch_lateral_targets(const LateralParams &p, cudaStream_t st);

struct FetchParams {
    HitSource src;
    const unsigned long long *tag_pool;  // fetch tags instead of hits when non-null
    int64_t n_showers;
    int64_t first, count;
    float4 *dst;
    unsigned long long *dst_tags;
    const unsigned long long *sur_tags;  // tags of the surrogate hits (hybrid path with record_tags)
};
cudaError_t launch_fetch(const FetchParams &p, cudaStream_t st);

}  // namespace supa
