/*
 * supa.h -- C ABI of the GB300 SUPA shower library (libsupa.so).
 *
 * SUPA (Sinha et al., "SUPA: A Lightweight Diagnostic Simulator for Machine
 * Learning in Particle Physics", arXiv 2202.05012) develops a shower by
 * applying one rule to every live particle at every slice of a layered
 * detector (Sec. 3, Algorithm 1): stop and deposit the energy, split into two
 * daughters, or pass through.  Deposits are grouped into readout layers
 * (Sec. 3, "layer configuration") and can be downsampled into per-layer
 * images (App. A.5, "Downsampling").  This library runs that process for
 * batches of showers on one GPU.
 *
 * Conventions for every entry point:
 *  - The return value is a status: SUPA_OK (0) or a negative SUPA_ERR_* code.
 *    supa_last_error() gives a message for the last failure on the calling
 *    thread.
 *  - Pointers named *_dev are device pointers; every other pointer is a host
 *    pointer.  Buffers passed in stay owned by the caller; the library only
 *    reads inputs and writes outputs.  Handles (supa_geometry, supa_batch)
 *    are created and destroyed by the library.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Calls
 *    that take a stream are asynchronous on it unless stated otherwise;
 *    device-side errors (pool overflow) surface at the next synchronising
 *    call on the batch (supa_batch_get_info).
 *  - Layouts: a hit is four float32 (x, y, z, E) = 16 bytes; images are
 *    float32 [shower][layer][ny][nx] with x fastest.
 */
#ifndef SUPA_H
#define SUPA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SUPA_OK 0
#define SUPA_ERR_INVALID_ARG (-1)
#define SUPA_ERR_OOM (-2)
#define SUPA_ERR_OVERFLOW (-3)
#define SUPA_ERR_TIMEOUT (-4)
#define SUPA_ERR_CUDA (-5)
#define SUPA_ERR_NOT_READY (-6)

#define SUPA_MAX_SLICES 255
#define SUPA_MAX_LAYERS 64
#define SUPA_MAX_GEOMS 8
#define SUPA_MAX_REGIONS 8

/* Split-angle laws p_theta and p_eps (Algorithm 1 "Parameters"; Table 2). */
#define SUPA_THETA_FIXED 0   /* theta = theta_lo                          */
#define SUPA_THETA_UNIFORM 1 /* theta ~ U(theta_lo, theta_hi)             */
#define SUPA_EPS_ZERO 0      /* eps = 0: symmetric splits (SUPAv1, v2)    */
#define SUPA_EPS_UNIFORM 1   /* eps ~ U(-f theta, f theta), f = eps_frac  */
/* Daughter kinematics (Sec. 3 "momentum conservation"; Algorithm 1).
 * MOMENTUM: daughter 0 gets E(theta/2+eps)/theta and is deflected by
 * theta/2-eps at azimuth omega, daughter 1 gets the rest and is deflected by
 * theta/2+eps at omega+pi (opening angle theta, E_0 delta_0 = E_1 delta_1).
 * LITERAL: both deflected by theta/2+eps, as the position lines of
 * Algorithm 1 read. */
#define SUPA_SPLIT_MOMENTUM 0
#define SUPA_SPLIT_LITERAL 1
/* Region of interest of each layer image (App. A.5). */
#define SUPA_ROI_FIXED 0 /* centred on the z axis                           */
#define SUPA_ROI_AXIS 1  /* centred on the incidence axis at mid-layer depth */

/* Geometry and model parameters (Algorithm 1 "Parameters"; Sec. 4.2 dead
 * material).  All arrays are host arrays of n_slices entries, copied.
 *
 * Lateral regions (Sec. 4.2: the slices may be divided into regions, each
 * with its own meta-parameters).  n_regions 0 or 1: none.  Otherwise
 * (2..SUPA_MAX_REGIONS) concentric regions around the z axis: a particle at
 * (x, y) on slice k is in region i when region_radius[i-1] <= r <
 * region_radius[i] (region_radius[-1] = 0, region_radius[n_regions-1] =
 * infinity), decided in float32 as x*x + y*y (one fma) < b*b with b the
 * float32 radius.  Region i then takes region_p_stop / region_p_split row i
 * ([n_regions][n_slices], row-major), region_theta_lo[i] / theta_hi[i] and
 * region_eps_frac[i] in place of p_stop, p_split, theta_lo, theta_hi and
 * eps_frac (theta_mode, eps_mode, split_mode, e_min and uz_min stay
 * global).  The same range rules apply per region; radii must be positive
 * and increasing. */
typedef struct {
    int32_t n_slices;              /* slices z_k = k*dz, k = 0..n_slices-1 (1..255) */
    float dz;                      /* slice gap Delta z (> 0)                       */
    const int32_t *slice_to_layer; /* layer of each slice, -1 = dead material       */
    int32_t n_layers;              /* readout layers (1..64)                        */
    const double *p_stop;          /* p_stop[k] in [0,1]                            */
    const double *p_split;         /* p_split[k], p_stop[k] + p_split[k] <= 1       */
    int32_t theta_mode;            /* SUPA_THETA_*                                  */
    double theta_lo, theta_hi;     /* radians, 0 < theta_lo <= theta_hi < pi/2      */
    int32_t eps_mode;              /* SUPA_EPS_*                                    */
    double eps_frac;               /* 0 <= eps_frac < 1/2                           */
    int32_t split_mode;            /* SUPA_SPLIT_*                                  */
    double e_min;                  /* energy cut: E < e_min stops (0 = no cut)      */
    double uz_min;                 /* a survivor with u_z <= uz_min escapes (> 0)   */
    int32_t nx, ny;                /* image cells per layer; nx*ny multiple of 4    */
    float wx, wy;                  /* cell size                                     */
    int32_t roi_mode;              /* SUPA_ROI_*                                    */
    int32_t n_regions;             /* lateral regions (0/1: none)                   */
    const double *region_radius;   /* [n_regions-1] increasing outer radii          */
    const double *region_p_stop;   /* [n_regions][n_slices]                         */
    const double *region_p_split;  /* [n_regions][n_slices]                         */
    const double *region_theta_lo; /* [n_regions]                                   */
    const double *region_theta_hi; /* [n_regions]                                   */
    const double *region_eps_frac; /* [n_regions]                                   */
} supa_geometry_desc;

/* One primary particle (Sec. 3 initial particle; Sec. 4.2 conditioning on
 * impact energy, angle and position): energy, impact point, polar angle from
 * the z axis and azimuth (radians).  `geom`: bits 0-15 index the launch's
 * geometry list, bits 16-31 give the slice the particle enters on (0 for a
 * shower; later slices start sub-showers, e.g. surrogate training data).
 * 24 bytes, no padding. */
typedef struct {
    float E, x0, y0, theta, phi;
    uint32_t geom;
} supa_primary;

/* Launch tuning; zero fields pick defaults (or the autotuned values). */
typedef struct {
    int32_t warps_per_block; /* warps of the persistent step kernel (<= 8)   */
    int32_t blocks_per_sm;   /* step-kernel blocks per SM (1..4; 4 selects a  */
                             /* 64-register build, fewer an 80-register one) */
    int32_t stack_depth;     /* particles held per warp in shared memory     */
    int32_t flush_threshold; /* hits staged per warp in shared memory before */
                             /* a coalesced flush to HBM (<= 1024; 0: 128);   */
                             /* -1: each step's hits written straight from   */
                             /* the lanes (no staging)                       */
    int32_t record_tags;     /* 1: also keep each hit's lineage id           */
    int32_t lpt_order;       /* 1: hand out showers by decreasing energy     */
    int32_t voxel_ctas_per_sm; /* downsampling CTAs per SM (0: as many as fit);
                                  1 leaves room on every SM for step-kernel
                                  blocks of another batch to run alongside  */
    int64_t max_hits;        /* hit pool capacity (0: sized from free memory)*/
    int32_t record_warp_times; /* 1: every step-kernel warp records when it
                                  starts and when it runs out of showers
                                  (supa_batch_warp_times)                    */
} supa_launch_config;

/* Per-batch results after a simulation (device pointers stay owned by the
 * batch and valid until the next simulation or supa_destroy_batch). */
typedef struct {
    int64_t n_showers;
    int64_t n_hits;             /* total hits                                  */
    int64_t n_steps;            /* particle-slice visits (particle-steps)      */
    int32_t max_layers;         /* stride of layer_sums_dev                    */
    int32_t status;             /* SUPA_OK or the device-side error            */
    const int64_t *offsets_dev; /* [n+1] first hit of each shower, shower order */
    const uint32_t *counts_dev; /* [n] hits per shower                         */
    const uint32_t *steps_dev;  /* [n] particle-steps per shower               */
    const double *layer_sums_dev; /* [n][max_layers] FP64 deposit per layer    */
    const double *dead_dev;     /* [n] energy stopped in dead slices           */
    const double *leak_dev;     /* [n] energy alive after the last slice       */
    const double *escape_dev;   /* [n] energy of escaped particles             */
    int64_t n_diverted;         /* hybrid path: particles handed to the network */
    const double *sur_leak_dev; /* hybrid path: [n] energy the network did not
                                   deposit (NULL on the plain path)            */
} supa_batch_info;

typedef struct supa_geometry supa_geometry;
typedef struct supa_batch supa_batch;

/* Message for the last failed call on this thread ("" if none). */
const char *supa_last_error(void);

/* Validate a geometry and upload its per-slice tables (thresholds for the
 * stop/split/pass draw of Algorithm 1).  Rejects p outside [0,1],
 * p_stop + p_split > 1, layer ids out of range, and parameters whose lineage
 * ids could exceed 64 bits (more than 62 splits on one path). */
int supa_init_geometry(const supa_geometry_desc *desc, supa_geometry **out);
int supa_destroy_geometry(supa_geometry *g);

/* Allocate a reusable batch for up to max_showers showers over the given
 * geometries (1..SUPA_MAX_GEOMS, which must outlive the batch).  cfg may be
 * NULL.  Synchronous (allocates device memory). */
int supa_batch_create(const supa_geometry *const *geoms, int32_t n_geoms, int64_t max_showers,
                      const supa_launch_config *cfg, supa_batch **out);
int supa_destroy_batch(supa_batch *b);

/* Develop n showers (Algorithm 1 applied to every particle at every slice,
 * Sec. 3).  Shower i uses primary prim_dev[i] and the global id
 * shower_id_base + i, which keys its random stream together with the slice
 * and the particle's lineage id, so any shower can be replayed alone.
 * Asynchronous on `stream`; launches kernels only (no allocation, no host
 * synchronisation), so it can be captured in a CUDA graph. */
int supa_simulate(supa_batch *b, const supa_primary *prim_dev, int64_t n, uint64_t seed,
                  uint64_t shower_id_base, void *stream);

/* supa_batch_create + supa_simulate in one call; *out must be destroyed with
 * supa_destroy_batch. */
int supa_simulate_batch(const supa_geometry *const *geoms, int32_t n_geoms, const supa_primary *prim_dev,
                        int64_t n, uint64_t seed, uint64_t shower_id_base, const supa_launch_config *cfg,
                        supa_batch **out, void *stream);

/* Autotuner of the persistent step kernel's launch shape (no counterpart in
 * the paper, which runs one particle at a time): times supa_simulate on the
 * first min(n, 131072) showers of prim_dev for candidate register budgets
 * (blocks_per_sm 2..4), warps per block, shared-memory stack depths and flush
 * thresholds (coordinate descent), and writes the fastest into *cfg, keeping
 * its other fields (max_hits is taken per shower of the full batch).
 * *best_ms (may be NULL) receives the sample's time.  Synchronous; allocates
 * temporary batches. */
int supa_autotune(const supa_geometry *const *geoms, int32_t n_geoms, const supa_primary *prim_dev, int64_t n,
                  uint64_t seed, supa_launch_config *cfg, double *best_ms, void *stream);

/* Wait for the batch's last simulation on `stream` and report totals and
 * result pointers.  Returns SUPA_ERR_OVERFLOW if the hit pool or a particle
 * stack overflowed (re-run with a smaller batch or a larger max_hits). */
int supa_batch_get_info(supa_batch *b, supa_batch_info *info, void *stream);

/* Load balance of the last simulation of a batch created with
 * record_warp_times = 1 (no counterpart in the paper; the scheduling of an
 * uneven batch): for each warp of the persistent step kernel the GPU's
 * global timer (ns) when it started and when it found the shower queue
 * empty, [n_warps][2] uint64 into host memory dst (capacity warps).  Writes
 * min(n_warps, capacity) pairs and n_warps to *n_warps.  SUPA_ERR_INVALID_ARG
 * without record_warp_times, SUPA_ERR_NOT_READY before a simulation.
 * Synchronous. */
int supa_batch_warp_times(supa_batch *b, uint64_t *dst, int64_t capacity, int64_t *n_warps);

/* Copy hits [first_hit, first_hit + max_hits) of the batch, in shower order
 * (the point cloud of Sec. 3: each hit is (x, y, z, E)), into dst, a device
 * buffer if dst_is_device else a host buffer.  *n_written receives the count
 * (fewer at the end of the batch).  Requires supa_batch_get_info first.
 * Asynchronous on `stream` in both cases: a host destination (best pinned)
 * is complete once the stream reaches this point; the hits pass through a
 * batch-owned device staging buffer (grown to the largest host fetch, by a
 * synchronising allocation) and one copy-engine transfer. */
int supa_fetch_hits(supa_batch *b, int64_t first_hit, int64_t max_hits, void *dst, int32_t dst_is_device,
                    int64_t *n_written, void *stream);

/* Same ranges as supa_fetch_hits, lineage ids (uint64) of the hits; needs
 * record_tags = 1 at batch creation.  On the hybrid path a surrogate hit
 * carries the lineage id of the diverted particle that emitted it with bit 63
 * set (stepped hits never have bit 63: lineage ids stay below 2^63). */
int supa_fetch_hit_tags(supa_batch *b, int64_t first_hit, int64_t max_hits, uint64_t *dst_dev,
                        int64_t *n_written, void *stream);

/* Downsample showers [shower_begin, shower_end) of the batch into images
 * (App. A.5: per layer, a rectangular region of nx x ny cells; each cell sums
 * the energy of the points inside it).  grid_dev is float32
 * [shower_end - shower_begin][max_layers][ny][nx]; out_of_roi_dev (may be
 * NULL) receives per shower the FP64 energy outside every region.  All
 * geometries of the batch must share nx, ny, wx, wy.  Every cell is written.
 * May be enqueued directly after supa_simulate on the same stream (no host
 * synchronisation, so both can be captured in one CUDA graph); if that
 * simulation fails, supa_batch_get_info reports it and the images are
 * unspecified. */
int supa_voxelize(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *grid_dev,
                  double *out_of_roi_dev, void *stream);

/* supa_voxelize and the point cloud of the same showers in one pass over
 * their hits (App. A.5 images and Sec. 3 point clouds): hit i of shower s,
 * in the order of supa_fetch_hits, goes to float4 slot
 * offsets[s] + i - hits_base of hits_dev (offsets as in
 * supa_batch_info.offsets_dev; hits_dev device memory, 16-byte aligned,
 * covering slots offsets[shower_begin] - hits_base up to
 * offsets[shower_end] - hits_base, caller-owned).  The same result as
 * supa_voxelize followed by supa_fetch_hits of those showers, with the hits
 * read once instead of twice.  Asynchronous; may follow supa_simulate on the
 * same stream directly. */
int supa_voxelize_fetch(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *grid_dev,
                        double *out_of_roi_dev, float *hits_dev, int64_t hits_base, void *stream);

/* Shower-shape profiles of showers [shower_begin, shower_end), added to the
 * caller's FP64 accumulators (Sec. 5.1 layer energies; lateral spread):
 * longi_dev[l] += layer energy / E0 per shower (max_layers entries);
 * lat_dev[b] += hit energy / E0 for hits at transverse distance r from the
 * incidence axis through the impact point, b = floor(r / r_max * nbins),
 * the last bin collecting r >= r_max (nbins entries, 1..4096).
 * Asynchronous. */
int supa_profiles(supa_batch *b, int64_t shower_begin, int64_t shower_end, int32_t nbins, float r_max,
                  double *longi_dev, double *lat_dev, void *stream);

/* First-hit offsets of every shower from per-shower hit counts, without
 * allocating anything (the paper has no counterpart; this serves callers
 * that may not call cudaMalloc, e.g. code running under a host framework
 * whose memory pool owns every allocation, or code on a path that must not
 * wait on the allocator).  offsets_dev[0] = 0, offsets_dev[s+1] =
 * offsets_dev[s] + counts_dev[s] for s < n (int64, n + 1 entries): the scan
 * supa_simulate runs after each simulation.  Its scratch is a fixed 32 KiB
 * array inside the library's device image, present on every GPU that loads
 * the library until the process exits; n may be at most 16,769,024
 * (larger n: SUPA_ERR_INVALID_ARG, nothing launched).  The first call on a
 * device looks up the array's device address, so make that first call
 * before capturing a stream into a graph; the address is kept per device
 * and context, and the first call in a new context (after cudaDeviceReset)
 * looks it up again, so that call too belongs before any capture.  Entries
 * of the array are written before they are read within each call, so what
 * an earlier call left there does not matter.  All calls share the one array:
 * calls that overlap on the GPU (different streams, or different threads
 * without ordering) race and give wrong offsets.  Asynchronous on stream. */
int supa_shower_offsets_noalloc(const uint32_t *counts_dev, int64_t n, int64_t *offsets_dev, void *stream);

/* Check of the failure path of the tensor-core pipelines (the paper has no
 * counterpart): every pipeline wait in this library gives up after a bounded
 * time, records SUPA_ERR_TIMEOUT and lets the kernel return, so that a stuck
 * pipeline leaves a usable context instead of a hung GPU.  This call runs
 * one such wait, bounded at limit_cycles SM cycles (1..2^40), on a barrier
 * that nothing completes, synchronises `stream` and returns what the wait
 * reported: SUPA_ERR_TIMEOUT when it gave up as it must, SUPA_OK if it
 * completed, SUPA_ERR_CUDA on a CUDA error. */
int supa_check_wait_expiry(int64_t limit_cycles, void *stream);

/* Per-layer grids and resolutions (App. A.5 "Downsampling"; the grid
 * experiments use a CaloGAN-like detector with 3 x 96, 12 x 12 and 12 x 6
 * cells per layer at resolutions "1x", "2x", "3x").  Layer l has nx x ny
 * cells of wx x wy (x fastest), over a region placed like the geometry's
 * uniform grid (roi_mode).  At factor f every cell is split f times in both
 * directions: cells of wx/f x wy/f (float32), nx f x ny f of them. */
typedef struct supa_layer_grid {
    int32_t nx, ny;
    float wx, wy;
} supa_layer_grid;

/* Cells per shower of supa_voxelize_layers' output for these grids and
 * factors (1 <= factor <= 16, at most 8 factors, one grid per layer), or
 * SUPA_ERR_INVALID_ARG. */
int64_t supa_layer_images_cells(const supa_layer_grid *grids, int32_t n_grids, const int32_t *factors,
                                int32_t n_factors);

/* Images of showers [shower_begin, shower_end) at every factor from one
 * pass over their hits: images_dev float32 [n][cells] (16-byte aligned),
 * per shower for each factor in the given order, for each layer, ny f rows
 * of nx f cells; cell (i, j) sums the energy of the points with
 * floor((x - lo) / (wx/f)) = i and floor((y - lo_y) / (wy/f)) = j, both in
 * float32.  out_of_roi_dev (nullable) float64 [n][n_factors]: energy of the
 * points outside their layer's region at that factor.  n_grids must cover
 * supa_batch_info.max_layers; a shower's images must fit in shared memory
 * (at most 51,200 cells).  Asynchronous. */
int supa_voxelize_layers(supa_batch *b, int64_t shower_begin, int64_t shower_end, const supa_layer_grid *grids,
                         int32_t n_grids, const int32_t *factors, int32_t n_factors, float *images_dev,
                         double *out_of_roi_dev, void *stream);

/* Shower shape variables (Sec. 5.1 "Shower Shape Variables", App. A.1
 * "More shower shape variables") of showers [shower_begin, shower_end) of
 * the last simulation, from its point clouds (stepped and surrogate hits)
 * and FP64 layer sums.  Lateral coordinates of a point: (eta, phi) = (x, y)
 * minus the incidence axis through the impact point at the point's depth,
 * r = sqrt(eta^2 + phi^2).  layer_feats_dev float32 [n][L][18] with
 * L = supa_batch_info.max_layers, per layer i (0-based):
 *   n_i, Ebar_i, f_i = Ebar_i / E_tot, means of eta, phi, r, E over the
 *   points, their standard deviations, the energy-weighted centroids of
 *   eta, phi, r, the energy-weighted widths of eta, phi, r, and
 *   E_ratio = (E[1] - E[2]) / (E[1] + E[2]) of the two largest point
 *   energies (E[2] = 0 for one point); all 0 for an empty layer;
 * shower_feats_dev float32 [n][5]: E_tot, depth d (deepest layer with
 * energy, -1 if none), l_d = sum_i i Ebar_i, s_d = l_d / E_tot,
 * sigma_sd = sqrt(sum_i i^2 Ebar_i / E_tot - s_d^2).  Asynchronous. */
int supa_shower_shapes(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *layer_feats_dev,
                       float *shower_feats_dev, void *stream);

/* Downsample caller-provided hits: hits_dev float4 (x,y,z,E), shower s owns
 * hits [offsets_dev[s], offsets_dev[s+1]); a hit's layer is
 * slice_to_layer[rint(z/dz)] of geometry g; roi_x0_dev/roi_y0_dev are the low
 * corners of each region, float32 [n_showers][n_layers].  grid_dev is float32
 * [n_showers][n_layers][ny][nx]. */
int supa_voxelize_hits(const supa_geometry *g, const float *hits_dev, const int64_t *offsets_dev,
                       int64_t n_showers, const float *roi_x0_dev, const float *roi_y0_dev, float *grid_dev,
                       double *out_of_roi_dev, void *stream);

/* ---- surrogate network -------------------------------------------------
 * The paper has no counterpart: the hybrid path replaces the sub-showers of
 * particles below a cutoff energy E_s by a small network that predicts their
 * per-layer deposits.  The network maps 6 features (log E, the direction
 * cosines u_x, u_y, u_z, the position of the start slice within its layer,
 * the number of layers left behind the start layer) through three hidden
 * layers of 256 with GELU (its tanh form, z (1 + tanh(sqrt(2 / pi) (z +
 * 0.044715 z^3))) / 2) to 90 outputs: log-link outputs o_j of the means
 * mu_j = exp(o_j - 4) and log-variances s_j of the deposit fractions of
 * layers start + j, j = 0..29, and the mean lateral distances rho_j of
 * those deposits from the particle's axis.  Targets: fractions y_j and
 * energy-weighted mean distances R_j ([.][60]).  Loss, mean over samples and
 * layers: (y_j - mu_j)^2 / (2 v_j) + ln(v_j) / 2 + y_j (rho_j - R_j)^2 / 2
 * with v_j = exp(s_j) + 10^-8.  Compute: BF16
 * tensor-core GEMMs (tcgen05, TMA) with FP32 accumulation, FP32 master
 * weights and Adam (beta1 0.9, beta2 0.999, eps 1e-8).
 * Parameters are exchanged as a packed float32 vector of
 * supa_surrogate_param_count() values: W1 [256][6], b1 [256], W2 [256][256],
 * b2, W3 [256][256], b3, W4 [90][256], b4 [90] (row-major). */
typedef struct supa_surrogate supa_surrogate;

int32_t supa_surrogate_param_count(void);
/* batch: minibatch rows (a multiple of 128); params_host: initial values. */
int supa_surrogate_create(int32_t batch, const float *params_host, supa_surrogate **out);
int supa_surrogate_destroy(supa_surrogate *s);
/* Current FP32 master parameters (synchronous). */
int supa_surrogate_get_params(supa_surrogate *s, float *params_host);
/* Loss and gradients of one minibatch without an update (synchronous):
 * x_dev float32 [batch][6] (4-byte aligned), y_dev float32 [batch][60]
 * (8-byte aligned); a misaligned pointer is SUPA_ERR_INVALID_ARG. */
int supa_surrogate_gradients(supa_surrogate *s, const float *x_dev, const float *y_dev, float *grads_host,
                             double *loss_host, void *stream);
/* One Adam step on one minibatch (asynchronous; x_dev, y_dev as for
 * supa_surrogate_gradients); adds the minibatch loss to *loss_acc_dev
 * (device FP64) when it is not NULL. */
int supa_surrogate_train_step(supa_surrogate *s, const float *x_dev, const float *y_dev, float lr,
                              double *loss_acc_dev, void *stream);
/* Iterate averaging (Polyak-Ruppert) of the training: mode
 * SUPA_AVERAGE_START resets the average and from the next Adam step on adds
 * every step's FP32 parameters to it with equal weight; SUPA_AVERAGE_STOP
 * stops adding; SUPA_AVERAGE_APPLY replaces the parameters (and the BF16
 * copies the kernels read) by the average of the steps added so far (no
 * change if none was).  The Adam moments are kept.  Asynchronous on `stream`;
 * SUPA_ERR_INVALID_ARG for another mode. */
#define SUPA_AVERAGE_STOP 0
#define SUPA_AVERAGE_START 1
#define SUPA_AVERAGE_APPLY 2
int supa_surrogate_average(supa_surrogate *s, int32_t mode, void *stream);
/* One epoch over a training set of n samples (x_dev [n][6], y_dev [n][60]):
 * floor(n / batch) Adam steps on minibatches gathered in the order of the
 * permutation i -> (a i + c) mod n that `seed` picks.  Asynchronous; adds
 * each minibatch loss to *loss_acc_dev when it is not NULL.  x_dev 4-byte and
 * y_dev 8-byte aligned, else SUPA_ERR_INVALID_ARG.  Before its first step the
 * epoch's targets are copied once into the order the training pass reads
 * them: a device buffer of 256 bytes per row of the full minibatches, kept
 * with the surrogate (grown, after a synchronisation of `stream`, when a
 * larger epoch needs it; SUPA_ERR_OOM if it cannot be had). */
int supa_surrogate_train_epoch(supa_surrogate *s, const float *x_dev, const float *y_dev, int64_t n, uint64_t seed,
                               float lr, double *loss_acc_dev, void *stream);
/* Inference: x_dev float32 [n][6] (8-byte aligned) -> out_dev float32
 * [n][ld_out], 0 <= n < 2^31, 90 <= ld_out < 2^31, in one launch of the
 * fused network kernel (asynchronous; a pipeline timeout shows in
 * supa_surrogate_check).  Columns 0..89 of each row hold the outputs.  A
 * pitch that is a multiple of 4 floats at a 16-byte aligned out_dev is
 * written with TMA stores, which is faster; columns 90..min(ld_out, 96)-1
 * then receive the network's padding outputs, which are zero.  Other pitches
 * take plain coalesced stores and leave columns 90.. untouched.  Rows n..
 * are never written. */
int supa_surrogate_forward(supa_surrogate *s, const float *x_dev, int64_t n, float *out_dev, int64_t ld_out,
                           void *stream);
/* Synchronise and report a tensor-core pipeline that gave up waiting
 * (SUPA_ERR_TIMEOUT) since the last check. */
int supa_surrogate_check(supa_surrogate *s);

/* Deposit rule of the hybrid path for layer start + j of a particle of
 * energy E, from the network's mu_j and s_j. */
/* The network's first 30 outputs o_j give the deposit-fraction means
 * through a log link, mu_j = exp(o_j - 4).  MEAN: d_j = E f_j, f_j = mu_j,
 * and 0 where mu_j < 10^-6.  SAMPLE: the MEAN total E T, T = sum_j f_j,
 * split over the layers with f_j > 0 by a Dirichlet draw whose means are the
 * MEAN shares m_j = f_j / T: d_j = E T G_j / sum_i G_i with independent
 * G_j ~ Gamma(c m_j), so every layer's expected deposit is its MEAN deposit
 * and the particle's total is the MEAN total.  The concentration c matches
 * the predicted variances: T^2 (1 - sum m_j^2) / (c + 1) = sum of
 * exp(s_j) + 10^-8 (the training loss's variance floor) over the layers with
 * f_j > 0, c >= 1; where c would exceed 10^4 the MEAN
 * deposits are taken; a layer whose drawn share T G_j / sum_i G_i is below
 * 10^-6 gets nothing (the others' sum normalises).  The gamma variates
 * follow
 * Marsaglia and Tsang (ACM TOMS 26(3), 2000) on Philox stream tag 3 (counter
 * (shower id, slice | 3 << 16 | (4 j + attempt) << 20, lineage), key =
 * seed), at most four attempts per layer (then the mean c m_j). */
#define SUPA_SURROGATE_SAMPLE 0
#define SUPA_SURROGATE_MEAN 1

/* Switch a batch to the hybrid path: from the next supa_simulate on, a
 * particle whose energy is below e_s when it reaches a slice of a readout
 * layer is not stepped; it joins a device queue (at most queue_capacity
 * particles, else SUPA_ERR_OVERFLOW), the network predicts its deposits in
 * the next 30 layers, deposits follow `mode` (SUPA_SURROGATE_*; normals from
 * Philox keyed by shower, slice and lineage) and, scaled down when they add
 * up to more than E, are added to the layer sums and emitted as one hit per
 * non-empty layer after the shower's stepped hits: at the layer's mid depth,
 * displaced from the particle's straight line by max(0, rho_j) q (cos phi,
 * sin phi), one (q, phi) per particle (Philox stream tag 2, same keys): phi
 * uniform, q from the measured lateral law of plain sub-showers (their hits'
 * distances from the axis over the mean distance, a 65-point quantile
 * table, mean 1).  The energy left over is reported as sur_leak.  s = NULL or e_s <= 0 returns the batch to the plain
 * path.  s must outlive the batch.  Synchronous (allocates). */
int supa_batch_set_surrogate(supa_batch *b, supa_surrogate *s, float e_s, int64_t queue_capacity, int32_t mode);

/* Training set of the network from a plain simulation of sub-showers (each
 * primary entering on its start slice, see supa_primary.geom): x_dev float32
 * [n][6] features of the start; y_dev float32 [n][60]: deposit fractions of
 * layers start + 0..29 (FP64 layer sums / E), then the energy-weighted mean
 * distance of each of those layers' hits from the sub-shower's axis (0 for
 * an empty layer).  Synchronous. */
int supa_build_training_set(supa_batch *b, float e_s, float *x_dev, float *y_dev, void *stream);

/* The particles the last hybrid simulation of b diverted to the network, as
 * sub-shower primaries: each enters on its slice of diversion (geom = the
 * shower's geometry index | slice << 16) with its energy, position and
 * direction -- the inputs a matched training set is simulated from.  Writes
 * min(n, capacity) primaries to out_dev and the queue length n to *n_out.
 * Like the surrogate itself this has no counterpart in the SUPA paper.
 * Synchronous. */
int supa_export_diverted(supa_batch *b, supa_primary *out_dev, int64_t capacity, int64_t *n_out, void *stream);

/* Everything the surrogate did for one diverted particle of the last hybrid
 * simulation: its key and state when it was set aside, the network's outputs
 * and its drawn deposits (no counterpart in the SUPA paper). */
typedef struct supa_diverted_record {
    uint32_t shower;  /* index of the shower in the batch                 */
    int32_t slice;    /* slice of diversion k                             */
    int32_t layer;    /* readout layer of slice k                         */
    float x, y;       /* position on slice k                              */
    float tx, ty;     /* slopes u_x / u_z, u_y / u_z                      */
    float E;          /* energy                                           */
    uint64_t lineage; /* lineage id                                       */
    float lmu[30];    /* network outputs for layers layer + j: log-link   */
                      /*   output o_j of the deposit-fraction mean        */
                      /*   mu_j = exp(o_j - 4),                           */
    float s[30];      /*   log-variances of the fractions and the mean    */
    float rho[30];    /*   lateral distances                              */
    float dep[30];    /* deposits of layers layer + j (0 past the back)    */
    uint32_t n_hits;  /* hits emitted (layers with a deposit > 0)         */
    uint32_t reserved;
} supa_diverted_record;

/* Writes the records of min(n, capacity) diverted particles of the last
 * hybrid simulation of b to out_dev (device memory, 528 bytes each, in queue
 * order, which is not defined) and the queue length n to *n_out; capacity 0
 * with out_dev NULL only reports n.  The deposit rule and the hit rule can be
 * checked particle by particle from these records.  SUPA_ERR_INVALID_ARG if
 * b is not in hybrid mode, SUPA_ERR_NOT_READY before its first simulation.
 * Synchronous. */
int supa_export_surrogate(supa_batch *b, supa_diverted_record *out_dev, int64_t capacity, int64_t *n_out,
                          void *stream);

#ifdef __cplusplus
}
#endif
#endif /* SUPA_H */
