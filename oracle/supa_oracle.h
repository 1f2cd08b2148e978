/*
 * supa_oracle.h -- plain FP64 CPU oracle for SUPA particle splitting.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load or call this code.  The
 * product library (paper_2202_05012_gb300) never includes, links or calls it,
 * and this file includes nothing from the product.
 *
 * What it computes: Algorithm 1 of the SUPA paper (Sec. 3, "Propagation
 * Model") applied to every particle of every shower, slice by slice, followed
 * by the per-layer grouping of Sec. 3 and the downsampling of App. A.5.  Every
 * reading of a silent or garbled passage is listed beside the code that takes
 * it and in the design notes.
 */
#ifndef SUPA_ORACLE_H
#define SUPA_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_THETA_FIXED = 0, ORA_THETA_UNIFORM = 1 };
enum { ORA_EPS_ZERO = 0, ORA_EPS_UNIFORM = 1 };
enum { ORA_SPLIT_MOMENTUM = 0, ORA_SPLIT_LITERAL = 1 };
enum { ORA_ROI_FIXED = 0, ORA_ROI_AXIS = 1 };

/* Model parameters of Algorithm 1 ("Parameters" block) plus the stated
 * extensions (dead slices, Sec. 4.2; energy cut; escape cut). */
typedef struct {
    int n_slices;               /* slices z_0 .. z_{n_slices-1}            */
    double dz;                  /* slice gap Delta z                       */
    const int *slice_to_layer;  /* layer configuration; -1 = dead slice    */
    int n_layers;
    const double *p_stop;       /* per-slice stopping probability          */
    const double *p_split;      /* per-slice splitting probability         */
    int theta_mode;             /* p_theta: FIXED -> theta_lo, UNIFORM     */
    double theta_lo, theta_hi;
    int eps_mode;               /* p_eps: ZERO, or U(-f*theta, +f*theta)   */
    double eps_frac;            /* f (Table 2 uses 1/4)                    */
    int split_mode;             /* MOMENTUM (default) or LITERAL reading   */
    double e_min;               /* energy cut (0 = none)                   */
    double uz_min;              /* escape cut on the z direction cosine    */
    double e_s;                 /* hybrid path: a particle below e_s on a  */
                                /* readout slice is set aside, not stepped */
                                /* (0 = plain path)                        */
    /* Lateral regions (Sec. 4.2: slices divided into regions with their own
     * meta-parameters).  n_regions <= 1: none.  Otherwise region i holds
     * the particles with region_radius[i-1] <= r < region_radius[i]
     * (r^2 = x^2 + y^2 at the slice, compared in float32), and its
     * p_stop / p_split (rows of [n_regions][n_slices]), theta range and
     * eps_frac replace the geometry's. */
    int n_regions;
    const double *region_radius;    /* [n_regions - 1], increasing        */
    const double *region_p_stop;    /* [n_regions][n_slices]              */
    const double *region_p_split;   /* [n_regions][n_slices]              */
    const double *region_theta_lo;  /* [n_regions]                        */
    const double *region_theta_hi;  /* [n_regions]                        */
    const double *region_eps_frac;  /* [n_regions]                        */
} ora_geom;

/* One primary: initial energy, impact position and incidence angles
 * (Sec. 3 initial particle; Sec. 4.2 conditioning), and the slice it enters
 * on (0 for a shower; a later slice starts a sub-shower there). */
typedef struct {
    double E, x0, y0, theta, phi;
    int start_slice;
} ora_primary;

typedef struct {
    /* hits, in shower order, each shower sorted by (slice, lineage) */
    int64_t n_hits;
    double *hx, *hy, *hz, *hE;
    int32_t *hslice;
    uint64_t *hlineage;
    /* per shower */
    int64_t n_showers;
    int64_t *hit_offset;        /* n_showers + 1 */
    int64_t *steps;             /* particle-slice visits */
    double *layer_sum;          /* n_showers * n_layers */
    double *dead, *leak, *escape;
    int64_t *n_splits;
    int32_t *max_depth;         /* splits on the deepest lineage */
    int status;                 /* 0 ok, <0 error */
    /* hybrid path: particles set aside, in shower order */
    int64_t n_div;
    int64_t *div_shower;
    int32_t *div_k, *div_layer;
    double *div_x, *div_y, *div_ux, *div_uy, *div_uz, *div_E;
    uint64_t *div_lin;
} ora_result;

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ctr[4], key[2] -> out[4]. */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);

/* Simulate showers [0, n) whose global ids are shower_id_base + i.
 * Returns 0 on success.  n_threads <= 1 runs serially. */
int ora_simulate(const ora_geom *g, const ora_primary *prim, int64_t n,
                 uint64_t seed, uint64_t shower_id_base, int n_threads,
                 ora_result *out);
void ora_free_result(ora_result *r);

/* Downsampling (App. A.5): sum hit energies into per-layer cells.
 * grid is [n_showers][n_layers][ny][nx] (x fastest), zeroed by the caller.
 * Hit j of shower s lies in hx/hy/hz[hit_offset[s] + j]; its layer is
 * slice_to_layer[round(z / dz)].  roi_x0/roi_y0 are the low corners of the
 * region of interest, [n_showers][n_layers].  The cell index is decided in
 * float32, the precision of the product's kernel. */
void ora_voxelize(const float *hx, const float *hy, const float *hz, const float *hE,
                  const int64_t *hit_offset, int64_t n_showers,
                  float dz, const int *slice_to_layer, int n_slices, int n_layers,
                  const float *roi_x0, const float *roi_y0,
                  int nx, int ny, float wx, float wy,
                  double *grid, double *out_of_roi);

#ifdef __cplusplus
}
#endif
#endif
