/*
 * supa_oracle.c -- plain FP64 CPU oracle for SUPA particle splitting.
 *
 * TEST INFRASTRUCTURE ONLY (see supa_oracle.h).  Written for clarity, not
 * speed: one explicit particle stack per shower, every step spelled out in
 * the order of Algorithm 1.  Compile with -ffp-contract=off so that the
 * float32 decisions below are plain IEEE operations on every host.
 *
 * Readings of the paper taken here (each is also listed in the design notes):
 *  R1  Algorithm 1 draws alpha ~ U(0,1) per particle and slice.  Here
 *      alpha = r0 * 2^-32 from one Philox4x32-10 block keyed by
 *      (seed; shower id, slice, lineage); r1..r3 give theta, eps, omega.
 *  R2  A split always produces exactly two daughters (Sec. 3); the garbled
 *      "N <- p(delta(n=2))" of Algorithm 1 is read that way.
 *  R3  Table 2's "alpha" column is Algorithm 1's deviation angle eps.
 *  R4  Split kinematics (Sec. 3 "momentum conservation", Algorithm 1 energy
 *      line): daughter 0 carries E(theta/2+eps)/theta and is deflected by
 *      theta/2-eps at azimuth omega; daughter 1 carries the remainder
 *      E - E_0 and is deflected by theta/2+eps at azimuth omega+pi, so the
 *      opening angle is theta and E_0*delta_0 = E_1*delta_1.  The LITERAL
 *      reading deflects both by theta/2+eps.
 *  R5  Directions are 3-D unit vectors.  A deflection by (delta, phi) uses
 *      the orthonormal frame of Duff et al., "Building an Orthonormal Basis,
 *      Revisited" (JCGT 2017), evaluated for u_z > 0.
 *  R6  A decision happens at slice k (z_k = k*dz).  Survivors of slice k move
 *      in a straight line to z_{k+1}; survivors of the last slice leak.
 *  R7  A survivor with u_z <= uz_min escapes (its energy is booked as
 *      escaped) instead of propagating.
 *  R8  Stops in a slice that belongs to no layer (dead material, Sec. 4.2)
 *      deposit into a per-shower dead-energy counter and emit no hit.
 *  R9  The energy cut E < e_min forces a stop (an extension that makes
 *      multiplicity grow with the primary energy).  This comparison and the
 *      escape comparison are taken on the float32-rounded values, the
 *      precision in which the product's kernel takes them.
 *  R10 Lineage ids form a binary heap: the primary is 1, the daughters of l
 *      are 2l and 2l+1, a passing particle keeps its id.
 */
#include "supa_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- Philox4x32-10 (published constants of the Philox4x32 family) ------ */
#define PHILOX_M0 0xD2511F53u
#define PHILOX_M1 0xCD9E8D57u
#define PHILOX_W0 0x9E3779B9u
#define PHILOX_W1 0xBB67AE85u

void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)PHILOX_M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)PHILOX_M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += PHILOX_W0;
        k1 += PHILOX_W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* 24-bit uniform in [0,1): the top 24 bits of a 32-bit word (R1). */
static double unif24(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

/* ---- growable per-shower buffers --------------------------------------- */
typedef struct {
    double x, y, z, E;
    int32_t slice;
    uint64_t lineage;
} hit_t;

typedef struct {
    double x, y, ux, uy, uz, E;
    int32_t slice;
    int32_t depth;
    uint64_t lineage;
} particle_t;

typedef struct {
    hit_t *hits; int64_t n_hits, cap_hits;
    particle_t *stack; int64_t n_stack, cap_stack;
    particle_t *div; int64_t n_div, cap_div;  /* hybrid path: set aside */
} work_t;

static int push_div(work_t *w, particle_t q) {
    if (w->n_div == w->cap_div) {
        int64_t nc = w->cap_div ? 2 * w->cap_div : 64;
        particle_t *p = (particle_t *)realloc(w->div, (size_t)nc * sizeof(particle_t));
        if (!p) return -1;
        w->div = p; w->cap_div = nc;
    }
    w->div[w->n_div++] = q;
    return 0;
}

static int push_hit(work_t *w, hit_t h) {
    if (w->n_hits == w->cap_hits) {
        int64_t nc = w->cap_hits ? 2 * w->cap_hits : 256;
        hit_t *p = (hit_t *)realloc(w->hits, (size_t)nc * sizeof(hit_t));
        if (!p) return -1;
        w->hits = p; w->cap_hits = nc;
    }
    w->hits[w->n_hits++] = h;
    return 0;
}

static int push_particle(work_t *w, particle_t q) {
    if (w->n_stack == w->cap_stack) {
        int64_t nc = w->cap_stack ? 2 * w->cap_stack : 256;
        particle_t *p = (particle_t *)realloc(w->stack, (size_t)nc * sizeof(particle_t));
        if (!p) return -1;
        w->stack = p; w->cap_stack = nc;
    }
    w->stack[w->n_stack++] = q;
    return 0;
}

static int cmp_hit(const void *a, const void *b) {
    const hit_t *p = (const hit_t *)a, *q = (const hit_t *)b;
    if (p->slice != q->slice) return p->slice < q->slice ? -1 : 1;
    if (p->lineage != q->lineage) return p->lineage < q->lineage ? -1 : 1;
    return 0;
}

/* Deflect unit vector u by polar angle delta at azimuth phi (R5). */
static void deflect(const double u[3], double delta, double phi, double out[3]) {
    double a = -1.0 / (1.0 + u[2]);
    double b = u[0] * u[1] * a;
    double e1[3] = {1.0 + u[0] * u[0] * a, b, -u[0]};
    double e2[3] = {b, 1.0 + u[1] * u[1] * a, -u[1]};
    double cd = cos(delta), sd = sin(delta), cp = cos(phi), sp = sin(phi);
    for (int i = 0; i < 3; ++i)
        out[i] = cd * u[i] + sd * (cp * e1[i] + sp * e2[i]);
}

typedef struct {
    int64_t steps, n_splits;
    int32_t max_depth;
    double dead, leak, escape;
    double *layer_sum;  /* n_layers */
} shower_acc_t;

/* Book a survivor of slice k (R6, R7): leak, escape, or move to slice k+1. */
static int survive(const ora_geom *g, work_t *w, particle_t q, shower_acc_t *acc) {
    if (q.slice == g->n_slices - 1) { acc->leak += q.E; return 0; }
    if ((float)q.uz <= (float)g->uz_min) { acc->escape += q.E; return 0; }
    q.x += g->dz * q.ux / q.uz;
    q.y += g->dz * q.uy / q.uz;
    q.slice += 1;
    return push_particle(w, q);
}

/* One shower: Algorithm 1 applied to every particle at every slice. */
static int simulate_one(const ora_geom *g, const ora_primary *p, uint64_t seed,
                        uint64_t shower_id, work_t *w, shower_acc_t *acc) {
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    w->n_hits = 0; w->n_stack = 0; w->n_div = 0;
    memset(acc->layer_sum, 0, sizeof(double) * (size_t)g->n_layers);
    acc->steps = 0; acc->n_splits = 0; acc->max_depth = 0;
    acc->dead = acc->leak = acc->escape = 0.0;

    /* Initial particle (Sec. 3): at the impact point on z_0 with the
     * incidence direction (Sec. 4.2 conditioning). */
    particle_t q0;
    q0.x = p->x0; q0.y = p->y0;
    q0.ux = sin(p->theta) * cos(p->phi);
    q0.uy = sin(p->theta) * sin(p->phi);
    q0.uz = cos(p->theta);
    q0.E = p->E; q0.slice = p->start_slice; q0.depth = 0; q0.lineage = 1;
    if (q0.slice < 0 || q0.slice >= g->n_slices) return -1;
    if (push_particle(w, q0)) return -1;

    while (w->n_stack > 0) {
        particle_t q = w->stack[--w->n_stack];
        const int k = q.slice;
        /* Hybrid path: below e_s on a readout slice the particle is set
         * aside for the surrogate instead of being stepped (float32
         * comparison, the kernel's precision). */
        if (g->e_s > 0.0 && (float)q.E < (float)g->e_s && g->slice_to_layer[k] >= 0) {
            if (push_div(w, q)) return -1;
            continue;
        }
        acc->steps += 1;

        /* The particle's lateral region at this slice (R26) selects the
         * meta-parameters: r^2 = x^2 + y^2 against the squared radii, both in
         * float32 (the kernel's precision). */
        const double *p_stop = g->p_stop, *p_split = g->p_split;
        double theta_lo = g->theta_lo, theta_hi = g->theta_hi, eps_frac = g->eps_frac;
        if (g->n_regions > 1) {
            const float xf = (float)q.x, yf = (float)q.y;
            const float r2 = fmaf(xf, xf, yf * yf);
            int reg = 0;
            while (reg < g->n_regions - 1) {
                const float b = (float)g->region_radius[reg];
                if (r2 < b * b) break;
                ++reg;
            }
            p_stop = g->region_p_stop + (size_t)reg * (size_t)g->n_slices;
            p_split = g->region_p_split + (size_t)reg * (size_t)g->n_slices;
            theta_lo = g->region_theta_lo[reg];
            theta_hi = g->region_theta_hi[reg];
            eps_frac = g->region_eps_frac[reg];
        }

        /* Algorithm 1: draw theta, eps, alpha (and omega) for (shower, slice, lineage). */
        const uint32_t ctr[4] = {(uint32_t)shower_id, (uint32_t)k,
                                 (uint32_t)q.lineage, (uint32_t)(q.lineage >> 32)};
        uint32_t r[4];
        ora_philox4x32_10(ctr, key, r);
        const double alpha = (double)r[0] * (1.0 / 4294967296.0);
        double theta = theta_lo;
        if (g->theta_mode == ORA_THETA_UNIFORM)
            theta = theta_lo + (theta_hi - theta_lo) * unif24(r[1]);
        double eps = 0.0;
        if (g->eps_mode == ORA_EPS_UNIFORM)
            eps = -eps_frac * theta + 2.0 * eps_frac * theta * unif24(r[2]);

        const int stop = (alpha < p_stop[k]) || ((float)q.E < (float)g->e_min);
        if (stop) {
            /* "Active <- False": the particle deposits its energy at slice k. */
            const int layer = g->slice_to_layer[k];
            if (layer < 0) {
                acc->dead += q.E;
            } else {
                hit_t h = {q.x, q.y, (double)k * g->dz, q.E, k, q.lineage};
                if (push_hit(w, h)) return -1;
                acc->layer_sum[layer] += q.E;
            }
        } else if (alpha < p_stop[k] + p_split[k]) {
            /* Split into two daughters (R2, R4). */
            const double omega = 2.0 * M_PI * unif24(r[3]);
            const double E0 = q.E * (theta / 2.0 + eps) / theta;
            const double E1 = q.E - E0;
            double d0, d1;
            if (g->split_mode == ORA_SPLIT_LITERAL) {
                d0 = theta / 2.0 + eps; d1 = theta / 2.0 + eps;
            } else {
                d0 = theta / 2.0 - eps; d1 = theta / 2.0 + eps;
            }
            const double u[3] = {q.ux, q.uy, q.uz};
            double v0[3], v1[3];
            deflect(u, d0, omega, v0);
            deflect(u, d1, omega + M_PI, v1);
            acc->n_splits += 1;
            particle_t a = q, b = q;
            a.ux = v0[0]; a.uy = v0[1]; a.uz = v0[2]; a.E = E0;
            b.ux = v1[0]; b.uy = v1[1]; b.uz = v1[2]; b.E = E1;
            a.lineage = 2 * q.lineage; b.lineage = 2 * q.lineage + 1;
            a.depth = b.depth = q.depth + 1;
            if (a.depth > acc->max_depth) acc->max_depth = a.depth;
            if (survive(g, w, b, acc)) return -1;
            if (survive(g, w, a, acc)) return -1;
        } else {
            /* Pass through with the same velocity. */
            if (survive(g, w, q, acc)) return -1;
        }
    }
    qsort(w->hits, (size_t)w->n_hits, sizeof(hit_t), cmp_hit);
    return 0;
}

void ora_free_result(ora_result *r) {
    free(r->hx); free(r->hy); free(r->hz); free(r->hE);
    free(r->hslice); free(r->hlineage);
    free(r->hit_offset); free(r->steps); free(r->layer_sum);
    free(r->dead); free(r->leak); free(r->escape);
    free(r->n_splits); free(r->max_depth);
    free(r->div_shower); free(r->div_k); free(r->div_layer); free(r->div_x); free(r->div_y);
    free(r->div_ux); free(r->div_uy); free(r->div_uz); free(r->div_E); free(r->div_lin);
    memset(r, 0, sizeof(*r));
}

int ora_simulate(const ora_geom *g, const ora_primary *prim, int64_t n,
                 uint64_t seed, uint64_t shower_id_base, int n_threads,
                 ora_result *out) {
    memset(out, 0, sizeof(*out));
    out->n_showers = n;
    const int L = g->n_layers;
    out->hit_offset = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    out->steps = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    out->layer_sum = (double *)calloc((size_t)(n * L) + 1, sizeof(double));
    out->dead = (double *)calloc((size_t)n + 1, sizeof(double));
    out->leak = (double *)calloc((size_t)n + 1, sizeof(double));
    out->escape = (double *)calloc((size_t)n + 1, sizeof(double));
    out->n_splits = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    out->max_depth = (int32_t *)calloc((size_t)n + 1, sizeof(int32_t));
    hit_t **per_shower = (hit_t **)calloc((size_t)n + 1, sizeof(hit_t *));
    particle_t **per_div = (particle_t **)calloc((size_t)n + 1, sizeof(particle_t *));
    int64_t *div_count = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
    if (!out->hit_offset || !out->steps || !out->layer_sum || !out->dead || !out->leak ||
        !out->escape || !out->n_splits || !out->max_depth || !per_shower || !per_div || !div_count) {
        free(per_shower); free(per_div); free(div_count); ora_free_result(out); return -1;
    }
    int failed = 0;
    if (n_threads < 1) n_threads = 1;
#ifdef _OPENMP
#pragma omp parallel num_threads(n_threads) reduction(|| : failed)
#endif
    {
        work_t w = {0};
        shower_acc_t acc;
        acc.layer_sum = (double *)calloc((size_t)L + 1, sizeof(double));
        if (!acc.layer_sum) failed = 1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t s = 0; s < n; ++s) {
            if (failed) continue;
            if (simulate_one(g, &prim[s], seed, shower_id_base + (uint64_t)s, &w, &acc)) { failed = 1; continue; }
            out->steps[s] = acc.steps;
            out->n_splits[s] = acc.n_splits;
            out->max_depth[s] = acc.max_depth;
            out->dead[s] = acc.dead; out->leak[s] = acc.leak; out->escape[s] = acc.escape;
            memcpy(out->layer_sum + s * L, acc.layer_sum, sizeof(double) * (size_t)L);
            out->hit_offset[s + 1] = w.n_hits;  /* count for now */
            per_shower[s] = (hit_t *)malloc(sizeof(hit_t) * (size_t)(w.n_hits + 1));
            if (!per_shower[s]) { failed = 1; continue; }
            memcpy(per_shower[s], w.hits, sizeof(hit_t) * (size_t)w.n_hits);
            div_count[s] = w.n_div;
            if (w.n_div) {
                per_div[s] = (particle_t *)malloc(sizeof(particle_t) * (size_t)w.n_div);
                if (!per_div[s]) { failed = 1; continue; }
                memcpy(per_div[s], w.div, sizeof(particle_t) * (size_t)w.n_div);
            }
        }
        free(acc.layer_sum); free(w.hits); free(w.stack); free(w.div);
    }
    if (!failed) {
        int64_t nd = 0;
        for (int64_t s = 0; s < n; ++s) nd += div_count[s];
        out->n_div = nd;
        out->div_shower = (int64_t *)malloc(sizeof(int64_t) * (size_t)(nd + 1));
        out->div_k = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nd + 1));
        out->div_layer = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nd + 1));
        out->div_x = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_y = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_ux = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_uy = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_uz = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_E = (double *)malloc(sizeof(double) * (size_t)(nd + 1));
        out->div_lin = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nd + 1));
        if (!out->div_shower || !out->div_k || !out->div_layer || !out->div_x || !out->div_y || !out->div_ux ||
            !out->div_uy || !out->div_uz || !out->div_E || !out->div_lin) failed = 1;
        int64_t j = 0;
        for (int64_t s = 0; s < n && !failed; ++s) {
            for (int64_t i = 0; i < div_count[s]; ++i, ++j) {
                const particle_t *q = &per_div[s][i];
                out->div_shower[j] = s; out->div_k[j] = q->slice;
                out->div_layer[j] = g->slice_to_layer[q->slice];
                out->div_x[j] = q->x; out->div_y[j] = q->y;
                out->div_ux[j] = q->ux; out->div_uy[j] = q->uy; out->div_uz[j] = q->uz;
                out->div_E[j] = q->E; out->div_lin[j] = q->lineage;
            }
        }
    }
    for (int64_t s = 0; s < n; ++s) free(per_div[s]);
    free(per_div); free(div_count);
    if (!failed) {
        for (int64_t s = 0; s < n; ++s) out->hit_offset[s + 1] += out->hit_offset[s];
        const int64_t nh = out->hit_offset[n];
        out->n_hits = nh;
        out->hx = (double *)malloc(sizeof(double) * (size_t)(nh + 1));
        out->hy = (double *)malloc(sizeof(double) * (size_t)(nh + 1));
        out->hz = (double *)malloc(sizeof(double) * (size_t)(nh + 1));
        out->hE = (double *)malloc(sizeof(double) * (size_t)(nh + 1));
        out->hslice = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nh + 1));
        out->hlineage = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(nh + 1));
        if (!out->hx || !out->hy || !out->hz || !out->hE || !out->hslice || !out->hlineage) failed = 1;
        for (int64_t s = 0; s < n && !failed; ++s) {
            for (int64_t j = out->hit_offset[s]; j < out->hit_offset[s + 1]; ++j) {
                const hit_t *h = &per_shower[s][j - out->hit_offset[s]];
                out->hx[j] = h->x; out->hy[j] = h->y; out->hz[j] = h->z; out->hE[j] = h->E;
                out->hslice[j] = h->slice; out->hlineage[j] = h->lineage;
            }
        }
    }
    for (int64_t s = 0; s < n; ++s) free(per_shower[s]);
    free(per_shower);
    if (failed) { ora_free_result(out); out->status = -1; return -1; }
    return 0;
}

void ora_voxelize(const float *hx, const float *hy, const float *hz, const float *hE,
                  const int64_t *hit_offset, int64_t n_showers,
                  float dz, const int *slice_to_layer, int n_slices, int n_layers,
                  const float *roi_x0, const float *roi_y0,
                  int nx, int ny, float wx, float wy,
                  double *grid, double *out_of_roi) {
    for (int64_t s = 0; s < n_showers; ++s) {
        out_of_roi[s] = 0.0;
        for (int64_t j = hit_offset[s]; j < hit_offset[s + 1]; ++j) {
            /* The hit's slice from its depth, then its layer (Sec. 3 layer
             * configuration). */
            const int k = (int)rintf(hz[j] / dz);
            const int layer = (k >= 0 && k < n_slices) ? slice_to_layer[k] : -1;
            if (layer < 0) { out_of_roi[s] += (double)hE[j]; continue; }
            /* Cell of the region of interest: half-open [lo + i*w, lo + (i+1)*w). */
            const float fx = floorf((hx[j] - roi_x0[s * n_layers + layer]) / wx);
            const float fy = floorf((hy[j] - roi_y0[s * n_layers + layer]) / wy);
            if (fx >= 0.0f && fx < (float)nx && fy >= 0.0f && fy < (float)ny) {
                const int64_t cell = ((s * n_layers + layer) * (int64_t)ny + (int64_t)fy) * nx + (int64_t)fx;
                grid[cell] += (double)hE[j];
            } else {
                out_of_roi[s] += (double)hE[j];
            }
        }
    }
}
