// api.cu -- host implementation of the C ABI declared in include/supa.h.
//
// Owns geometry tables and batch buffers, validates arguments, sizes the
// persistent launch, and maps device-side error words to status codes.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "supa_internal.cuh"

using namespace supa;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(SUPA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define SUPA_CUDA(call)                                              \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);          \
    } while (0)

template <typename T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

// Threshold for "alpha < p" with alpha = r0 * 2^-32 and r0 a 32-bit word:
// r0 < p*2^32 <=> r0 < ceil(p*2^32) (the scaling by 2^32 is exact).
unsigned long long threshold(double p) {
    const double v = std::ceil(p * 4294967296.0);
    if (v <= 0.0) return 0ull;
    if (v >= 4294967296.0) return 4294967296ull;
    return (unsigned long long)v;
}

}  // namespace

namespace supa {
int set_last_error(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace supa

struct supa_geometry {
    GeomDev rec;  // slice_off = layer_off = 0
    std::vector<unsigned long long> t_stop, t_ss;  // [regions][n_slices]
    std::vector<RegionDev> regions;                // empty without lateral regions
    std::vector<int8_t> s2l;
    std::vector<float> zmid;
    std::vector<LayerInfo> linfo;
    int device = 0;
    GeomDev *d_rec = nullptr;
    unsigned long long *d_tstop = nullptr, *d_tss = nullptr;
    int8_t *d_s2l = nullptr;
    float *d_zmid = nullptr;
};

struct supa_batch {
    int device = 0;
    std::vector<const supa_geometry *> geoms;
    int64_t max_showers = 0;
    int max_layers = 1;
    bool tags = false, lpt = false;
    bool regions = false;  // some geometry has lateral regions
    // tables
    GeomDev *d_geoms = nullptr;
    unsigned long long *d_tstop = nullptr, *d_tss = nullptr;
    RegionDev *d_regions = nullptr;
    int8_t *d_s2l = nullptr;
    float *d_zmid = nullptr;
    LayerInfo *d_linfo = nullptr;
    // hybrid path
    supa_surrogate *sur = nullptr;
    float e_s = 0.0f;
    int sq_cap = 0;
    int sur_mode = SUPA_SURROGATE_SAMPLE;
    SurInfer inf;
    SurRec *d_sq_rec = nullptr;
    float *d_sq_feat = nullptr, *d_dep = nullptr;
    uint8_t *d_pcnt = nullptr;
    unsigned *d_sq_count = nullptr;
    uint32_t *d_scount = nullptr, *d_scursor = nullptr, *d_tot = nullptr;
    int64_t *d_soff = nullptr;
    float4 *d_sur_hits = nullptr;
    unsigned long long *d_sur_tags = nullptr;  // lineage tags of the surrogate hits (record_tags)
    double *d_sur_leak = nullptr;
    unsigned long long *d_scan_tmp2 = nullptr;
    int64_t n_diverted = 0;
    // inputs
    supa_primary *d_prim = nullptr;
    uint32_t *d_queue = nullptr, *d_bucket = nullptr;
    // hit pool
    float4 *d_pool = nullptr;
    unsigned long long *d_tags = nullptr;
    int *d_page_next = nullptr;
    int n_pages = 0;
    // per shower
    unsigned long long *d_hit_start = nullptr;
    uint32_t *d_hit_count = nullptr, *d_steps = nullptr;
    double *d_lsum = nullptr, *d_dead = nullptr, *d_leak = nullptr, *d_escape = nullptr;
    int64_t *d_offsets = nullptr;
    unsigned long long *d_scan_tmp = nullptr;
    // control: [0] queue head, [1] page counter, [2] error; totals [0] steps, [1] hits
    int *d_ctrl = nullptr;
    unsigned long long *d_totals = nullptr;
    SpillRec *d_spill = nullptr;
    unsigned long long *d_warp_times = nullptr;  // [warps][2] (record_warp_times)
    int spill_cap = 0;
    // launch shape
    int grid = 0, block = 0, stack_cap = 0, stage_cap = 0, flush_thr = 0, minb = 3, voxel_ctas = 0;
    size_t smem = 0;
    int warp_bytes = 0;
    // state
    int64_t last_n = -1;
    bool info_valid = false;
    int64_t n_hits = 0, n_steps = 0;
    float4 *d_stage = nullptr;
    int64_t stage_cap_hits = 0;
};

extern "C" {

const char *supa_last_error(void) { return g_last_error.c_str(); }

int supa_init_geometry(const supa_geometry_desc *d, supa_geometry **out) {
    if (!d || !out) return fail(SUPA_ERR_INVALID_ARG, "supa_init_geometry: null argument");
    *out = nullptr;
    if (d->n_slices < 1 || d->n_slices > SUPA_MAX_SLICES)
        return fail(SUPA_ERR_INVALID_ARG, "n_slices must be in [1, %d], got %d", SUPA_MAX_SLICES, d->n_slices);
    if (d->n_layers < 1 || d->n_layers > SUPA_MAX_LAYERS)
        return fail(SUPA_ERR_INVALID_ARG, "n_layers must be in [1, %d], got %d", SUPA_MAX_LAYERS, d->n_layers);
    if (!d->slice_to_layer || !d->p_stop || !d->p_split)
        return fail(SUPA_ERR_INVALID_ARG, "slice_to_layer, p_stop and p_split are required");
    if (!(d->dz > 0.0f) || !std::isfinite(d->dz)) return fail(SUPA_ERR_INVALID_ARG, "dz must be positive");
    if (d->theta_mode != SUPA_THETA_FIXED && d->theta_mode != SUPA_THETA_UNIFORM)
        return fail(SUPA_ERR_INVALID_ARG, "unknown theta_mode %d", d->theta_mode);
    if (d->eps_mode != SUPA_EPS_ZERO && d->eps_mode != SUPA_EPS_UNIFORM)
        return fail(SUPA_ERR_INVALID_ARG, "unknown eps_mode %d", d->eps_mode);
    if (d->split_mode != SUPA_SPLIT_MOMENTUM && d->split_mode != SUPA_SPLIT_LITERAL)
        return fail(SUPA_ERR_INVALID_ARG, "unknown split_mode %d", d->split_mode);
    if (d->roi_mode != SUPA_ROI_FIXED && d->roi_mode != SUPA_ROI_AXIS)
        return fail(SUPA_ERR_INVALID_ARG, "unknown roi_mode %d", d->roi_mode);
    const double th_hi = d->theta_mode == SUPA_THETA_FIXED ? d->theta_lo : d->theta_hi;
    if (!(d->theta_lo > 0.0) || !(th_hi >= d->theta_lo) || !(th_hi < M_PI / 2))
        return fail(SUPA_ERR_INVALID_ARG, "need 0 < theta_lo <= theta_hi < pi/2");
    const double ef = d->eps_mode == SUPA_EPS_UNIFORM ? d->eps_frac : 0.0;
    if (!(ef >= 0.0 && ef < 0.5)) return fail(SUPA_ERR_INVALID_ARG, "eps_frac must be in [0, 1/2)");
    if (!(d->e_min >= 0.0) || !std::isfinite(d->e_min)) return fail(SUPA_ERR_INVALID_ARG, "e_min must be >= 0");
    if (!(d->uz_min > 0.0 && d->uz_min < 1.0)) return fail(SUPA_ERR_INVALID_ARG, "uz_min must be in (0, 1)");
    if (d->nx < 1 || d->ny < 1 || (int64_t)d->nx * d->ny % 4 != 0 || (int64_t)d->nx * d->ny > (1 << 24))
        return fail(SUPA_ERR_INVALID_ARG, "nx*ny must be a positive multiple of 4 (got %d x %d)", d->nx, d->ny);
    if (!(d->wx > 0.0f) || !(d->wy > 0.0f)) return fail(SUPA_ERR_INVALID_ARG, "cell sizes must be positive");
    // Lineage ids are heap indices (primary 1, daughters 2l, 2l+1) held in
    // 64 bits: at most 62 splits on one path.  Without an energy cut a path
    // splits at most once per slice.
    if (d->n_slices > 62 && !(d->e_min > 0.0))
        return fail(SUPA_ERR_INVALID_ARG, "more than 62 slices needs e_min > 0 to bound the lineage depth");
    const int n_reg = d->n_regions > 1 ? d->n_regions : 1;
    double ef_max = ef;
    if (n_reg > 1) {
        if (n_reg > SUPA_MAX_REGIONS)
            return fail(SUPA_ERR_INVALID_ARG, "n_regions must be <= %d, got %d", SUPA_MAX_REGIONS, n_reg);
        if (!d->region_radius || !d->region_p_stop || !d->region_p_split || !d->region_theta_lo ||
            !d->region_theta_hi || !d->region_eps_frac)
            return fail(SUPA_ERR_INVALID_ARG, "lateral regions need every region_* array");
        for (int i = 0; i < n_reg - 1; ++i)
            if (!(d->region_radius[i] > (i ? d->region_radius[i - 1] : 0.0)) || !std::isfinite(d->region_radius[i]))
                return fail(SUPA_ERR_INVALID_ARG, "region radii must be positive, finite and increasing");
        for (int i = 0; i < n_reg; ++i) {
            const double lo = d->region_theta_lo[i];
            const double hi = d->theta_mode == SUPA_THETA_FIXED ? lo : d->region_theta_hi[i];
            if (!(lo > 0.0) || !(hi >= lo) || !(hi < M_PI / 2))
                return fail(SUPA_ERR_INVALID_ARG, "region %d: need 0 < theta_lo <= theta_hi < pi/2", i);
            const double f = d->eps_mode == SUPA_EPS_UNIFORM ? d->region_eps_frac[i] : 0.0;
            if (!(f >= 0.0 && f < 0.5)) return fail(SUPA_ERR_INVALID_ARG, "region %d: eps_frac must be in [0, 1/2)", i);
            ef_max = std::max(ef_max, f);
        }
    }

    supa_geometry *g = new supa_geometry();
    const int n = d->n_slices;
    g->t_stop.resize((size_t)n * n_reg);
    g->t_ss.resize((size_t)n * n_reg);
    g->s2l.resize(n);
    std::vector<int> kmin(d->n_layers, 1 << 30), kmax(d->n_layers, -1);
    for (int k = 0; k < n; ++k) {
        const double ps = d->p_stop[k], pp = d->p_split[k];
        if (!(ps >= 0.0 && ps <= 1.0 && pp >= 0.0 && pp <= 1.0) || ps + pp > 1.0 + 1e-12) {
            delete g;
            return fail(SUPA_ERR_INVALID_ARG, "slice %d: need p_stop, p_split in [0,1] and p_stop + p_split <= 1", k);
        }
        const int l = d->slice_to_layer[k];
        if (l < -1 || l >= d->n_layers) {
            delete g;
            return fail(SUPA_ERR_INVALID_ARG, "slice %d: layer %d out of range", k, l);
        }
        g->t_stop[k] = threshold(ps);
        g->t_ss[k] = threshold(ps + pp);
        for (int i = 0; n_reg > 1 && i < n_reg; ++i) {
            const double rs = d->region_p_stop[(size_t)i * n + k], rp = d->region_p_split[(size_t)i * n + k];
            if (!(rs >= 0.0 && rs <= 1.0 && rp >= 0.0 && rp <= 1.0) || rs + rp > 1.0 + 1e-12) {
                delete g;
                return fail(SUPA_ERR_INVALID_ARG, "region %d, slice %d: need p_stop, p_split in [0,1] and sum <= 1", i, k);
            }
            g->t_stop[(size_t)i * n + k] = threshold(rs);
            g->t_ss[(size_t)i * n + k] = threshold(rs + rp);
        }
        g->s2l[k] = (int8_t)l;
        if (l >= 0) {
            kmin[l] = std::min(kmin[l], k);
            kmax[l] = std::max(kmax[l], k);
        }
    }
    g->zmid.resize(d->n_layers);
    g->linfo.resize(d->n_layers);
    for (int l = 0; l < d->n_layers; ++l) {
        if (kmax[l] < 0) {
            delete g;
            return fail(SUPA_ERR_INVALID_ARG, "layer %d has no slice", l);
        }
        int cnt = 0;
        for (int k = 0; k < n; ++k) cnt += d->slice_to_layer[k] == l;
        g->linfo[l].k_first = (int16_t)kmin[l];
        g->linfo[l].n_slices = (int16_t)cnt;
        // mid depth of the layer, float32 as the downsampling kernel uses it
        g->zmid[l] = (d->dz * (float)(kmin[l] + kmax[l])) * 0.5f;
    }
    GeomDev &r = g->rec;
    r.n_slices = n;
    r.n_layers = d->n_layers;
    r.slice_off = 0;
    r.layer_off = 0;
    r.dz = d->dz;
    r.e_min = (float)d->e_min;
    r.uz_min = (float)d->uz_min;
    r.theta_lo = (float)d->theta_lo;
    r.theta_span = d->theta_mode == SUPA_THETA_UNIFORM ? (float)(d->theta_hi - d->theta_lo) : 0.0f;
    r.eps_frac = (float)ef;
    r.split_literal = d->split_mode == SUPA_SPLIT_LITERAL;
    r.nx = d->nx;
    r.ny = d->ny;
    r.wx = d->wx;
    r.wy = d->wy;
    r.roi_axis = d->roi_mode == SUPA_ROI_AXIS;
    // Each split leaves a daughter at most q = 1/2 + eps_frac of its parent's
    // energy and only particles with E >= e_min split, so a primary below
    // e_min * q^-61 splits at most 62 times on any path.
    r.e0_max = d->n_slices <= 62 ? INFINITY : (float)std::min(3.0e38, d->e_min * std::pow(0.5 + ef_max, -61.0));
    r.thr_off = 0;
    r.n_regions = n_reg;
    r.region_off = 0;
    for (int i = 0; n_reg > 1 && i < n_reg; ++i) {
        const float b = i < n_reg - 1 ? (float)d->region_radius[i] : INFINITY;
        const double lo = d->region_theta_lo[i];
        const double span = d->theta_mode == SUPA_THETA_UNIFORM ? d->region_theta_hi[i] - lo : 0.0;
        const double f = d->eps_mode == SUPA_EPS_UNIFORM ? d->region_eps_frac[i] : 0.0;
        g->regions.push_back(make_float4(b * b, (float)lo, (float)span, (float)f));
    }

    cudaError_t e = cudaGetDevice(&g->device);
    if (e == cudaSuccess) e = dalloc(&g->d_rec, 1);
    if (e == cudaSuccess) e = dalloc(&g->d_tstop, g->t_stop.size());
    if (e == cudaSuccess) e = dalloc(&g->d_tss, g->t_ss.size());
    if (e == cudaSuccess) e = dalloc(&g->d_s2l, n);
    if (e == cudaSuccess) e = dalloc(&g->d_zmid, d->n_layers);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_rec, &g->rec, sizeof(GeomDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tstop, g->t_stop.data(), g->t_stop.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_tss, g->t_ss.data(), g->t_ss.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_s2l, g->s2l.data(), n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(g->d_zmid, g->zmid.data(), d->n_layers * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        supa_destroy_geometry(g);
        return cuda_fail(e, "supa_init_geometry");
    }
    *out = g;
    return SUPA_OK;
}

int supa_destroy_geometry(supa_geometry *g) {
    if (!g) return SUPA_OK;
    cudaFree(g->d_rec);
    cudaFree(g->d_tstop);
    cudaFree(g->d_tss);
    cudaFree(g->d_s2l);
    cudaFree(g->d_zmid);
    delete g;
    return SUPA_OK;
}

static void free_hybrid(supa_batch *b) {
    void *ptrs[] = {b->d_sq_rec, b->d_sq_feat, b->d_dep, b->d_pcnt, b->d_sq_count, b->d_scount, b->d_scursor, b->d_tot,
                    b->d_soff, b->d_sur_hits, b->d_sur_tags, b->d_sur_leak, b->d_scan_tmp2};
    for (void *p : ptrs) cudaFree(p);
    surrogate_infer_free(&b->inf);
    b->d_sq_rec = nullptr;
    b->d_sq_feat = b->d_dep = nullptr;
    b->d_pcnt = nullptr;
    b->d_sq_count = nullptr;
    b->d_scount = b->d_scursor = b->d_tot = nullptr;
    b->d_soff = nullptr;
    b->d_sur_hits = nullptr;
    b->d_sur_tags = nullptr;
    b->d_sur_leak = nullptr;
    b->d_scan_tmp2 = nullptr;
    b->sur = nullptr;
    b->e_s = 0.0f;
    b->sq_cap = 0;
}

int supa_destroy_batch(supa_batch *b) {
    if (!b) return SUPA_OK;
    free_hybrid(b);
    cudaFree(b->d_linfo);
    void *ptrs[] = {b->d_geoms, b->d_tstop, b->d_tss, b->d_regions, b->d_s2l, b->d_zmid, b->d_prim, b->d_queue,
                    b->d_bucket, b->d_pool, b->d_tags, b->d_page_next, b->d_hit_start, b->d_hit_count,
                    b->d_steps, b->d_lsum, b->d_dead, b->d_leak, b->d_escape, b->d_offsets, b->d_scan_tmp,
                    b->d_ctrl, b->d_totals, b->d_spill, b->d_stage, b->d_warp_times};
    for (void *p : ptrs) cudaFree(p);
    delete b;
    return SUPA_OK;
}

int supa_batch_create(const supa_geometry *const *geoms, int32_t n_geoms, int64_t max_showers,
                      const supa_launch_config *cfg_in, supa_batch **out) {
    if (!geoms || !out) return fail(SUPA_ERR_INVALID_ARG, "supa_batch_create: null argument");
    *out = nullptr;
    if (n_geoms < 1 || n_geoms > SUPA_MAX_GEOMS)
        return fail(SUPA_ERR_INVALID_ARG, "n_geoms must be in [1, %d]", SUPA_MAX_GEOMS);
    if (max_showers < 1 || max_showers > ((int64_t)1 << 32) - 1)
        return fail(SUPA_ERR_INVALID_ARG, "max_showers must be in [1, 2^32)");
    supa_launch_config cfg{};
    if (cfg_in) cfg = *cfg_in;
    for (int i = 0; i < n_geoms; ++i)
        if (!geoms[i]) return fail(SUPA_ERR_INVALID_ARG, "geometry %d is null", i);

    supa_batch *b = new supa_batch();
    cudaError_t e = cudaGetDevice(&b->device);
    if (e != cudaSuccess) {
        delete b;
        return cuda_fail(e, "cudaGetDevice");
    }
    b->geoms.assign(geoms, geoms + n_geoms);
    b->max_showers = max_showers;
    b->tags = cfg.record_tags != 0;
    b->lpt = cfg.lpt_order != 0;

    // concatenated geometry tables
    std::vector<GeomDev> recs;
    std::vector<unsigned long long> ts, tss;
    std::vector<RegionDev> regs;
    std::vector<int8_t> s2l;
    std::vector<float> zm;
    std::vector<LayerInfo> li;
    for (int i = 0; i < n_geoms; ++i) {
        GeomDev r = geoms[i]->rec;
        r.slice_off = (int)s2l.size();
        r.layer_off = (int)zm.size();
        r.thr_off = (int)ts.size();
        r.region_off = (int)regs.size();
        recs.push_back(r);
        regs.insert(regs.end(), geoms[i]->regions.begin(), geoms[i]->regions.end());
        ts.insert(ts.end(), geoms[i]->t_stop.begin(), geoms[i]->t_stop.end());
        tss.insert(tss.end(), geoms[i]->t_ss.begin(), geoms[i]->t_ss.end());
        s2l.insert(s2l.end(), geoms[i]->s2l.begin(), geoms[i]->s2l.end());
        zm.insert(zm.end(), geoms[i]->zmid.begin(), geoms[i]->zmid.end());
        li.insert(li.end(), geoms[i]->linfo.begin(), geoms[i]->linfo.end());
        b->max_layers = std::max(b->max_layers, r.n_layers);
    }
    b->regions = !regs.empty();

    // launch shape
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const int wpb = cfg.warps_per_block > 0 ? cfg.warps_per_block : 8;
    if (wpb > 8) {
        supa_destroy_batch(b);
        return fail(SUPA_ERR_INVALID_ARG, "warps_per_block must be <= 8");
    }
    // register budget: the 64-register build for 4 blocks per SM, else 80
    b->minb = cfg.blocks_per_sm >= 4 ? 4 : 3;
    b->voxel_ctas = std::max(0, cfg.voxel_ctas_per_sm);
    b->block = wpb * 32;
    b->stack_cap = cfg.stack_depth > 0 ? cfg.stack_depth : 128;
    if (b->stack_cap < 64 || b->stack_cap % 2) {
        supa_destroy_batch(b);
        return fail(SUPA_ERR_INVALID_ARG, "stack_depth must be an even number >= 64");
    }
    if (cfg.flush_threshold < -1 || cfg.flush_threshold > 1024) {
        supa_destroy_batch(b);
        return fail(SUPA_ERR_INVALID_ARG, "flush_threshold must be -1 (direct hit writes) or in [0, 1024]");
    }
    b->flush_thr = cfg.flush_threshold == 0 ? 128 : std::max(0, cfg.flush_threshold);
    b->stage_cap = b->flush_thr > 0 ? b->flush_thr + 32 : 0;
    b->warp_bytes = (int)warp_smem_bytes(b->stack_cap, b->stage_cap, b->tags);
    b->smem = (size_t)b->warp_bytes * wpb;
    int occ = 0;
    e = step_kernel_attributes(b->minb, b->regions, b->flush_thr > 0, b->block, b->smem, &occ);
    if (e != cudaSuccess || occ < 1) {
        supa_destroy_batch(b);
        if (e != cudaSuccess) return cuda_fail(e, "step kernel occupancy");
        return fail(SUPA_ERR_INVALID_ARG, "step kernel does not fit on an SM (%zu B shared memory)", b->smem);
    }
    const int bps = cfg.blocks_per_sm > 0 ? std::min(cfg.blocks_per_sm, occ) : occ;
    b->grid = bps * sms;
    const int64_t n_warps = (int64_t)b->grid * wpb;
    b->spill_cap = 2048;

    // hit pool
    int64_t max_hits = cfg.max_hits;
    if (max_hits <= 0) {
        size_t free_b = 0, total_b = 0;
        cudaMemGetInfo(&free_b, &total_b);
        const int64_t want = max_showers * 2048 + (4 << 20);
        const int64_t cap = (int64_t)(free_b * 0.4) / (b->tags ? 24 : 16);
        max_hits = std::min(want, cap);
    }
    b->n_pages = (int)((max_hits + kPageHits - 1) / kPageHits + n_warps + 1);

    const int64_t n = max_showers;
    if (e == cudaSuccess) e = dalloc(&b->d_geoms, n_geoms);
    if (e == cudaSuccess) e = dalloc(&b->d_tstop, ts.size());
    if (e == cudaSuccess) e = dalloc(&b->d_tss, tss.size());
    if (e == cudaSuccess) e = dalloc(&b->d_regions, std::max<size_t>(regs.size(), 1));
    if (e == cudaSuccess) e = dalloc(&b->d_s2l, s2l.size());
    if (e == cudaSuccess) e = dalloc(&b->d_zmid, zm.size());
    if (e == cudaSuccess) e = dalloc(&b->d_linfo, li.size());
    if (e == cudaSuccess) e = dalloc(&b->d_prim, n);
    if (e == cudaSuccess && b->lpt) e = dalloc(&b->d_queue, n);
    if (e == cudaSuccess && b->lpt) e = dalloc(&b->d_bucket, 256);
    if (e == cudaSuccess) e = dalloc(&b->d_pool, (size_t)b->n_pages * kPageHits);
    if (e == cudaSuccess && b->tags) e = dalloc(&b->d_tags, (size_t)b->n_pages * kPageHits);
    if (e == cudaSuccess) e = dalloc(&b->d_page_next, b->n_pages);
    if (e == cudaSuccess) e = dalloc(&b->d_hit_start, n);
    if (e == cudaSuccess) e = dalloc(&b->d_hit_count, n);
    if (e == cudaSuccess) e = dalloc(&b->d_steps, n);
    if (e == cudaSuccess) e = dalloc(&b->d_lsum, (size_t)n * b->max_layers);
    if (e == cudaSuccess) e = dalloc(&b->d_dead, n);
    if (e == cudaSuccess) e = dalloc(&b->d_leak, n);
    if (e == cudaSuccess) e = dalloc(&b->d_escape, n);
    if (e == cudaSuccess) e = dalloc(&b->d_offsets, n + 1);
    if (e == cudaSuccess) e = dalloc(&b->d_scan_tmp, scan_tmp_elems(n) + 1);
    if (e == cudaSuccess) e = dalloc(&b->d_ctrl, 4);
    if (e == cudaSuccess) e = dalloc(&b->d_totals, 2);
    if (e == cudaSuccess) e = dalloc(&b->d_spill, (size_t)n_warps * b->spill_cap);
    if (e == cudaSuccess && cfg.record_warp_times) e = dalloc(&b->d_warp_times, (size_t)n_warps * 2);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_geoms, recs.data(), recs.size() * sizeof(GeomDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tstop, ts.data(), ts.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_tss, tss.data(), tss.size() * 8, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !regs.empty())
        e = cudaMemcpy(b->d_regions, regs.data(), regs.size() * sizeof(RegionDev), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_s2l, s2l.data(), s2l.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_zmid, zm.data(), zm.size() * 4, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(b->d_linfo, li.data(), li.size() * sizeof(LayerInfo), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        supa_destroy_batch(b);
        if (e == cudaErrorMemoryAllocation) {
            cudaGetLastError();
            return fail(SUPA_ERR_OOM, "supa_batch_create: out of device memory (max_hits = %lld)", (long long)max_hits);
        }
        return cuda_fail(e, "supa_batch_create");
    }
    *out = b;
    return SUPA_OK;
}

static SurParams sur_params(const supa_batch *b, uint64_t seed, uint64_t shower_id_base);

int supa_simulate(supa_batch *b, const supa_primary *prim_dev, int64_t n, uint64_t seed, uint64_t shower_id_base,
                  void *stream) {
    if (!b || (!prim_dev && n > 0)) return fail(SUPA_ERR_INVALID_ARG, "supa_simulate: null argument");
    if (n < 0 || n > b->max_showers)
        return fail(SUPA_ERR_INVALID_ARG, "n = %lld exceeds the batch capacity %lld", (long long)n,
                    (long long)b->max_showers);
    if (shower_id_base + (uint64_t)n > (1ull << 32))
        return fail(SUPA_ERR_INVALID_ARG, "shower ids must stay below 2^32");
    cudaStream_t st = (cudaStream_t)stream;
    b->info_valid = false;
    b->last_n = n;
    if (n > 0) SUPA_CUDA(cudaMemcpyAsync(b->d_prim, prim_dev, n * sizeof(supa_primary), cudaMemcpyDeviceToDevice, st));
    SUPA_CUDA(cudaMemsetAsync(b->d_ctrl, 0, 4 * sizeof(int), st));
    SUPA_CUDA(cudaMemsetAsync(b->d_totals, 0, 2 * sizeof(unsigned long long), st));
    if (b->lpt && n > 0) SUPA_CUDA(launch_lpt_queue(b->d_prim, n, b->d_queue, b->d_bucket, st));
    StepParams p{};
    p.prim = b->d_prim;
    p.queue = b->lpt ? b->d_queue : nullptr;
    p.n = n;
    p.n_geoms = (int)b->geoms.size();
    p.seed = seed;
    p.shower_id_base = shower_id_base;
    p.geoms = b->d_geoms;
    p.t_stop = b->d_tstop;
    p.t_ss = b->d_tss;
    p.regions = b->d_regions;
    p.stage_cap = b->stage_cap;
    p.flush_thr = b->flush_thr;
    p.s2l = b->d_s2l;
    p.pool = b->d_pool;
    p.tag_pool = b->d_tags;
    p.page_next = b->d_page_next;
    p.n_pages = b->n_pages;
    p.page_counter = b->d_ctrl + 1;
    p.hit_start = b->d_hit_start;
    p.hit_count = b->d_hit_count;
    p.steps = b->d_steps;
    p.lsum = b->d_lsum;
    p.lsum_stride = b->max_layers;
    p.dead = b->d_dead;
    p.leak = b->d_leak;
    p.escape = b->d_escape;
    p.queue_head = b->d_ctrl;
    p.error = b->d_ctrl + 2;
    p.totals = b->d_totals;
    p.spill = b->d_spill;
    p.warp_times = b->d_warp_times;
    p.spill_cap = b->spill_cap;
    p.stack_cap = b->stack_cap;
    p.warp_smem_bytes = b->warp_bytes;
    const bool hybrid = b->sur != nullptr;
    if (hybrid) {
        p.e_s = b->e_s;
        p.linfo = b->d_linfo;
        p.sq_rec = b->d_sq_rec;
        p.sq_feat = b->d_sq_feat;
        p.sq_count = b->d_sq_count;
        p.sq_cap = b->sq_cap;
        SUPA_CUDA(cudaMemsetAsync(b->d_sq_count, 0, sizeof(unsigned), st));
        SUPA_CUDA(cudaMemsetAsync(b->d_scount, 0, (size_t)std::max<int64_t>(n, 1) * 4, st));
        SUPA_CUDA(cudaMemsetAsync(b->d_scursor, 0, (size_t)std::max<int64_t>(n, 1) * 4, st));
        SUPA_CUDA(cudaMemsetAsync(b->d_sur_leak, 0, (size_t)std::max<int64_t>(n, 1) * 8, st));
    }
    if (n > 0) SUPA_CUDA(launch_step(b->minb, b->regions, b->flush_thr > 0, p, b->grid, b->block, b->smem, st));
    if (!hybrid) {
        SUPA_CUDA(launch_scan_counts(b->d_hit_count, n, b->d_offsets, b->d_scan_tmp, st));
        return SUPA_OK;
    }
    // hybrid: network over the queue, deposits, surrogate hit segments
    SUPA_CUDA(surrogate_infer_run(b->sur, &b->inf, b->d_sq_feat, b->d_sq_count, st));
    const SurParams sp = sur_params(b, seed, shower_id_base);
    SUPA_CUDA(launch_sur_deposits(sp, st));
    SUPA_CUDA(launch_scan_counts(b->d_scount, n, b->d_soff, b->d_scan_tmp2, st));
    SUPA_CUDA(launch_sur_hits(sp, st));
    SUPA_CUDA(launch_add_counts(b->d_hit_count, b->d_scount, n, b->d_tot, st));
    SUPA_CUDA(launch_scan_counts(b->d_tot, n, b->d_offsets, b->d_scan_tmp, st));
    return SUPA_OK;
}

// Kernel arguments of the surrogate side of a hybrid batch.
static SurParams sur_params(const supa_batch *b, uint64_t seed, uint64_t shower_id_base) {
    SurParams sp{};
    sp.mode = b->sur_mode;
    sp.rec = b->d_sq_rec;
    sp.count = b->d_sq_count;
    sp.cap = b->sq_cap;
    sp.out = b->inf.OUT;
    sp.out_ld = b->inf.ld;
    sp.prim = b->d_prim;
    sp.geoms = b->d_geoms;
    sp.zmid = b->d_zmid;
    sp.seed = seed;
    sp.shower_id_base = shower_id_base;
    sp.dep = b->d_dep;
    sp.pcnt = b->d_pcnt;
    sp.lsum = b->d_lsum;
    sp.lsum_stride = b->max_layers;
    sp.sur_leak = b->d_sur_leak;
    sp.scount = b->d_scount;
    sp.soff = b->d_soff;
    sp.scursor = b->d_scursor;
    sp.hits = b->d_sur_hits;
    sp.tags = b->d_sur_tags;
    return sp;
}

int supa_batch_set_surrogate(supa_batch *b, supa_surrogate *s, float e_s, int64_t queue_capacity, int32_t mode) {
    if (!b) return fail(SUPA_ERR_INVALID_ARG, "supa_batch_set_surrogate: null batch");
    if (mode != SUPA_SURROGATE_SAMPLE && mode != SUPA_SURROGATE_MEAN)
        return fail(SUPA_ERR_INVALID_ARG, "unknown surrogate mode %d", mode);
    free_hybrid(b);
    b->last_n = -1;
    b->info_valid = false;
    if (!s || !(e_s > 0.0f)) return SUPA_OK;
    if (queue_capacity < 128 || queue_capacity > (int64_t)1 << 30)
        return fail(SUPA_ERR_INVALID_ARG, "queue_capacity must be in [128, 2^30]");
    const int cap = (int)((queue_capacity + 127) / 128 * 128);
    const int64_t n = b->max_showers;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dalloc(&b->d_sq_rec, cap);
    if (e == cudaSuccess) e = dalloc(&b->d_sq_feat, (size_t)cap * kSurIn);
    if (e == cudaSuccess) e = dalloc(&b->d_dep, (size_t)cap * kSurLayers);
    if (e == cudaSuccess) e = dalloc(&b->d_pcnt, (size_t)cap);
    if (e == cudaSuccess) e = dalloc(&b->d_sq_count, 1);
    if (e == cudaSuccess) e = dalloc(&b->d_scount, n);
    if (e == cudaSuccess) e = dalloc(&b->d_scursor, n);
    if (e == cudaSuccess) e = dalloc(&b->d_tot, n);
    if (e == cudaSuccess) e = dalloc(&b->d_soff, n + 1);
    if (e == cudaSuccess) e = dalloc(&b->d_sur_hits, (size_t)cap * kSurLayers);
    if (e == cudaSuccess && b->tags) e = dalloc(&b->d_sur_tags, (size_t)cap * kSurLayers);
    if (e == cudaSuccess) e = dalloc(&b->d_sur_leak, n);
    if (e == cudaSuccess) e = dalloc(&b->d_scan_tmp2, scan_tmp_elems(n) + 1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_hybrid(b);
        return fail(SUPA_ERR_OOM, "supa_batch_set_surrogate: out of device memory");
    }
    const int rc = surrogate_infer_init(s, cap, &b->inf);
    if (rc != SUPA_OK) {
        free_hybrid(b);
        return rc;
    }
    b->sur = s;
    b->e_s = e_s;
    b->sur_mode = mode;
    b->sq_cap = cap;
    return SUPA_OK;
}

int supa_build_training_set(supa_batch *b, float e_s, float *x_dev, float *y_dev, void *stream) {
    if (!b || !x_dev || !y_dev || !(e_s > 0.0f))
        return fail(SUPA_ERR_INVALID_ARG, "supa_build_training_set: bad argument");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    if (b->sur) return fail(SUPA_ERR_INVALID_ARG, "training sets come from plain (not hybrid) simulations");
    cudaStream_t st = (cudaStream_t)stream;
    int *bad = b->d_ctrl + 3;
    SUPA_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
    SUPA_CUDA(launch_training_set(b->d_prim, b->last_n, b->d_geoms, b->d_s2l, b->d_linfo, b->d_lsum, b->max_layers,
                                  e_s, x_dev, y_dev, bad, st));
    LateralParams lp{};
    lp.src.pool = b->d_pool;
    lp.src.page_next = b->d_page_next;
    lp.src.hit_start = b->d_hit_start;
    lp.src.hit_count = b->d_hit_count;
    lp.prim = b->d_prim;
    lp.geoms = b->d_geoms;
    lp.s2l = b->d_s2l;
    lp.n = b->last_n;
    lp.y = y_dev;
    SUPA_CUDA(launch_lateral_targets(lp, st));
    int h = 0;
    SUPA_CUDA(cudaMemcpyAsync(&h, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    if (h) return fail(SUPA_ERR_INVALID_ARG, "a sub-shower starts on a slice outside every readout layer");
    return SUPA_OK;
}

int supa_export_diverted(supa_batch *b, supa_primary *out_dev, int64_t capacity, int64_t *n_out, void *stream) {
    if (!b || !n_out || capacity < 0 || (capacity > 0 && !out_dev))
        return fail(SUPA_ERR_INVALID_ARG, "supa_export_diverted: bad argument");
    *n_out = 0;
    if (!b->sur) return fail(SUPA_ERR_INVALID_ARG, "supa_export_diverted: the batch is not in hybrid mode");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    SUPA_CUDA(cudaMemcpyAsync(&h, b->d_sq_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    const int64_t n = std::min<int64_t>((int64_t)h, (int64_t)b->sq_cap);
    SUPA_CUDA(launch_export_diverted(b->d_sq_rec, std::min(n, capacity), b->d_prim, out_dev, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    *n_out = n;
    return SUPA_OK;
}

int supa_batch_warp_times(supa_batch *b, uint64_t *dst, int64_t capacity, int64_t *n_warps) {
    if (!b || !n_warps || capacity < 0 || (capacity > 0 && !dst))
        return fail(SUPA_ERR_INVALID_ARG, "supa_batch_warp_times: bad argument");
    *n_warps = 0;
    if (!b->d_warp_times) return fail(SUPA_ERR_INVALID_ARG, "the batch was created without record_warp_times");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    const int64_t nw = (int64_t)b->grid * (b->block / 32);
    SUPA_CUDA(cudaDeviceSynchronize());
    if (capacity > 0)
        SUPA_CUDA(cudaMemcpy(dst, b->d_warp_times, (size_t)std::min(nw, capacity) * 16, cudaMemcpyDeviceToHost));
    *n_warps = nw;
    return SUPA_OK;
}

int supa_export_surrogate(supa_batch *b, supa_diverted_record *out_dev, int64_t capacity, int64_t *n_out,
                          void *stream) {
    if (!b || !n_out || capacity < 0 || (capacity > 0 && !out_dev))
        return fail(SUPA_ERR_INVALID_ARG, "supa_export_surrogate: bad argument");
    *n_out = 0;
    if (!b->sur) return fail(SUPA_ERR_INVALID_ARG, "supa_export_surrogate: the batch is not in hybrid mode");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned h = 0;
    SUPA_CUDA(cudaMemcpyAsync(&h, b->d_sq_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    const int64_t n = std::min<int64_t>((int64_t)h, (int64_t)b->sq_cap);
    SUPA_CUDA(launch_export_surrogate(sur_params(b, 0, 0), std::min(n, capacity), out_dev, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    *n_out = n;
    return SUPA_OK;
}

int supa_simulate_batch(const supa_geometry *const *geoms, int32_t n_geoms, const supa_primary *prim_dev, int64_t n,
                        uint64_t seed, uint64_t shower_id_base, const supa_launch_config *cfg, supa_batch **out,
                        void *stream) {
    if (!out) return fail(SUPA_ERR_INVALID_ARG, "supa_simulate_batch: null out");
    int rc = supa_batch_create(geoms, n_geoms, n > 0 ? n : 1, cfg, out);
    if (rc != SUPA_OK) return rc;
    rc = supa_simulate(*out, prim_dev, n, seed, shower_id_base, stream);
    if (rc != SUPA_OK) {
        supa_destroy_batch(*out);
        *out = nullptr;
    }
    return rc;
}

int supa_autotune(const supa_geometry *const *geoms, int32_t n_geoms, const supa_primary *prim_dev, int64_t n,
                  uint64_t seed, supa_launch_config *cfg, double *best_ms, void *stream) {
    if (!geoms || !prim_dev || !cfg || n < 1) return fail(SUPA_ERR_INVALID_ARG, "supa_autotune: bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t sample = std::min<int64_t>(n, 1 << 17);
    supa_launch_config best = *cfg;
    if (best.max_hits > 0) best.max_hits = (int64_t)((double)best.max_hits * sample / n) + (1 << 20);
    if (best.blocks_per_sm <= 0) best.blocks_per_sm = 3;
    if (best.warps_per_block <= 0) best.warps_per_block = 8;
    if (best.stack_depth <= 0) best.stack_depth = 128;
    cudaEvent_t e0, e1;
    SUPA_CUDA(cudaEventCreate(&e0));
    SUPA_CUDA(cudaEventCreate(&e1));
    auto eval = [&](const supa_launch_config &c) -> double {
        supa_batch *b = nullptr;
        if (supa_batch_create(geoms, n_geoms, sample, &c, &b) != SUPA_OK) return INFINITY;
        double ms = INFINITY;
        supa_batch_info info;
        if (supa_simulate(b, prim_dev, sample, seed, 0, stream) == SUPA_OK &&
            supa_batch_get_info(b, &info, stream) == SUPA_OK) {
            for (int rep = 0; rep < 2; ++rep) {
                float t = 0.f;
                if (cudaEventRecord(e0, st) != cudaSuccess) break;
                if (supa_simulate(b, prim_dev, sample, seed, 0, stream) != SUPA_OK) break;
                if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) break;
                cudaEventElapsedTime(&t, e0, e1);
                ms = std::min(ms, (double)t);
            }
        }
        supa_destroy_batch(b);
        return ms;
    };
    double best_t = eval(best);
    auto consider = [&](supa_launch_config c) {
        const double t = eval(c);
        if (t < best_t) {
            best_t = t;
            best = c;
        }
    };
    const int shapes[][2] = {{2, 8}, {3, 8}, {4, 8}, {2, 4}, {3, 4}, {4, 4}};
    const supa_launch_config start = best;
    for (auto &s : shapes) {
        supa_launch_config c = start;
        c.blocks_per_sm = s[0];
        c.warps_per_block = s[1];
        if (c.blocks_per_sm != start.blocks_per_sm || c.warps_per_block != start.warps_per_block) consider(c);
    }
    for (int depth : {96, 128, 192, 256}) {
        supa_launch_config c = best;
        c.stack_depth = depth;
        if (depth != best.stack_depth) consider(c);
    }
    if (best.flush_threshold == 0) best.flush_threshold = 128;
    for (int ft : {-1, 64, 128, 256}) {
        supa_launch_config c = best;
        c.flush_threshold = ft;
        if (ft != best.flush_threshold) consider(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!std::isfinite(best_t)) return fail(SUPA_ERR_CUDA, "supa_autotune: no candidate launch shape ran");
    cfg->blocks_per_sm = best.blocks_per_sm;
    cfg->warps_per_block = best.warps_per_block;
    cfg->stack_depth = best.stack_depth;
    cfg->flush_threshold = best.flush_threshold;
    if (best_ms) *best_ms = best_t;
    g_last_error.clear();
    return SUPA_OK;
}

int supa_batch_get_info(supa_batch *b, supa_batch_info *info, void *stream) {
    if (!b || !info) return fail(SUPA_ERR_INVALID_ARG, "supa_batch_get_info: null argument");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has run on this batch");
    cudaStream_t st = (cudaStream_t)stream;
    int ctrl[4];
    unsigned long long tot[2];
    long long nh = 0;
    SUPA_CUDA(cudaMemcpyAsync(ctrl, b->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaMemcpyAsync(tot, b->d_totals, sizeof(tot), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaMemcpyAsync(&nh, b->d_offsets + b->last_n, sizeof(nh), cudaMemcpyDeviceToHost, st));
    unsigned diverted = 0;
    if (b->sur) SUPA_CUDA(cudaMemcpyAsync(&diverted, b->d_sq_count, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    SUPA_CUDA(cudaStreamSynchronize(st));
    memset(info, 0, sizeof(*info));
    info->n_showers = b->last_n;
    info->n_hits = nh;
    info->n_steps = (int64_t)tot[0];
    info->max_layers = b->max_layers;
    info->offsets_dev = b->d_offsets;
    info->counts_dev = b->sur ? b->d_tot : b->d_hit_count;
    info->steps_dev = b->d_steps;
    info->layer_sums_dev = b->d_lsum;
    info->dead_dev = b->d_dead;
    info->leak_dev = b->d_leak;
    info->escape_dev = b->d_escape;
    info->n_diverted = diverted;
    info->sur_leak_dev = b->sur ? b->d_sur_leak : nullptr;
    b->n_diverted = diverted;
    if (b->sur) {
        int gemm_err = 0;
        const int rc = supa_surrogate_check(b->sur);
        if (rc != SUPA_OK) gemm_err = rc;
        if (gemm_err) {
            info->status = gemm_err;
            return gemm_err;
        }
    }
    if (ctrl[2] & kErrQueueOverflow) {
        info->status = SUPA_ERR_OVERFLOW;
        return fail(SUPA_ERR_OVERFLOW, "%u particles fell below E_s but the surrogate queue holds %d; raise "
                    "queue_capacity", diverted, b->sq_cap);
    }
    if (ctrl[2] == kErrBadPrimary) {
        info->status = SUPA_ERR_INVALID_ARG;
        return fail(SUPA_ERR_INVALID_ARG, "a primary was invalid (geometry index, energy <= 0 or above the lineage "
                    "bound, polar angle outside [0, pi/2), or a non-finite field); its shower is empty");
    }
    if (ctrl[2] != 0) {
        info->status = SUPA_ERR_OVERFLOW;
        return fail(SUPA_ERR_OVERFLOW, "simulation overflowed its %s (error word %d); use fewer showers per batch%s",
                    (ctrl[2] & kErrPoolOverflow) ? "hit pool" : "particle spill stack", ctrl[2],
                    (ctrl[2] & kErrPoolOverflow) ? " or a larger max_hits" : "");
    }
    b->n_hits = nh;
    b->n_steps = (int64_t)tot[0];
    b->info_valid = true;
    return SUPA_OK;
}

static int fetch_common(supa_batch *b, int64_t first, int64_t max_hits, void *dst, bool dev, bool tags,
                        int64_t *n_written, void *stream) {
    if (!b || !dst || !n_written) return fail(SUPA_ERR_INVALID_ARG, "supa_fetch_hits: null argument");
    if (!b->info_valid) return fail(SUPA_ERR_NOT_READY, "call supa_batch_get_info after the simulation first");
    if (tags && !b->tags) return fail(SUPA_ERR_INVALID_ARG, "the batch was created without record_tags");
    if (first < 0 || max_hits < 0) return fail(SUPA_ERR_INVALID_ARG, "negative range");
    const int64_t count = std::max<int64_t>(0, std::min(max_hits, b->n_hits - first));
    *n_written = count;
    if (count == 0) return SUPA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    FetchParams p{};
    p.src.pool = b->d_pool;
    p.src.page_next = b->d_page_next;
    p.src.hit_start = b->d_hit_start;
    p.src.hit_count = b->d_hit_count;
    p.src.offsets = b->d_offsets;
    if (b->sur) {
        p.src.sur_hits = b->d_sur_hits;
        p.src.sur_off = b->d_soff;
        p.src.sur_count = b->d_scount;
    }
    p.tag_pool = tags ? b->d_tags : nullptr;
    p.sur_tags = tags && b->sur ? b->d_sur_tags : nullptr;
    p.n_showers = b->last_n;
    if (dev) {
        p.first = first;
        p.count = count;
        p.dst = tags ? nullptr : (float4 *)dst;
        p.dst_tags = tags ? (unsigned long long *)dst : nullptr;
        SUPA_CUDA(launch_fetch(p, st));
        return SUPA_OK;
    }
    // host destination: one gather into the batch's device staging buffer,
    // then one copy-engine transfer; both asynchronous on the stream, so the
    // transfer can run beside other kernels (e.g. the images) on other
    // streams.  The staging buffer is reused by the next host fetch of this
    // batch, in stream order.
    if (b->stage_cap_hits < count) {
        SUPA_CUDA(cudaStreamSynchronize(st));
        cudaFree(b->d_stage);
        b->d_stage = nullptr;
        b->stage_cap_hits = 0;
        SUPA_CUDA(dalloc(&b->d_stage, (size_t)count));
        b->stage_cap_hits = count;
    }
    p.first = first;
    p.count = count;
    p.dst = b->d_stage;
    SUPA_CUDA(launch_fetch(p, st));
    SUPA_CUDA(cudaMemcpyAsync(dst, b->d_stage, (size_t)count * 16, cudaMemcpyDeviceToHost, st));
    return SUPA_OK;
}

int supa_fetch_hits(supa_batch *b, int64_t first_hit, int64_t max_hits, void *dst, int32_t dst_is_device,
                    int64_t *n_written, void *stream) {
    return fetch_common(b, first_hit, max_hits, dst, dst_is_device != 0, false, n_written, stream);
}

int supa_fetch_hit_tags(supa_batch *b, int64_t first_hit, int64_t max_hits, uint64_t *dst_dev, int64_t *n_written,
                        void *stream) {
    return fetch_common(b, first_hit, max_hits, dst_dev, true, true, n_written, stream);
}

// Two image buffers of at least one layer each must fit in shared memory.
static const size_t kMaxLayerBytes = 108 * 1024;

static int voxelize_impl(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *grid_dev,
                         double *out_of_roi_dev, float4 *hits_dev, int64_t hits_base, void *stream) {
    if (!b || !grid_dev) return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize: null argument");
    // Stream order is enough: the images read what the last supa_simulate on
    // this stream wrote, so both calls can sit in one captured graph.
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    if (shower_begin < 0 || shower_end < shower_begin || shower_end > b->last_n)
        return fail(SUPA_ERR_INVALID_ARG, "shower range [%lld, %lld) outside the batch", (long long)shower_begin,
                    (long long)shower_end);
    const GeomDev &g0 = b->geoms[0]->rec;
    for (auto *g : b->geoms)
        if (g->rec.nx != g0.nx || g->rec.ny != g0.ny || g->rec.wx != g0.wx || g->rec.wy != g0.wy)
            return fail(SUPA_ERR_INVALID_ARG, "all geometries of the batch must share the image grid");
    cudaStream_t st = (cudaStream_t)stream;
    const int64_t n = shower_end - shower_begin;
    if (n == 0) return SUPA_OK;
    const size_t cells = (size_t)g0.nx * g0.ny;
    if ((size_t)(grid_dev) % 16 != 0) return fail(SUPA_ERR_INVALID_ARG, "grid_dev must be 16-byte aligned");
    if (cells * 4 > kMaxLayerBytes) return fail(SUPA_ERR_INVALID_ARG, "one layer image exceeds 108 KiB");
    VoxParams p{};
    p.src.pool = b->d_pool;
    p.src.page_next = b->d_page_next;
    p.src.hit_start = b->d_hit_start;
    p.src.hit_count = b->d_hit_count;
    if (b->sur) {
        p.src.sur_hits = b->d_sur_hits;
        p.src.sur_off = b->d_soff;
        p.src.sur_count = b->d_scount;
    }
    p.s_begin = shower_begin;
    p.n_showers = n;
    p.L = b->max_layers;
    vox_plan(p.L, g0.nx, g0.ny, &p.G, &p.n_groups, &p.list_cap);
    p.nx = g0.nx;
    p.ny = g0.ny;
    p.wx = g0.wx;
    p.wy = g0.wy;
    p.prim = b->d_prim;
    p.geoms = b->d_geoms;
    p.single_geom = 0;
    p.s2l = b->d_s2l;
    p.zmid = b->d_zmid;
    p.grid = grid_dev;
    p.oor = out_of_roi_dev;
    p.ctas_per_sm = b->voxel_ctas;
    p.hits_out = hits_dev;
    p.offsets = b->d_offsets;
    p.hits_base = hits_base;
    SUPA_CUDA(launch_voxelize(p, st));
    return SUPA_OK;
}

int supa_voxelize(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *grid_dev, double *out_of_roi_dev,
                  void *stream) {
    return voxelize_impl(b, shower_begin, shower_end, grid_dev, out_of_roi_dev, nullptr, 0, stream);
}

int supa_voxelize_fetch(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *grid_dev,
                        double *out_of_roi_dev, float *hits_dev, int64_t hits_base, void *stream) {
    if (!hits_dev) return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_fetch: null hit buffer");
    if ((size_t)hits_dev % 16 != 0) return fail(SUPA_ERR_INVALID_ARG, "hits_dev must be 16-byte aligned");
    if (hits_base < 0) return fail(SUPA_ERR_INVALID_ARG, "hits_base must be >= 0");
    return voxelize_impl(b, shower_begin, shower_end, grid_dev, out_of_roi_dev, reinterpret_cast<float4 *>(hits_dev),
                         hits_base, stream);
}

int supa_profiles(supa_batch *b, int64_t shower_begin, int64_t shower_end, int32_t nbins, float r_max,
                  double *longi_dev, double *lat_dev, void *stream) {
    if (!b || !longi_dev || !lat_dev) return fail(SUPA_ERR_INVALID_ARG, "supa_profiles: null argument");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    if (shower_begin < 0 || shower_end < shower_begin || shower_end > b->last_n)
        return fail(SUPA_ERR_INVALID_ARG, "shower range outside the batch");
    if (nbins < 1 || nbins > 4096 || !(r_max > 0.0f)) return fail(SUPA_ERR_INVALID_ARG, "bad binning");
    ProfileParams p{};
    p.src.pool = b->d_pool;
    p.src.page_next = b->d_page_next;
    p.src.hit_start = b->d_hit_start;
    p.src.hit_count = b->d_hit_count;
    if (b->sur) {
        p.src.sur_hits = b->d_sur_hits;
        p.src.sur_off = b->d_soff;
        p.src.sur_count = b->d_scount;
    }
    p.prim = b->d_prim;
    p.lsum = b->d_lsum;
    p.s_begin = shower_begin;
    p.n_showers = shower_end - shower_begin;
    p.L = b->max_layers;
    p.nbins = nbins;
    p.r_max = r_max;
    p.longi = longi_dev;
    p.lat = lat_dev;
    SUPA_CUDA(launch_profiles(p, (cudaStream_t)stream));
    return SUPA_OK;
}

// Cell layout of the per-layer, multi-resolution images (shared by the
// size query and the call).
static int64_t layer_grid_layout(const supa_layer_grid *grids, int32_t n_grids, const int32_t *factors,
                                 int32_t n_factors, GridParams *p) {
    if (!grids || !factors || n_grids < 1 || n_grids > SUPA_MAX_LAYERS || n_factors < 1 ||
        n_factors > kMaxGridFactors)
        return -1;
    int64_t cells = 0;
    for (int r = 0; r < n_factors; ++r) {
        const int f = factors[r];
        if (f < 1 || f > 16) return -1;
        for (int l = 0; l < n_grids; ++l) {
            const supa_layer_grid &g = grids[l];
            if (g.nx < 1 || g.ny < 1 || g.nx > 4096 || g.ny > 4096 || !(g.wx > 0.0f) || !(g.wy > 0.0f) ||
                !std::isfinite(g.wx) || !std::isfinite(g.wy))
                return -1;
            if (p) p->base[r][l] = (int)cells;
            cells += (int64_t)g.nx * f * g.ny * f;
            if (cells > ((int64_t)1 << 30)) return -1;
        }
    }
    if (p) {
        p->n_layers = n_grids;
        p->n_res = n_factors;
        for (int r = 0; r < n_factors; ++r) p->factor[r] = factors[r];
        for (int l = 0; l < n_grids; ++l) p->grid[l] = {grids[l].nx, grids[l].ny, grids[l].wx, grids[l].wy};
        p->cells = (int)cells;
    }
    return cells;
}

int64_t supa_layer_images_cells(const supa_layer_grid *grids, int32_t n_grids, const int32_t *factors,
                                int32_t n_factors) {
    const int64_t c = layer_grid_layout(grids, n_grids, factors, n_factors, nullptr);
    if (c < 0) fail(SUPA_ERR_INVALID_ARG, "supa_layer_images_cells: bad grids or factors");
    return c < 0 ? SUPA_ERR_INVALID_ARG : c;
}

int supa_voxelize_layers(supa_batch *b, int64_t shower_begin, int64_t shower_end, const supa_layer_grid *grids,
                         int32_t n_grids, const int32_t *factors, int32_t n_factors, float *images_dev,
                         double *out_of_roi_dev, void *stream) {
    if (!b || !images_dev) return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_layers: null argument");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    if (shower_begin < 0 || shower_end < shower_begin || shower_end > b->last_n)
        return fail(SUPA_ERR_INVALID_ARG, "shower range outside the batch");
    if ((uintptr_t)images_dev & 15) return fail(SUPA_ERR_INVALID_ARG, "images_dev must be 16-byte aligned");
    GridParams p{};
    const int64_t cells = layer_grid_layout(grids, n_grids, factors, n_factors, &p);
    if (cells < 0) return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_layers: bad grids or factors");
    if (n_grids < b->max_layers)
        return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_layers: %d grids for %d layers", n_grids, b->max_layers);
    if (grid_smem_bytes((int)cells) > 200 * 1024)
        return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_layers: %lld cells per shower exceed shared memory",
                    (long long)cells);
    p.src.pool = b->d_pool;
    p.src.page_next = b->d_page_next;
    p.src.hit_start = b->d_hit_start;
    p.src.hit_count = b->d_hit_count;
    if (b->sur) {
        p.src.sur_hits = b->d_sur_hits;
        p.src.sur_off = b->d_soff;
        p.src.sur_count = b->d_scount;
    }
    p.prim = b->d_prim;
    p.geoms = b->d_geoms;
    p.s2l = b->d_s2l;
    p.zmid = b->d_zmid;
    p.s_begin = shower_begin;
    p.n_showers = shower_end - shower_begin;
    p.single_geom = b->geoms.size() == 1 ? 1 : 0;
    p.images = images_dev;
    p.oor = out_of_roi_dev;
    SUPA_CUDA(launch_voxelize_layers(p, (cudaStream_t)stream));
    return SUPA_OK;
}

int supa_shower_shapes(supa_batch *b, int64_t shower_begin, int64_t shower_end, float *layer_feats_dev,
                       float *shower_feats_dev, void *stream) {
    if (!b || !layer_feats_dev || !shower_feats_dev)
        return fail(SUPA_ERR_INVALID_ARG, "supa_shower_shapes: null argument");
    if (b->last_n < 0) return fail(SUPA_ERR_NOT_READY, "no simulation has been enqueued on this batch");
    if (shower_begin < 0 || shower_end < shower_begin || shower_end > b->last_n)
        return fail(SUPA_ERR_INVALID_ARG, "shower range outside the batch");
    ShapeParams p{};
    p.src.pool = b->d_pool;
    p.src.page_next = b->d_page_next;
    p.src.hit_start = b->d_hit_start;
    p.src.hit_count = b->d_hit_count;
    if (b->sur) {
        p.src.sur_hits = b->d_sur_hits;
        p.src.sur_off = b->d_soff;
        p.src.sur_count = b->d_scount;
    }
    p.prim = b->d_prim;
    p.geoms = b->d_geoms;
    p.s2l = b->d_s2l;
    p.lsum = b->d_lsum;
    p.s_begin = shower_begin;
    p.n_showers = shower_end - shower_begin;
    p.L = b->max_layers;
    p.layer_feats = layer_feats_dev;
    p.shower_feats = shower_feats_dev;
    SUPA_CUDA(launch_shower_shapes(p, (cudaStream_t)stream));
    return SUPA_OK;
}

int supa_voxelize_hits(const supa_geometry *g, const float *hits_dev, const int64_t *offsets_dev, int64_t n_showers,
                       const float *roi_x0_dev, const float *roi_y0_dev, float *grid_dev, double *out_of_roi_dev,
                       void *stream) {
    if (!g || !offsets_dev || !roi_x0_dev || !roi_y0_dev || !grid_dev || (!hits_dev && n_showers > 0))
        return fail(SUPA_ERR_INVALID_ARG, "supa_voxelize_hits: null argument");
    if (n_showers < 0) return fail(SUPA_ERR_INVALID_ARG, "negative shower count");
    if ((size_t)(grid_dev) % 16 != 0 || (size_t)(hits_dev) % 16 != 0)
        return fail(SUPA_ERR_INVALID_ARG, "hits_dev and grid_dev must be 16-byte aligned");
    const size_t cells = (size_t)g->rec.nx * g->rec.ny;
    if (cells * 4 > kMaxLayerBytes) return fail(SUPA_ERR_INVALID_ARG, "one layer image exceeds 108 KiB");
    if (n_showers == 0) return SUPA_OK;
    cudaStream_t st = (cudaStream_t)stream;
    VoxParams p{};
    p.src.hits = (const float4 *)hits_dev;
    p.src.offsets = offsets_dev;
    p.s_begin = 0;
    p.n_showers = n_showers;
    p.L = g->rec.n_layers;
    vox_plan(p.L, g->rec.nx, g->rec.ny, &p.G, &p.n_groups, &p.list_cap);
    p.nx = g->rec.nx;
    p.ny = g->rec.ny;
    p.wx = g->rec.wx;
    p.wy = g->rec.wy;
    p.geoms = g->d_rec;
    p.single_geom = 1;
    p.s2l = g->d_s2l;
    p.zmid = g->d_zmid;
    p.roi_x0 = roi_x0_dev;
    p.roi_y0 = roi_y0_dev;
    p.grid = grid_dev;
    p.oor = out_of_roi_dev;
    SUPA_CUDA(launch_voxelize(p, st));
    return SUPA_OK;
}

}  // extern "C"
