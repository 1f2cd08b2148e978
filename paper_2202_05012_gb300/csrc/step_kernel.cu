// step_kernel.cu -- persistent particle-step kernel: SUPA Algorithm 1 applied
// to every live particle of every shower (Sec. 3, "Propagation Model").
//
// Work decomposition (GB300-first, not the paper's serial loop):
//  * A persistent grid; each warp takes one shower at a time from a device
//    work queue (one atomicAdd per shower) and develops it completely.
//  * Each lane holds one live particle in registers.  At a split the lane
//    keeps daughter 0 and pushes daughter 1 onto the warp's particle stack in
//    shared memory (ballot + popc compaction, no atomics; two 16-byte words
//    per particle); empty lanes refill from the stack.  A stack that outgrows shared memory spills its oldest
//    half to a per-warp region of global scratch.
//  * Stops become float4 hits in the warp's current page of the hit pool, in
//    one of two builds.  STAGED (the default): hits are staged in shared
//    memory (ballot + popc compaction) and flushed with coalesced 16-byte
//    stores once flush_thr are staged.  Direct: the stopping lanes of one
//    iteration write consecutive 16-byte slots straight from registers, so a
//    warp's stores of one iteration are contiguous and L2 merges them into
//    full sectors (about 1.5 % faster on 90-slice showers of 1-100 GeV: no
//    shared-memory round trip).
//  * Deposits are summed exactly in 64-bit fixed point (units of 2^-32) in
//    shared memory -- per layer, and dead / leaked / escaped energy -- with
//    32-bit shared-memory atomics on the integer pipe (GB300's FP64 rate is a
//    small fraction of its FP32 rate), and delivered per shower as FP64.
//    Integer sums are exact and do not depend on the order of the additions.
// Every random draw is keyed by (seed; shower id, slice, lineage id), so the
// result does not depend on which warp runs a shower or in which order.
#include "philox.cuh"
#include "supa_internal.cuh"

namespace supa {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct WarpSmem {
    float4 *stage;                  // STAGED build: staged hits
    unsigned long long *stage_tag;  // and their lineage ids (record_tags)
    float4 *sa, *sb;   // particle stack: (x, y, ux, uy), (uz, E, lin lo, lin hi)
    unsigned long long *lsum;  // [SUPA_MAX_LAYERS] fixed point, units of 2^-32
    unsigned long long *acc;   // [kAccDead, kAccLeak, kAccEscape], fixed point
    uint8_t *sk;
};

__host__ __device__ inline size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

__device__ inline WarpSmem carve(unsigned char *base, int C, int H, bool tags) {
    WarpSmem w;
    size_t o = 0;
    w.sa = reinterpret_cast<float4 *>(base + o);
    o += size_t(16) * C;
    w.sb = reinterpret_cast<float4 *>(base + o);
    o += size_t(16) * C;
    w.lsum = reinterpret_cast<unsigned long long *>(base + o);
    w.acc = w.lsum + SUPA_MAX_LAYERS;
    o += size_t(8) * (SUPA_MAX_LAYERS + 4);
    w.sk = base + o;
    o = align16(o + size_t(C));
    w.stage = reinterpret_cast<float4 *>(base + o);
    o += size_t(16) * H;
    w.stage_tag = reinterpret_cast<unsigned long long *>(base + o);
    (void)tags;
    return w;
}

constexpr int kAccDead = 0, kAccLeak = 1, kAccEscape = 2;

// acc += v exactly, on a 64-bit fixed-point sum in shared memory, with 32-bit
// shared-memory atomics: the low word's atomic returns the old value, so the
// carry out of it is known and goes to the high word with v's high part.
__device__ __forceinline__ void add_fixed(unsigned long long *acc, unsigned long long v) {
    uint32_t *w = reinterpret_cast<uint32_t *>(acc);
    const uint32_t lo = (uint32_t)v;
    const uint32_t old = atomicAdd(w, lo);
    const uint32_t hi = (uint32_t)(v >> 32) + (uint32_t)(old + lo < old);
    if (hi) atomicAdd(w + 1, hi);
}

struct Particle {
    float x, y, ux, uy, uz, E;
    unsigned long long lin;
    int k;
};

__device__ __forceinline__ void smem_store(const WarpSmem &w, int i, const Particle &q) {
    w.sa[i] = make_float4(q.x, q.y, q.ux, q.uy);
    w.sb[i] = make_float4(q.uz, q.E, __uint_as_float((uint32_t)q.lin), __uint_as_float((uint32_t)(q.lin >> 32)));
    w.sk[i] = (uint8_t)q.k;
}

__device__ __forceinline__ Particle smem_load(const WarpSmem &w, int i) {
    Particle q;
    const float4 a = w.sa[i], b = w.sb[i];
    q.x = a.x; q.y = a.y; q.ux = a.z; q.uy = a.w; q.uz = b.x; q.E = b.y;
    q.lin = ((unsigned long long)__float_as_uint(b.w) << 32) | __float_as_uint(b.z);
    q.k = w.sk[i];
    return q;
}

__device__ __forceinline__ SpillRec to_rec(const Particle &q) {
    SpillRec r;
    r.x = q.x; r.y = q.y; r.ux = q.ux; r.uy = q.uy; r.uz = q.uz; r.E = q.E;
    r.lin_lo = (uint32_t)q.lin; r.lin_hi = (uint32_t)(q.lin >> 32); r.k = q.k;
    return r;
}

__device__ __forceinline__ Particle from_rec(const SpillRec &r) {
    Particle q;
    q.x = r.x; q.y = r.y; q.ux = r.ux; q.uy = r.uy; q.uz = r.uz; q.E = r.E;
    q.lin = ((unsigned long long)r.lin_hi << 32) | r.lin_lo; q.k = r.k;
    return q;
}

// Deflect unit vector (ux,uy,uz) by polar angle delta toward w (a unit vector
// perpendicular to u): u' = cos(delta) u + sin(delta) w, renormalised.
__device__ __forceinline__ void deflect(float ux, float uy, float uz, float wx, float wy, float wz, float sd,
                                        float cd, float &ox, float &oy, float &oz) {
    ox = fmaf(cd, ux, sd * wx);
    oy = fmaf(cd, uy, sd * wy);
    oz = fmaf(cd, uz, sd * wz);
    const float inv = rsqrtf(fmaf(ox, ox, fmaf(oy, oy, oz * oz)));
    ox *= inv; oy *= inv; oz *= inv;
}

// A survivor of slice k either leaks (last slice), escapes (u_z too small)
// or moves in a straight line to slice k+1.  Returns true if still alive.
__device__ __forceinline__ bool advance(Particle &q, const GeomDev &g, unsigned long long *acc) {
    if (q.k == g.n_slices - 1) { add_fixed(acc + kAccLeak, fixed32(q.E)); return false; }
    if (q.uz <= g.uz_min) { add_fixed(acc + kAccEscape, fixed32(q.E)); return false; }
    // 1/u_z from the SFU (one rounding of about an ulp; u_z > uz_min is a
    // normal number)
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(q.uz));
    q.x = fmaf(g.dz, q.ux * r, q.x);
    q.y = fmaf(g.dz, q.uy * r, q.y);
    q.k += 1;
    return true;
}

// sin and cos of a deflection angle.  Split angles are small (|d| <= 0.5
// for every Table 2 law), where the Taylor series to degree 9 / 10 is exact
// to below float32 rounding (next terms d^11/11! < 1.3e-11, d^12/12! < 6e-13);
// larger angles use the library sincosf.
__device__ __forceinline__ void small_sincos(float d, float *s, float *c) {
    if (fabsf(d) <= 0.5f) {
        const float d2 = d * d;
        *s = d * fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, 1.0f / 362880.0f, -1.0f / 5040.0f), 1.0f / 120.0f),
                               -1.0f / 6.0f), 1.0f);
        *c = fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, -1.0f / 3628800.0f, 1.0f / 40320.0f), -1.0f / 720.0f),
                                    1.0f / 24.0f), -0.5f), 1.0f);
    } else {
        sincosf(d, s, c);
    }
}

struct PageCursor {
    int page;  // current page (-1: none)
    int off;   // next free slot in the page
};

// Take a fresh page from the pool and link it after the current one.
// Lane-uniform.  Returns false if the pool is exhausted.
__device__ __forceinline__ bool next_page(const StepParams &p, PageCursor &pc, int lane) {
    int np = 0;
    if (lane == 0) {
        np = atomicAdd(p.page_counter, 1);
        if (np < p.n_pages && pc.page >= 0) p.page_next[pc.page] = np;
    }
    np = __shfl_sync(kFull, np, 0);
    if (np >= p.n_pages) return false;
    pc.page = np;
    pc.off = 0;
    return true;
}

// STAGED build: write `count` staged hits to the page chain.  Lane-uniform.
__device__ __forceinline__ bool flush(const StepParams &p, const WarpSmem &w, int count, PageCursor &pc, int lane) {
    int done = 0;
    while (done < count) {
        if (pc.off == kPageHits && !next_page(p, pc, lane)) return false;
        const int m = min(count - done, kPageHits - pc.off);
        const size_t base = (size_t)pc.page * kPageHits + pc.off;
        for (int j = lane; j < m; j += 32) p.pool[base + j] = w.stage[done + j];
        if (p.tag_pool)
            for (int j = lane; j < m; j += 32) p.tag_pool[base + j] = w.stage_tag[done + j];
        pc.off += m;
        done += m;
    }
    __syncwarp();
    return true;
}

}  // namespace

size_t warp_smem_bytes(int stack_cap, int stage_cap, bool tags) {
    // particle stack: 2 x 16 B + the slice byte per particle; fixed-point
    // sums; the STAGED build's hit staging (16 B, + 8 B with tags, per slot)
    const size_t o = align16(size_t(32) * stack_cap + size_t(8) * (SUPA_MAX_LAYERS + 4) + size_t(stack_cap));
    return align16(o + size_t(16) * stage_cap + (tags ? size_t(8) * stage_cap : 0));
}

// MINB: resident 256-thread blocks per SM the register budget is cut for
// (3: 80 registers, 4: 64).  REGIONS: some geometry of the batch has lateral
// regions (without, the threshold tables line up with the slice tables).
template <int MINB, bool REGIONS, bool STAGED>
__global__ void __launch_bounds__(256, MINB) supa_step_kernel(const StepParams p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warp_global = blockIdx.x * (blockDim.x >> 5) + wib;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int C = p.stack_cap;
    const bool tags = p.tag_pool != nullptr;
    const WarpSmem w = carve(smem_raw + (size_t)wib * p.warp_smem_bytes, C, p.stage_cap, tags);
    SpillRec *spill = p.spill + (size_t)warp_global * p.spill_cap;
    const uint32_t key0 = (uint32_t)p.seed, key1 = (uint32_t)(p.seed >> 32);

    PageCursor pc{-1, kPageHits};
    unsigned long long warp_steps = 0, warp_hits = 0;
    unsigned long long t_start = 0;
    if (p.warp_times && lane == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));

    while (true) {
        int q = 0;
        if (lane == 0) q = atomicAdd(p.queue_head, 1);
        q = __shfl_sync(kFull, q, 0);
        if (q >= p.n) break;
        if ((*((volatile int *)p.error) & (kErrPoolOverflow | kErrSpillOverflow)) != 0) break;
        const int64_t s = p.queue ? (int64_t)p.queue[q] : (int64_t)q;
        const supa_primary pr = p.prim[s];
        const uint32_t gi = pr.geom & 0xFFFFu;  // geometry index
        const int k0 = (int)(pr.geom >> 16);    // slice the particle enters on (0 for a shower)
        if (gi >= (uint32_t)p.n_geoms || k0 >= p.geoms[gi].n_slices || !(pr.E > 0.0f) ||
            !(pr.E <= p.geoms[gi].e0_max) || !(pr.E < 1073741824.0f) ||
            !(pr.theta >= 0.0f && pr.theta < 1.5707963f) || !isfinite(pr.phi) || !isfinite(pr.x0) ||
            !isfinite(pr.y0)) {
            // invalid primary: report it and leave an empty shower behind
            if (lane == 0) {
                atomicOr(p.error, kErrBadPrimary);
                p.hit_start[s] = 0; p.hit_count[s] = 0; p.steps[s] = 0;
                p.dead[s] = 0.0; p.leak[s] = 0.0; p.escape[s] = 0.0;
            }
            for (int l = lane; l < p.lsum_stride; l += 32) p.lsum[(size_t)s * p.lsum_stride + l] = 0.0;
            continue;
        }
        const GeomDev g = p.geoms[gi];
        const uint32_t sid = (uint32_t)(p.shower_id_base + (uint64_t)s);

        for (int l = lane; l < g.n_layers; l += 32) w.lsum[l] = 0ull;
        if (lane < 3) w.acc[lane] = 0ull;
        if (pc.off == kPageHits && !next_page(p, pc, lane)) {
            if (lane == 0) atomicOr(p.error, kErrPoolOverflow);
            break;
        }
        const unsigned long long start = (unsigned long long)pc.page * kPageHits + pc.off;

        // Initial particle (Sec. 3): impact point on its entry slice (0 for a
        // shower's primary), incidence direction.
        Particle cur;
        bool have = (lane == 0);
        {
            float st, ct, sp, cp;
            sincosf(pr.theta, &st, &ct);
            sincosf(pr.phi, &sp, &cp);
            cur.x = pr.x0; cur.y = pr.y0;
            cur.ux = st * cp; cur.uy = st * sp; cur.uz = ct;
            cur.E = pr.E; cur.lin = 1ull; cur.k = k0;
        }
        int stack_n = 0, spill_n = 0, staged = 0;
        uint32_t n_hits = 0, n_steps = 0;
        bool failed = false;
        __syncwarp();

        while (true) {
            // ---- refill empty lanes from the stack (and the spill region) ----
            const unsigned empty = __ballot_sync(kFull, !have);
            const int n_empty = __popc(empty);
            if (n_empty > stack_n && spill_n > 0) {
                const int m = min(spill_n, min(C - stack_n, C / 2));
                for (int j = lane; j < m; j += 32) smem_store(w, stack_n + j, from_rec(spill[spill_n - m + j]));
                stack_n += m;
                spill_n -= m;
                __syncwarp();
            }
            const int n_pop = min(n_empty, stack_n);
            if (!have) {
                const int r = __popc(empty & lt_mask);
                if (r < n_pop) {
                    cur = smem_load(w, stack_n - 1 - r);
                    have = true;
                }
            }
            stack_n -= n_pop;
            __syncwarp();
            const unsigned act = __ballot_sync(kFull, have);
            if (act == 0) break;

            // ---- hybrid path: hand particles below E_s (in a readout layer)
            //      to the surrogate queue instead of stepping them ----
            if (p.e_s > 0.0f) {
                int lay = -1;
                const bool divert = have && cur.E < p.e_s && (lay = __ldg(p.s2l + g.slice_off + cur.k)) >= 0;
                const unsigned dm = __ballot_sync(kFull, divert);
                if (dm) {
                    unsigned base = 0;
                    if (lane == 0) base = atomicAdd(p.sq_count, (unsigned)__popc(dm));
                    base = __shfl_sync(kFull, base, 0);
                    if (divert) {
                        const unsigned idx = base + (unsigned)__popc(dm & lt_mask);
                        if (idx < (unsigned)p.sq_cap) {
                            SurRec rec;
                            rec.shower = (uint32_t)s;
                            rec.k = (int16_t)cur.k;
                            rec.layer = (int16_t)lay;
                            rec.x = cur.x;
                            rec.y = cur.y;
                            const float r = __frcp_rn(cur.uz);
                            rec.tx = cur.ux * r;
                            rec.ty = cur.uy * r;
                            rec.E = cur.E;
                            rec.lin_lo = (uint32_t)cur.lin;
                            rec.lin_hi = (uint32_t)(cur.lin >> 32);
                            p.sq_rec[idx] = rec;
                            float f[kSurIn];
                            surrogate_features(cur.E, cur.ux, cur.uy, cur.uz, cur.k, lay, g.n_layers,
                                               p.linfo[g.layer_off + lay], p.e_s, f);
#pragma unroll
                            for (int i = 0; i < kSurIn; ++i) p.sq_feat[(size_t)idx * kSurIn + i] = f[i];
                        } else {
                            atomicOr(p.error, kErrQueueOverflow);
                        }
                        have = false;
                    }
                }
            }

            // ---- one step of Algorithm 1 for every active lane ----
            bool push = false, hit = false;
            Particle dau;
            if (have) {
                n_steps += 1;
                const uint4 r = philox4x32_10(
                    make_uint4(sid, (uint32_t)cur.k, (uint32_t)cur.lin, (uint32_t)(cur.lin >> 32)), key0, key1);
                const int so = g.slice_off + cur.k;
                int to = REGIONS ? g.thr_off + cur.k : so;
                float th_lo = g.theta_lo, th_span = g.theta_span, eps_frac = g.eps_frac;
                if (REGIONS && g.n_regions > 1) {
                    // lateral region at this slice (Sec. 4.2): r^2 against the
                    // squared outer radii, float32
                    const float r2 = fmaf(cur.x, cur.x, __fmul_rn(cur.y, cur.y));
                    const RegionDev *rt = p.regions + g.region_off;
                    int reg = 0;
                    RegionDev rv = __ldg(rt);
                    while (reg < g.n_regions - 1 && !(r2 < rv.x)) rv = __ldg(rt + ++reg);
                    to += reg * g.n_slices;
                    th_lo = rv.y;
                    th_span = rv.z;
                    eps_frac = rv.w;
                }
                const unsigned long long r0 = r.x;
                if (r0 < __ldg(p.t_stop + to) || cur.E < g.e_min) {
                    // stop: deposit the energy at slice k
                    const int layer = __ldg(p.s2l + so);
                    if (layer < 0) {
                        add_fixed(w.acc + kAccDead, fixed32(cur.E));
                    } else {
                        hit = true;  // written from cur below (a stopped lane keeps it)
                        add_fixed(&w.lsum[layer], fixed32(cur.E));
                    }
                    have = false;
                } else {
                    if (r0 < __ldg(p.t_ss + to)) {
                        // split into two daughters
                        const float theta = fmaf(th_span, u24(r.y), th_lo);
                        // E_0 / E = (theta/2 + eps)/theta = 1/2 + eps_frac (2U - 1)
                        const float f = fmaf(eps_frac, fmaf(2.0f, u24(r.z), -1.0f), 0.5f);
                        const float d1 = theta * f;                               // theta/2 + eps
                        const float d0 = g.split_literal ? d1 : theta * (1.0f - f);  // theta/2 - eps
                        float sw, cw;
                        // omega = 2 pi U: sin and cos from the SFU over [-pi, pi)
                        // (absolute error ~5e-7), sin(2 pi U) = -sin(2 pi (U - 1/2))
                        __sincosf(6.28318531f * (u24(r.w) - 0.5f), &sw, &cw);
                        sw = -sw;
                        cw = -cw;
                        // orthonormal frame (e1, e2) perpendicular to u (Duff et al. 2017)
                        const float a = -1.0f / (1.0f + cur.uz);
                        const float b = cur.ux * cur.uy * a;
                        const float e1x = fmaf(cur.ux * cur.ux, a, 1.0f), e1y = b, e1z = -cur.ux;
                        const float e2x = b, e2y = fmaf(cur.uy * cur.uy, a, 1.0f), e2z = -cur.uy;
                        const float wx = fmaf(cw, e1x, sw * e2x);
                        const float wy = fmaf(cw, e1y, sw * e2y);
                        const float wz = fmaf(cw, e1z, sw * e2z);
                        float s0, c0, s1, c1;
                        small_sincos(d0, &s0, &c0);
                        small_sincos(d1, &s1, &c1);
                        dau = cur;
                        deflect(cur.ux, cur.uy, cur.uz, -wx, -wy, -wz, s1, c1, dau.ux, dau.uy, dau.uz);
                        deflect(cur.ux, cur.uy, cur.uz, wx, wy, wz, s0, c0, cur.ux, cur.uy, cur.uz);
                        const float E0 = cur.E * f;
                        dau.E = cur.E - E0;
                        cur.E = E0;
                        dau.lin = 2ull * cur.lin + 1ull;
                        cur.lin = 2ull * cur.lin;
                        push = advance(dau, g, w.acc);
                    }
                    have = advance(cur, g, w.acc);
                }
            }

            // ---- push daughters 1 onto the warp stack ----
            const unsigned pm = __ballot_sync(kFull, push);
            const int np = __popc(pm);
            if (np) {
                if (stack_n + np > C) {
                    // spill the oldest half of the stack to global scratch
                    const int m = C / 2;
                    if (spill_n + m > p.spill_cap) {
                        if (lane == 0) atomicOr(p.error, kErrSpillOverflow);
                        failed = true;
                        break;
                    }
                    for (int j = lane; j < m; j += 32) spill[spill_n + j] = to_rec(smem_load(w, j));
                    __syncwarp();
                    for (int j0 = m; j0 < stack_n; j0 += 32) {
                        const int j = j0 + lane;
                        Particle t;
                        if (j < stack_n) t = smem_load(w, j);
                        __syncwarp();
                        if (j < stack_n) smem_store(w, j - m, t);
                        __syncwarp();
                    }
                    stack_n -= m;
                    spill_n += m;
                }
                if (push) smem_store(w, stack_n + __popc(pm & lt_mask), dau);
                stack_n += np;
                __syncwarp();
            }

            // ---- hits: staged in shared memory and flushed past the threshold
            //      (STAGED), or written straight to the page chain ----
            if (STAGED) {
                const unsigned hm = __ballot_sync(kFull, hit);
                const int nh = __popc(hm);
                if (nh) {
                    if (hit) {
                        const int idx = staged + __popc(hm & lt_mask);
                        w.stage[idx] = make_float4(cur.x, cur.y, (float)cur.k * g.dz, cur.E);
                        if (tags) w.stage_tag[idx] = cur.lin;
                    }
                    staged += nh;
                    n_hits += nh;
                    __syncwarp();
                    if (staged >= p.flush_thr) {
                        if (!flush(p, w, staged, pc, lane)) {
                            if (lane == 0) atomicOr(p.error, kErrPoolOverflow);
                            failed = true;
                            break;
                        }
                        staged = 0;
                    }
                }
            } else {
                const unsigned hm = __ballot_sync(kFull, hit);
                const int nh = __popc(hm);
                if (nh) {
                    const int idx = __popc(hm & lt_mask);
                    const int room = kPageHits - pc.off;  // >= 1
                    if (hit && idx < room) {
                        const size_t a = (size_t)pc.page * kPageHits + pc.off + idx;
                        p.pool[a] = make_float4(cur.x, cur.y, (float)cur.k * g.dz, cur.E);
                        if (tags) p.tag_pool[a] = cur.lin;
                    }
                    if (nh >= room) {
                        // the page is full: the rest go to a fresh page linked after it
                        if (!next_page(p, pc, lane)) {
                            if (lane == 0) atomicOr(p.error, kErrPoolOverflow);
                            failed = true;
                            break;
                        }
                        if (hit && idx >= room) {
                            const size_t a = (size_t)pc.page * kPageHits + (idx - room);
                            p.pool[a] = make_float4(cur.x, cur.y, (float)cur.k * g.dz, cur.E);
                            if (tags) p.tag_pool[a] = cur.lin;
                        }
                        pc.off = nh - room;
                    } else {
                        pc.off += nh;
                    }
                    n_hits += nh;
                }
            }
        }
        if (failed) break;
        if (STAGED && staged && !flush(p, w, staged, pc, lane)) {
            if (lane == 0) atomicOr(p.error, kErrPoolOverflow);
            break;
        }

        // ---- per-shower records ----
        for (int o = 16; o > 0; o >>= 1) {
            n_steps += __shfl_xor_sync(kFull, n_steps, o);
        }
        __syncwarp();
        for (int l = lane; l < g.n_layers; l += 32) p.lsum[(size_t)s * p.lsum_stride + l] = from_fixed32(w.lsum[l]);
        for (int l = g.n_layers + lane; l < p.lsum_stride; l += 32) p.lsum[(size_t)s * p.lsum_stride + l] = 0.0;
        if (lane == 0) {
            p.hit_start[s] = start;
            p.hit_count[s] = n_hits;
            p.steps[s] = n_steps;
            p.dead[s] = from_fixed32(w.acc[kAccDead]);
            p.leak[s] = from_fixed32(w.acc[kAccLeak]);
            p.escape[s] = from_fixed32(w.acc[kAccEscape]);
        }
        warp_steps += n_steps;
        warp_hits += n_hits;
        __syncwarp();
    }
    if (lane == 0 && (warp_steps | warp_hits)) {
        atomicAdd(&p.totals[0], warp_steps);
        atomicAdd(&p.totals[1], warp_hits);
    }
    if (p.warp_times && lane == 0) {
        unsigned long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        p.warp_times[2 * warp_global] = t_start;
        p.warp_times[2 * warp_global + 1] = t_end;
    }
}

namespace {
using StepKernel = void (*)(const StepParams);

// The builds of the step kernel: [64-register][lateral regions][staged hits].
StepKernel pick(int minb, bool regions, bool staged) {
    static const StepKernel k[2][2][2] = {
        {{supa_step_kernel<3, false, false>, supa_step_kernel<3, false, true>},
         {supa_step_kernel<3, true, false>, supa_step_kernel<3, true, true>}},
        {{supa_step_kernel<4, false, false>, supa_step_kernel<4, false, true>},
         {supa_step_kernel<4, true, false>, supa_step_kernel<4, true, true>}}};
    return k[minb >= 4][regions][staged];
}
}  // namespace

cudaError_t launch_step(int minb, bool regions, bool staged, const StepParams &p, int grid, int block, size_t smem,
                        cudaStream_t st) {
    pick(minb, regions, staged)<<<grid, block, smem, st>>>(p);
    return cudaGetLastError();
}

cudaError_t step_kernel_attributes(int minb, bool regions, bool staged, int block, size_t smem, int *blocks_per_sm) {
    const StepKernel k = pick(minb, regions, staged);
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // largest shared-memory carve-out, so downsampling CTAs of another batch
    // can share the SM with these blocks
    e = cudaFuncSetAttribute(reinterpret_cast<const void *>(k), cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k, block, smem);
}

}  // namespace supa
