// hits.cuh -- walking the hits of one shower (stepped hits along their page
// chain or contiguous range, then the shower's surrogate segment) in the
// kernels that consume point clouds.
#pragma once
#include "supa_internal.cuh"

namespace supa {

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

}  // namespace supa
