// Host-side argument checks shared by the C-ABI entry points.
#pragma once

#include <cmath>

#include "kernels.cuh"

namespace darb {

inline bool finitef(float x) { return std::isfinite(x); }

inline bool valid_tile(int t) { return t == 8 || t == 16 || t == 32; }

inline bool valid_camera(const darb_camera *c) {
    if (!c) return false;
    if (c->width <= 0 || c->height <= 0 || c->width > 65536 || c->height > 65536) return false;
    if (!(c->fx > 0.0f) || !(c->fy > 0.0f) || !finitef(c->fx) || !finitef(c->fy)) return false;
    if (!finitef(c->cx) || !finitef(c->cy) || !(c->near_plane > 0.0f) || !finitef(c->near_plane)) return false;
    for (int i = 0; i < 16; ++i)
        if (!finitef(c->viewmat[i])) return false;
    for (int i = 0; i < 3; ++i)
        if (!finitef(c->bg[i])) return false;
    return true;
}

inline bool valid_kernel(const darb_kernel_params *k) {
    if (!k || k->kind < 0 || k->kind >= kNumKernels || !(k->psi > 0.0f) || !finitef(k->psi) || !(k->q_max > 0.0f) ||
        !finitef(k->q_max))
        return false;
    if (k->kind != DARB_GENERIC) return true;
    return k->base >= 0 && k->base <= 5 && k->xi > 0.0f && finitef(k->xi) && k->beta >= 0.5f && k->beta <= 4.0f &&
           k->lobes >= 1 && k->lobes <= 64;
}

inline bool valid_splats(const darb_splats *s) {
    if (!s || s->n < 0 || s->sh_degree < 0 || s->sh_degree > 3) return false;
    if (s->n == 0) return true;
    const void *p[5] = {s->means, s->scales, s->quats, s->opacities, s->sh};
    for (const void *q : p)
        if (!q || !aligned16(q)) return false;
    return true;
}

constexpr uint64_t kMaxCapacity = (1ull << 30) - 1;

// darb_bin_sort with a switch: allow_fork false keeps every launch on the caller's stream (no
// library side stream is created or used).
darb_status bin_sort_entry(const darb_projected *proj, int32_t n, int32_t tile, const darb_camera *cam,
                           const darb_kernel_params *kparams, void *workspace, size_t workspace_bytes,
                           uint64_t capacity, int32_t strategy, const darb_binning *out, uint64_t *num_instances_host,
                           darb_stream stream, bool allow_fork);

}  // namespace darb
