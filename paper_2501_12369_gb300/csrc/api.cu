// The C ABI of libdarb.so (declared in include/darb.h): argument validation, workspace
// carving and kernel launches.  No entry point here allocates device memory.
#include <algorithm>
#include <cstdlib>

#include "trace.h"
#include "validate.h"

bool darb::pdl_enabled() {
    static const bool on = [] {
        const char *e = std::getenv("DARB_PDL");
        return !(e && e[0] == '0');
    }();
    return on;
}

using namespace darb;

namespace {

bool valid_projected(const darb_projected *o) {
    if (!o) return false;
    const void *p[9] = {o->depth,   o->radius,  o->tile_rect,     o->mean2d,   o->conic_o,
                        o->rgb,     o->clamped, o->tiles_touched, o->tile_runs};
    for (const void *q : p)
        if (!q || !aligned16(q)) return false;
    return true;
}

// Compositing reads the projected records only through tile runs, so an empty scene (n = 0)
// may pass NULL buffers; otherwise every buffer must be valid.
bool valid_projected_or_empty(const darb_projected *o) {
    if (!o) return false;
    const void *p[9] = {o->depth,   o->radius,  o->tile_rect,     o->mean2d,   o->conic_o,
                        o->rgb,     o->clamped, o->tiles_touched, o->tile_runs};
    bool all_null = true;
    for (const void *q : p) all_null &= (q == nullptr);
    return all_null || valid_projected(o);
}

ProjectedOut as_out(const darb_projected *o) {
    ProjectedOut r;
    r.depth = o->depth;
    r.radius = o->radius;
    r.tile_rect = reinterpret_cast<int4 *>(o->tile_rect);
    r.mean2d = reinterpret_cast<float2 *>(o->mean2d);
    r.conic_o = reinterpret_cast<float4 *>(o->conic_o);
    r.rgb = o->rgb;
    r.clamped = o->clamped;
    r.tiles_touched = o->tiles_touched;
    r.tile_runs = o->tile_runs;
    return r;
}

}  // namespace

extern "C" {

const char *darb_status_string(darb_status s) {
    switch (s) {
    case DARB_OK: return "ok";
    case DARB_ERR_INVALID_ARG: return "invalid argument";
    case DARB_ERR_WORKSPACE: return "workspace too small";
    case DARB_ERR_CAPACITY: return "instance capacity exceeded";
    case DARB_ERR_CUDA: return "CUDA error";
    case DARB_ERR_TIMEOUT: return "device wait timed out";
    case DARB_ERR_ADMISSION: return "request not admitted";
    case DARB_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

darb_status darb_kernel_defaults(int32_t kind, darb_kernel_params *out) {
    // psi: Sec. B listings ("correctionFactor"), Table 2 for the inverse multiquadric and the
    // Gaussian; q_max / strictness: the listings' main-lobe limits.
    // base / xi / beta / lobes: the kernel as a member of Table 1's family (descriptive; the
    // inverse quadric 1 / (1 + q) of the Sec. B.4 listing is none, base -1).
    static const darb_kernel_params table[kNumKernels - 1] = {
        {DARB_GAUSSIAN, 1.0f, 9.0f, 0, DARB_BASE_GAUSSIAN, 2.0f, 2.0f, 1},
        {DARB_HALF_COSINE, 1.36f, 9.0f, 0, DARB_BASE_HALF_COSINE, (float)(18.0 / kPiD), 2.0f, 1},
        {DARB_RAISED_COSINE, 0.655f, 6.25f, 0, DARB_BASE_RAISED_COSINE, (float)(2.5 / kPiD), 1.0f, 1},
        {DARB_MOD_SINC, 1.18f, 9.0f, 0, DARB_BASE_MOD_SINC, (float)(3.0 / kPiD), 1.0f, 1},
        {DARB_INV_QUADRIC, 1.38f, 9.0f, 1, -1, 1.0f, 2.0f, 1},
        {DARB_INV_MULTIQUADRIC, 1.61f, 9.0f, 1, DARB_BASE_INV_MULTIQUADRIC, 1.0f, 2.0f, 1},
        {DARB_PARABOLA, 1.3f, 9.0f, 0, DARB_BASE_PARABOLA, 9.0f, 2.0f, 1},
    };
    if (!out || kind < 0 || kind >= kNumKernels - 1) return DARB_ERR_INVALID_ARG;  // DARB_GENERIC: darb_kernel_generic
    *out = table[kind];
    return DARB_OK;
}

darb_status darb_kernel_generic(int32_t base, float xi, float beta, int32_t lobes, darb_kernel_params *out) {
    if (!out || base < 0 || base > 5 || !(xi > 0.0f) || !std::isfinite(xi) || !(beta >= 0.5f && beta <= 4.0f) ||
        lobes < 1 || lobes > 64)
        return DARB_ERR_INVALID_ARG;
    const double pi = kPiD;
    const double u_max[6] = {INFINITY, pi / 2, lobes * pi, (lobes + 1) * pi / 2, INFINITY, 1.0};
    const double q_dom = std::isinf(u_max[base]) ? INFINITY : std::pow((double)xi * u_max[base], 2.0 / beta);
    darb_kernel_params k{};
    k.kind = DARB_GENERIC;
    k.psi = 1.0f;
    k.q_max = (float)std::min(9.0, q_dom);
    k.q_max_strict = 0;
    k.base = base;
    k.xi = xi;
    k.beta = beta;
    k.lobes = lobes;
    *out = k;
    return DARB_OK;
}

darb_status darb_kernel_psi(const darb_kernel_params *kparams, double *scratch, double *psi, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_kernel(kparams) || !scratch || !psi) return DARB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    double sums[2] = {0.0, 0.0};
    DARB_CUDA_TRY(launch_psi_moment(*kparams, scratch, st));
    DARB_CUDA_TRY(cudaMemcpyAsync(sums, scratch, sizeof(sums), cudaMemcpyDeviceToHost, st));
    DARB_CUDA_TRY(cudaStreamSynchronize(st));
    if (!(sums[1] > 0.0)) return DARB_ERR_INVALID_ARG;
    *psi = sums[0] / (3.0 * sums[1]);
    return DARB_OK;
}

darb_status darb_tile_grid(const darb_camera *cam, int32_t tile, int32_t *tiles_x, int32_t *tiles_y) {
    if (!valid_camera(cam) || !valid_tile(tile) || !tiles_x || !tiles_y) return DARB_ERR_INVALID_ARG;
    *tiles_x = tile_count(cam->width, tile);
    *tiles_y = tile_count(cam->height, tile);
    return DARB_OK;
}

darb_status darb_preprocess(const darb_splats *splats, const darb_camera *cam, const darb_kernel_params *kparams,
                            int32_t tile, const darb_projected *out, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_splats(splats) || !valid_camera(cam) || !valid_kernel(kparams) || !valid_tile(tile))
        return DARB_ERR_INVALID_ARG;
    if (splats->n == 0) return DARB_OK;
    if (!valid_projected(out)) return DARB_ERR_INVALID_ARG;
    DARB_CUDA_TRY(launch_preprocess(splats->n, *splats, make_cam(*cam), kparams->psi, tile, kparams->q_max, as_out(out),
                                    reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

bool valid_strategy(int s) { return s == DARB_SORT_DEPTH_THEN_TILE || s == DARB_SORT_KEYS64; }

darb_status darb_bin_sort_workspace_size(int32_t n, int32_t tile, const darb_camera *cam, uint64_t capacity,
                                         int32_t strategy, size_t *bytes) {
    if (n < 0 || !valid_tile(tile) || !valid_camera(cam) || !bytes || capacity > kMaxCapacity ||
        !valid_strategy(strategy))
        return DARB_ERR_INVALID_ARG;
    *bytes = sort_workspace_bytes(n, capacity, tile_count(cam->width, tile), tile_count(cam->height, tile), strategy);
    return DARB_OK;
}

darb_status darb_bin_sort(const darb_projected *proj, int32_t n, int32_t tile, const darb_camera *cam,
                          const darb_kernel_params *kparams, void *workspace, size_t workspace_bytes,
                          uint64_t capacity, int32_t strategy, const darb_binning *out, uint64_t *num_instances_host,
                          darb_stream stream) {
    DARB_TRACE(__func__);
    return darb::bin_sort_entry(proj, n, tile, cam, kparams, workspace, workspace_bytes, capacity, strategy, out,
                                num_instances_host, stream, true);
}
}  // extern "C"

darb_status darb::bin_sort_entry(const darb_projected *proj, int32_t n, int32_t tile, const darb_camera *cam,
                                 const darb_kernel_params *kparams, void *workspace, size_t workspace_bytes,
                                 uint64_t capacity, int32_t strategy, const darb_binning *out,
                                 uint64_t *num_instances_host, darb_stream stream, bool allow_fork) {
    if (n < 0 || !valid_tile(tile) || !valid_camera(cam) || !valid_kernel(kparams) || capacity > kMaxCapacity ||
        !out || !valid_strategy(strategy))
        return DARB_ERR_INVALID_ARG;
    if (!out->ranges || !out->num_instances || !out->status || !aligned16(out->ranges)) return DARB_ERR_INVALID_ARG;
    const bool need_keys = strategy == DARB_SORT_KEYS64;
    if (capacity > 0 && (!out->values || !aligned16(out->values) || (need_keys && !out->keys) ||
                         (out->keys && !aligned16(out->keys))))
        return DARB_ERR_INVALID_ARG;
    if (n > 0 && !valid_projected(proj)) return DARB_ERR_INVALID_ARG;
    const int tiles_x = tile_count(cam->width, tile), tiles_y = tile_count(cam->height, tile);
    const size_t need = sort_workspace_bytes(n, capacity, tiles_x, tiles_y, strategy);
    if (!workspace || workspace_bytes < need || !aligned16(workspace)) return DARB_ERR_WORKSPACE;
    ProjectedIn pin{};
    if (n > 0) {
        pin.depth = proj->depth;
        pin.radius = proj->radius;
        pin.tile_rect = reinterpret_cast<const int4 *>(proj->tile_rect);
        pin.tiles_touched = proj->tiles_touched;
        pin.mean2d = reinterpret_cast<const float2 *>(proj->mean2d);
        pin.conic_o = reinterpret_cast<const float4 *>(proj->conic_o);
        pin.tile_runs = proj->tile_runs;
    }
    const BinOut bo{out->keys, out->values, out->ranges, out->num_instances, out->status};
    bool exceeded = false;
    const SpanCtx sc = make_span_ctx(kparams->q_max, tile, cam->width, cam->height);
    DARB_CUDA_TRY(launch_bin_sort(n, pin, tiles_x, tiles_y, sc, capacity, strategy, workspace, bo,
                                  num_instances_host, &exceeded, reinterpret_cast<cudaStream_t>(stream), allow_fork));
    return exceeded ? DARB_ERR_CAPACITY : DARB_OK;
}

extern "C" {

darb_status darb_render_fwd(const darb_projected *proj, const darb_binning *bins, const darb_camera *cam,
                            const darb_kernel_params *kparams, int32_t tile, const darb_image *out,
                            darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_projected_or_empty(proj) || !bins || !bins->ranges || !valid_camera(cam) || !valid_kernel(kparams) ||
        !valid_tile(tile) || !out || !out->image || !out->t_final || !out->last || !out->n_contrib)
        return DARB_ERR_INVALID_ARG;
    const int tiles_x = tile_count(cam->width, tile), tiles_y = tile_count(cam->height, tile);
    DARB_CUDA_TRY(launch_render_fwd(kparams->kind, tile, tiles_x, tiles_y, bins->ranges, bins->values,
                                    reinterpret_cast<const float2 *>(proj->mean2d),
                                    reinterpret_cast<const float4 *>(proj->conic_o), proj->rgb, make_cam(*cam),
                                    kparams->q_max, kparams->q_max_strict ? 1 : 0, make_spec(*kparams), out->image,
                                    out->t_final, out->last,
                                    out->n_contrib, reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_render_fwd_l1(const darb_projected *proj, const darb_binning *bins, const darb_camera *cam,
                               const darb_kernel_params *kparams, int32_t tile, const darb_image *out,
                               const float *target, float *dL_dimage, float *loss, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_projected_or_empty(proj) || !bins || !bins->ranges || !valid_camera(cam) || !valid_kernel(kparams) ||
        !valid_tile(tile) || !out || !out->t_final || !out->last || !target || !dL_dimage || !loss)
        return DARB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    DARB_CUDA_TRY(launch_zero(st, loss, sizeof(float)));
    const int tiles_x = tile_count(cam->width, tile), tiles_y = tile_count(cam->height, tile);
    DARB_CUDA_TRY(launch_render_fwd(kparams->kind, tile, tiles_x, tiles_y, bins->ranges, bins->values,
                                    reinterpret_cast<const float2 *>(proj->mean2d),
                                    reinterpret_cast<const float4 *>(proj->conic_o), proj->rgb, make_cam(*cam),
                                    kparams->q_max, kparams->q_max_strict ? 1 : 0, make_spec(*kparams), out->image,
                                    out->t_final, out->last, out->n_contrib, st, target, dL_dimage, loss));
    return DARB_OK;
}

darb_status darb_render_bwd(const darb_projected *proj, int32_t n, const darb_binning *bins, const darb_camera *cam,
                            const darb_kernel_params *kparams, int32_t tile, const darb_image *fwd,
                            const float *dL_dimage, float *grad2d, darb_stream stream) {
    DARB_TRACE(__func__);
    if (n < 0 || !valid_projected_or_empty(proj) || !bins || !bins->ranges || !valid_camera(cam) ||
        !valid_kernel(kparams) || !valid_tile(tile) || !fwd || !fwd->t_final || !fwd->last || !dL_dimage ||
        (n > 0 && (!grad2d || !aligned16(grad2d))))
        return DARB_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    if (n > 0) DARB_CUDA_TRY(launch_zero(st, grad2d, (size_t)n * 12 * sizeof(float)));
    const int tiles_x = tile_count(cam->width, tile), tiles_y = tile_count(cam->height, tile);
    DARB_CUDA_TRY(launch_render_bwd(kparams->kind, tile, tiles_x, tiles_y, bins->ranges, bins->values,
                                    reinterpret_cast<const float2 *>(proj->mean2d),
                                    reinterpret_cast<const float4 *>(proj->conic_o), proj->rgb, make_cam(*cam),
                                    kparams->q_max, kparams->q_max_strict ? 1 : 0, make_spec(*kparams), fwd->t_final,
                                    fwd->last, dL_dimage,
                                    grad2d, st));
    return DARB_OK;
}

darb_status darb_preprocess_bwd(const darb_splats *splats, const darb_camera *cam, const darb_kernel_params *kparams,
                                const darb_projected *proj, const float *grad2d, const darb_splat_grads *out,
                                darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_splats(splats) || !valid_camera(cam) || !valid_kernel(kparams)) return DARB_ERR_INVALID_ARG;
    if (splats->n == 0) return DARB_OK;
    if (!valid_projected(proj) || !grad2d || !aligned16(grad2d) || !out || !out->dmeans || !out->dscales ||
        !out->dquats || !out->dopacities || !out->dsh)
        return DARB_ERR_INVALID_ARG;
    GradOut g{out->dmeans, out->dscales, out->dquats, out->dopacities, out->dsh};
    DARB_CUDA_TRY(launch_preprocess_bwd(splats->n, *splats, make_cam(*cam), kparams->psi, proj->radius, proj->clamped,
                                        grad2d, g, reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_l1_loss(const float *image, const float *target, int32_t width, int32_t height, float *dL_dimage,
                         float *loss, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!image || !target || !dL_dimage || !loss || width <= 0 || height <= 0) return DARB_ERR_INVALID_ARG;
    DARB_CUDA_TRY(launch_l1_loss(image, target, 3 * width * height, dL_dimage, loss,
                                 reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_l1_dssim_workspace_size(int32_t width, int32_t height, size_t *bytes) {
    if (width <= 0 || height <= 0 || width > 65536 || height > 65536 || !bytes) return DARB_ERR_INVALID_ARG;
    *bytes = l1_dssim_workspace_bytes(width, height);
    return DARB_OK;
}

darb_status darb_l1_dssim_loss(const float *image, const float *target, int32_t width, int32_t height, float lambda,
                               void *workspace, size_t workspace_bytes, float *dL_dimage, float *loss,
                               darb_stream stream) {
    DARB_TRACE(__func__);
    if (!image || !target || !dL_dimage || !loss || !workspace || width <= 0 || height <= 0 || width > 65536 ||
        height > 65536 || !(lambda >= 0.0f && lambda <= 1.0f))
        return DARB_ERR_INVALID_ARG;
    if (workspace_bytes < l1_dssim_workspace_bytes(width, height)) return DARB_ERR_WORKSPACE;
    DARB_CUDA_TRY(launch_l1_dssim(image, target, width, height, lambda, workspace, dL_dimage, loss,
                                  reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

namespace {

bool train_params_complete(const darb_train_params *p) {
    if (!p || p->n < 0 || p->sh_degree < 0 || p->sh_degree > 3) return false;
    if (p->n == 0) return true;
    const void *q[] = {p->means, p->log_scales, p->quats, p->opacity_logits, p->sh, p->scales, p->opacities};
    for (const void *x : q)
        if (!x || !aligned16(x)) return false;
    return true;
}

bool adam_state_complete(const darb_adam_state *s) {
    if (!s) return false;
    const void *q[] = {s->m_means, s->v_means, s->m_scales, s->v_scales, s->m_quats, s->v_quats,
                       s->m_opac,  s->v_opac,  s->m_sh,     s->v_sh};
    for (const void *x : q)
        if (!x) return false;
    return true;
}

}  // namespace

darb_status darb_densify_stats(const float *grad2d, const int32_t *radius, int32_t n, int32_t width, int32_t height,
                               float *accum, float *count, int32_t *max_radius, darb_stream stream) {
    DARB_TRACE(__func__);
    if (n < 0 || width <= 0 || height <= 0) return DARB_ERR_INVALID_ARG;
    if (n == 0) return DARB_OK;
    if (!grad2d || !aligned16(grad2d) || !radius || !accum || !count || !max_radius) return DARB_ERR_INVALID_ARG;
    DARB_CUDA_TRY(launch_densify_stats(grad2d, radius, n, width, height, accum, count, max_radius,
                                       reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_densify_workspace_size(int32_t n, size_t *bytes) {
    if (n < 0 || !bytes) return DARB_ERR_INVALID_ARG;
    *bytes = densify_workspace_bytes(n);
    return DARB_OK;
}

darb_status darb_densify(const darb_train_params *in, const darb_adam_state *in_state, const float *accum,
                         const float *count, const int32_t *max_radius, const float *split_normals,
                         const darb_densify_cfg *cfg, void *workspace, size_t workspace_bytes, int32_t capacity,
                         const darb_train_params *out, const darb_adam_state *out_state, uint32_t *n_out,
                         darb_stream stream) {
    DARB_TRACE(__func__);
    if (!train_params_complete(in) || !train_params_complete(out) || !adam_state_complete(in_state) ||
        !adam_state_complete(out_state) || !cfg || !workspace || !n_out || out->sh_degree != in->sh_degree ||
        capacity < 0 || (int64_t)capacity < 2 * (int64_t)in->n || !(cfg->split_scale_div > 0.0f) ||
        !std::isfinite(cfg->grad_threshold) || !std::isfinite(cfg->dense_scale))
        return DARB_ERR_INVALID_ARG;
    if (in->n > 0 && (!accum || !count || !max_radius || !split_normals)) return DARB_ERR_INVALID_ARG;
    if (in->means == out->means || in->sh == out->sh || in_state->m_sh == out_state->m_sh) return DARB_ERR_INVALID_ARG;
    if (workspace_bytes < densify_workspace_bytes(in->n)) return DARB_ERR_WORKSPACE;
    DARB_CUDA_TRY(launch_densify(*in, *in_state, accum, count, max_radius, split_normals, *cfg, workspace, *out,
                                 *out_state, n_out, reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_reset_opacity(const darb_train_params *params, float max_opacity, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!train_params_complete(params) || !(max_opacity > 0.0f && max_opacity < 1.0f)) return DARB_ERR_INVALID_ARG;
    DARB_CUDA_TRY(launch_reset_opacity(*params, max_opacity, reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_adam_step(const darb_train_params *params, const darb_splat_grads *grads,
                           const darb_adam_state *state, const darb_adam_config *cfg, darb_stream stream) {
    DARB_TRACE(__func__);
    if (!params || !grads || !state || !cfg || params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3 ||
        cfg->step < 1 || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) || !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) ||
        !(cfg->eps > 0.0f))
        return DARB_ERR_INVALID_ARG;
    if (params->n == 0) return DARB_OK;
    const void *p[] = {params->means, params->log_scales, params->quats, params->opacity_logits, params->sh,
                       params->scales, params->opacities, grads->dmeans, grads->dscales, grads->dquats,
                       grads->dopacities, grads->dsh, state->m_means, state->v_means, state->m_scales,
                       state->v_scales, state->m_quats, state->v_quats, state->m_opac, state->v_opac,
                       state->m_sh, state->v_sh};
    for (const void *q : p)
        if (!q || !aligned16(q)) return DARB_ERR_INVALID_ARG;  // float4 lanes over every group
    DARB_CUDA_TRY(launch_adam(*params, *grads, *state, *cfg, reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

darb_status darb_preprocess_bwd_adam(const darb_train_params *params, const darb_camera *cam,
                                     const darb_kernel_params *kparams, const darb_projected *proj,
                                     const float *grad2d, const darb_adam_state *state, const darb_adam_config *cfg,
                                     darb_stream stream) {
    DARB_TRACE(__func__);
    if (!params || !state || !cfg || params->n < 0 || params->sh_degree < 0 || params->sh_degree > 3 ||
        !valid_camera(cam) || !valid_kernel(kparams) || cfg->step < 1 || !(cfg->beta1 >= 0.0f && cfg->beta1 < 1.0f) ||
        !(cfg->beta2 >= 0.0f && cfg->beta2 < 1.0f) || !(cfg->eps > 0.0f))
        return DARB_ERR_INVALID_ARG;
    if (params->n == 0) return DARB_OK;
    if (!valid_projected(proj) || !grad2d || !aligned16(grad2d)) return DARB_ERR_INVALID_ARG;
    const void *p[] = {params->means, params->log_scales, params->quats, params->opacity_logits, params->sh,
                       params->scales, params->opacities, state->m_means, state->v_means, state->m_scales,
                       state->v_scales, state->m_quats, state->v_quats, state->m_opac, state->v_opac,
                       state->m_sh, state->v_sh};
    for (const void *q : p)
        if (!q || !aligned16(q)) return DARB_ERR_INVALID_ARG;  // float4 lanes over every group
    DARB_CUDA_TRY(launch_preprocess_bwd_adam(params->n, params->sh_degree, *params, *state, make_adam_consts(*cfg),
                                             make_cam(*cam), kparams->psi, proj->radius, proj->clamped, grad2d,
                                             reinterpret_cast<cudaStream_t>(stream)));
    return DARB_OK;
}

}  // extern "C"
