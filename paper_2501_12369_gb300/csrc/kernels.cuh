// Internal launch interface between the C ABI (api.cu) and the kernel files.
#pragma once

#include "common.cuh"

namespace darb {

struct ProjectedOut {
    float *depth;
    int *radius;
    int4 *tile_rect;
    float2 *mean2d;
    float4 *conic_o;
    float *rgb;
    uint8_t *clamped;
    uint32_t *tiles_touched;
    uint64_t *tile_runs;
};

struct GradOut {
    float *dmeans, *dscales, *dquats, *dopacities, *dsh;
};

// preprocess.cu
cudaError_t launch_preprocess(int n, const darb_splats &sp, const Cam &cam, float psi, int tile, float qmax,
                              const ProjectedOut &out, cudaStream_t st);
cudaError_t launch_preprocess_bwd(int n, const darb_splats &sp, const Cam &cam, float psi,
                                  const int *radius, const uint8_t *clamped, const float *grad2d,
                                  const GradOut &out, cudaStream_t st);

cudaError_t launch_preprocess_bwd_adam(int n, int sh_degree, const darb_train_params &p, const darb_adam_state &s,
                                       const AdamConsts &ac, const Cam &cam, float psi, const int *radius,
                                       const uint8_t *clamped, const float *grad2d, cudaStream_t st);

// One view of a batched forward render (device memory).  tile_begin: index of the view's first
// tile among all views' tiles, in view order.  t_final, last, n_contrib may be null.
struct BatchView {
    const uint2 *ranges;
    const uint32_t *values;
    const float2 *mean2d;
    const float4 *conic_o;
    const float *rgb;
    float *image;
    float *t_final;
    uint32_t *last;
    uint32_t *n_contrib;
    int W, H, tiles_x, tile_begin;
    float bg[3];
    float pad_;
};

// render.cu: persistent launch over all views' tiles; queue is a device counter (reset here).
// max_ctas > 0 caps the grid (else SMs x resident CTAs).
cudaError_t launch_render_fwd_batch(int kind, int tile, const BatchView *views, int n_views, int total_tiles,
                                    uint32_t *queue, float qmax, int strict, const KernelSpec &ks, int max_ctas,
                                    cudaStream_t st);

// psi.cu: the moment integrals of darb_kernel_psi into sums[0] (r^4 F) and sums[1] (r^2 F).
cudaError_t launch_psi_moment(const darb_kernel_params &k, double *sums, cudaStream_t st);

// ssim.cu: the L1 + D-SSIM image loss and its gradient.
// Zeroes up to three device regions (byte counts multiple of 4) in one kernel launch, which,
// unlike a memset, overlaps its start with the preceding kernel's drain.
cudaError_t launch_zero(cudaStream_t st, void *p0, size_t b0, void *p1 = nullptr, size_t b1 = 0, void *p2 = nullptr,
                        size_t b2 = 0);

size_t l1_dssim_workspace_bytes(int W, int H);
cudaError_t launch_l1_dssim(const float *image, const float *target, int W, int H, float lam, void *workspace,
                            float *dL, float *loss, cudaStream_t st);

// density.cu: adaptive density control.
size_t densify_workspace_bytes(int n);
cudaError_t launch_densify_stats(const float *grad2d, const int *radius, int n, int W, int H, float *accum,
                                 float *count, int *max_radius, cudaStream_t st);
cudaError_t launch_densify(const darb_train_params &in, const darb_adam_state &sin, const float *accum,
                           const float *count, const int *max_radius, const float *normals,
                           const darb_densify_cfg &cfg, void *workspace, const darb_train_params &out,
                           const darb_adam_state &sout, uint32_t *n_out, cudaStream_t st);
cudaError_t launch_reset_opacity(const darb_train_params &p, float max_opacity, cudaStream_t st);

// binning.cu
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // splats per scan/duplicate CTA
// Shape of the one-pass sort CTAs: threads x items per thread keys per partition (4096).
#ifndef DARB_SORT_THREADS
#define DARB_SORT_THREADS 512
#endif
constexpr int kSortThreads = DARB_SORT_THREADS;
constexpr int kSortItems = 4096 / kSortThreads;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per onesweep partition
constexpr int kMaxPasses = 8;

struct ProjectedIn {
    const float *depth;
    const int *radius;
    const int4 *tile_rect;
    const uint32_t *tiles_touched;
    const float2 *mean2d;   // with conic_o: the ellipse whose row spans give the member tiles
    const float4 *conic_o;
    const uint64_t *tile_runs;  // the row spans packed (kRunsUnpacked: recompute them)
};

struct BinOut {
    uint64_t *keys;  // may be null for DARB_SORT_DEPTH_THEN_TILE
    uint32_t *values;
    uint32_t *ranges;
    uint32_t *num_instances;
    uint32_t *status;
};

int sort_tile_bits(int n_tiles);
size_t sort_workspace_bytes(int n, uint64_t capacity, int tiles_x, int tiles_y, int strategy);
// Enqueues the whole bin/sort.  With num_instances_host non-null it synchronises once after the
// scan; if M exceeds the capacity it sets *capacity_exceeded and enqueues nothing more.  With
// allow_fork the per-tile counts run on a library side stream of the device beside the depth
// passes (forked from and joined back to st with events; concurrent calls of one device are
// serialised while they enqueue).
cudaError_t launch_bin_sort(int n, const ProjectedIn &proj, int tiles_x, int tiles_y, const SpanCtx &sc,
                            uint64_t capacity,
                            int strategy, void *workspace, const BinOut &out, uint64_t *num_instances_host,
                            bool *capacity_exceeded, cudaStream_t st, bool allow_fork = true);

// render.cu
// With l1_target non-null the kernel's epilogue also writes the L1 loss gradient to l1_dL and
// adds the loss to *l1_loss (which the caller zeroes).
cudaError_t launch_render_fwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict, const KernelSpec &ks,
                              float *image, float *t_final, uint32_t *last, uint32_t *n_contrib,
                              cudaStream_t st, const float *l1_target = nullptr, float *l1_dL = nullptr,
                              float *l1_loss = nullptr);
cudaError_t launch_render_bwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict, const KernelSpec &ks,
                              const float *t_final, const uint32_t *last, const float *dL_dimage,
                              float *grad2d, cudaStream_t st);

// train.cu
cudaError_t launch_l1_loss(const float *image, const float *target, int count, float *dL, float *loss,
                           cudaStream_t st);
cudaError_t launch_adam(const darb_train_params &p, const darb_splat_grads &g, const darb_adam_state &s,
                        const darb_adam_config &c, cudaStream_t st);

}  // namespace darb
