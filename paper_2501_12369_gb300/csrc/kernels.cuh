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
};

struct GradOut {
    float *dmeans, *dscales, *dquats, *dopacities, *dsh;
};

// preprocess.cu
cudaError_t launch_preprocess(int n, const darb_splats &sp, const Cam &cam, float psi, int tile,
                              const ProjectedOut &out, cudaStream_t st);
cudaError_t launch_preprocess_bwd(int n, const darb_splats &sp, const Cam &cam, float psi,
                                  const int *radius, const uint8_t *clamped, const float *grad2d,
                                  const GradOut &out, cudaStream_t st);

// binning.cu
constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;  // splats per scan/duplicate CTA
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // keys per onesweep partition
constexpr int kMaxPasses = 8;

struct SortWorkspace {
    uint64_t *keys_alt;
    uint32_t *vals_alt;
    uint32_t *block_sums;     // [nb]
    uint32_t *block_offsets;  // [nb]
    uint32_t *hist;           // [kMaxPasses][256]
    uint32_t *digit_base;     // [kMaxPasses][256]
    uint32_t *lookback;       // [passes][n_parts][256]
    uint32_t *part_counter;   // [kMaxPasses]
    size_t zero_bytes;        // bytes from hist to the end of part_counter, zeroed per call
};

size_t sort_workspace_bytes(int n, uint64_t capacity, int passes);
SortWorkspace carve_sort_workspace(void *base, int n, uint64_t capacity, int passes);

cudaError_t launch_count_instances(int n, const uint32_t *tiles_touched, const SortWorkspace &ws,
                                   uint32_t *num_instances, uint32_t *status, uint64_t capacity,
                                   cudaStream_t st);
cudaError_t launch_duplicate_and_sort(int n, const uint32_t *tiles_touched, const int4 *rect,
                                      const float *depth, int tiles_x, int tile_bits,
                                      uint64_t capacity, uint64_t grid_instances,
                                      const SortWorkspace &ws, uint64_t *keys, uint32_t *values,
                                      uint32_t *ranges, const uint32_t *num_instances,
                                      uint32_t *status, cudaStream_t st);

// render.cu
cudaError_t launch_render_fwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict,
                              float *image, float *t_final, uint32_t *last, uint32_t *n_contrib,
                              cudaStream_t st);
cudaError_t launch_render_bwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict,
                              const float *t_final, const uint32_t *last, const float *dL_dimage,
                              float *grad2d, cudaStream_t st);

// train.cu
cudaError_t launch_l1_loss(const float *image, const float *target, int count, float *dL, float *loss,
                           cudaStream_t st);
cudaError_t launch_adam(const darb_train_params &p, const darb_splat_grads &g, const darb_adam_state &s,
                        const darb_adam_config &c, cudaStream_t st);

}  // namespace darb
