// Batched multi-view forward rendering: many cameras of one splat set per call.
//
// Per view, steps 1-3 (preprocess, depth order, duplication, tile sort) run as in the
// single-view path; views are spread round-robin over `depth` streams so that the sorts of
// small views overlap.  Step 4 is one persistent launch over the tiles of every view
// (k_render_fwd_batch), which keeps all SMs busy across view boundaries.  Nothing in a call
// synchronises with the host or allocates, so a whole batch can be captured into a CUDA graph
// and replayed.
//
// Workspace layout (each region 256-byte aligned): view descriptors, the work-queue counter,
// per-view instance counts and statuses (when the caller passes none), then per view the
// projected splats and the sorted instance values and tile ranges, then one sort workspace
// per stream slot.
#include <algorithm>
#include <mutex>
#include <vector>

#include "trace.h"
#include "validate.h"

namespace darb {
namespace {

constexpr int kMaxBatchDepth = 8;
constexpr int kMaxDevicesBatch = 64;
constexpr int kBlobWords = 960;  // 3840 B of descriptor bytes per upload launch (parameter space)

struct Blob {
    uint32_t words[kBlobWords];
};

// Copies parameter bytes to device memory: host data reaches the device through kernel
// parameters, which stream capture records by value (no host buffer must outlive the call).
__global__ void k_upload(uint32_t *__restrict__ dst, int n_words, Blob blob) {
    pdl_entry();
    for (int i = threadIdx.x; i < n_words; i += blockDim.x) dst[i] = blob.words[i];
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

// Bytes of one view's projected arrays for n splats (each array 256-aligned).
size_t projected_bytes(int n) {
    const size_t N = (size_t)n;
    return a256(4 * N) + a256(4 * N) + a256(16 * N) + a256(8 * N) + a256(16 * N) + a256(12 * N) + a256(N) +
           a256(4 * N) + a256(8 * N);
}

struct BatchLayout {
    size_t desc, queue, counts, status, views, per_view, slots, per_slot, total;
    size_t values_off, ranges_off;  // within a view's block, after the projected arrays
};

BatchLayout batch_layout(int n, const darb_camera *cams, int n_views, int tile, uint64_t capacity, int depth) {
    BatchLayout L{};
    size_t off = 0;
    L.desc = off;
    off += a256(sizeof(BatchView) * (size_t)n_views);
    L.queue = off;
    off += 256;
    L.counts = off;
    off += a256(4 * (size_t)n_views);
    L.status = off;
    off += a256(4 * (size_t)n_views);
    int max_tiles = 0;
    size_t sort_ws = 0;
    for (int v = 0; v < n_views; ++v) {
        const int tx = tile_count(cams[v].width, tile), ty = tile_count(cams[v].height, tile);
        max_tiles = std::max(max_tiles, tx * ty);
        sort_ws = std::max(sort_ws, sort_workspace_bytes(n, capacity, tx, ty, DARB_SORT_DEPTH_THEN_TILE));
    }
    L.values_off = projected_bytes(n);
    L.ranges_off = L.values_off + a256(4 * (size_t)capacity);
    L.per_view = L.ranges_off + a256(8 * (size_t)max_tiles);
    L.views = off;
    off += L.per_view * (size_t)n_views;
    L.per_slot = a256(sort_ws);
    L.slots = off;
    off += L.per_slot * (size_t)depth;
    L.total = off + 256;  // slack for aligning the caller's pointer
    return L;
}

ProjectedOut view_projected(unsigned char *base, int n) {
    const size_t N = (size_t)n;
    ProjectedOut p{};
    size_t o = 0;
    p.depth = reinterpret_cast<float *>(base + o);
    o += a256(4 * N);
    p.radius = reinterpret_cast<int *>(base + o);
    o += a256(4 * N);
    p.tile_rect = reinterpret_cast<int4 *>(base + o);
    o += a256(16 * N);
    p.mean2d = reinterpret_cast<float2 *>(base + o);
    o += a256(8 * N);
    p.conic_o = reinterpret_cast<float4 *>(base + o);
    o += a256(16 * N);
    p.rgb = reinterpret_cast<float *>(base + o);
    o += a256(12 * N);
    p.clamped = reinterpret_cast<uint8_t *>(base + o);
    o += a256(N);
    p.tiles_touched = reinterpret_cast<uint32_t *>(base + o);
    o += a256(4 * N);
    p.tile_runs = reinterpret_cast<uint64_t *>(base + o);
    return p;
}

// Side streams and fork/join events, created once per device and reused; a per-device mutex
// keeps the enqueue of one call (record, wait, launches) from interleaving with another's.
struct DevicePool {
    std::mutex mu;
    bool ready = false;
    cudaStream_t side[kMaxBatchDepth] = {};
    cudaEvent_t fork = nullptr;
    cudaEvent_t join[kMaxBatchDepth] = {};
};

DevicePool g_pools[kMaxDevicesBatch];

cudaError_t pool_init(DevicePool &P) {
    if (P.ready) return cudaSuccess;
    cudaError_t e = cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming);
    if (e != cudaSuccess) return e;
    for (int i = 0; i < kMaxBatchDepth; ++i) {
        e = cudaStreamCreateWithFlags(&P.side[i], cudaStreamNonBlocking);
        if (e != cudaSuccess) return e;
        e = cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return e;
    }
    P.ready = true;
    return cudaSuccess;
}

bool valid_params(const darb_batch_params *bp) {
    return bp && bp->n_views > 0 && bp->n_views <= DARB_MAX_BATCH_VIEWS &&
           (bp->tile == 8 || bp->tile == 16 || bp->tile == 32) && bp->depth >= 1 && bp->depth <= kMaxBatchDepth &&
           bp->capacity >= 1 && bp->capacity <= kMaxCapacity && bp->max_ctas >= 0;
}

}  // namespace
}  // namespace darb

using namespace darb;

extern "C" {

darb_status darb_render_batch_workspace_size(int32_t n, const darb_camera *cams, const darb_batch_params *bp,
                                             size_t *bytes) {
    if (n < 0 || !cams || !valid_params(bp) || !bytes) return DARB_ERR_INVALID_ARG;
    for (int v = 0; v < bp->n_views; ++v)
        if (!valid_camera(&cams[v])) return DARB_ERR_INVALID_ARG;
    *bytes = batch_layout(n, cams, bp->n_views, bp->tile, bp->capacity, bp->depth).total;
    return DARB_OK;
}

darb_status darb_render_batch(const darb_splats *splats, const darb_camera *cams, const darb_kernel_params *kparams,
                              const darb_batch_params *bp, void *workspace, size_t workspace_bytes,
                              const darb_image *outs, uint32_t *num_instances, uint32_t *status,
                              darb_stream stream) {
    DARB_TRACE(__func__);
    if (!valid_splats(splats) || !cams || !valid_kernel(kparams) || !valid_params(bp) || !workspace || !outs)
        return DARB_ERR_INVALID_ARG;
    const int n = splats->n, V = bp->n_views, tile = bp->tile, D = bp->depth;
    for (int v = 0; v < V; ++v)
        if (!valid_camera(&cams[v]) || !outs[v].image) return DARB_ERR_INVALID_ARG;
    const BatchLayout L = batch_layout(n, cams, V, tile, bp->capacity, D);
    if (workspace_bytes < L.total) return DARB_ERR_WORKSPACE;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DARB_ERR_CUDA;
    if (dev < 0 || dev >= kMaxDevicesBatch) return DARB_ERR_INVALID_ARG;
    DevicePool &P = g_pools[dev];
    std::lock_guard<std::mutex> lock(P.mu);
    if (pool_init(P) != cudaSuccess) return DARB_ERR_CUDA;

    unsigned char *w = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(workspace) + 255) &
                                                         ~(uintptr_t)255);
    BatchView *desc = reinterpret_cast<BatchView *>(w + L.desc);
    uint32_t *queue = reinterpret_cast<uint32_t *>(w + L.queue);
    uint32_t *counts = num_instances ? num_instances : reinterpret_cast<uint32_t *>(w + L.counts);
    uint32_t *stats = status ? status : reinterpret_cast<uint32_t *>(w + L.status);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);

    // host-side descriptors, then their upload through kernel parameters
    std::vector<BatchView> hv(V);
    int total_tiles = 0;
    for (int v = 0; v < V; ++v) {
        unsigned char *vb = w + L.views + L.per_view * (size_t)v;
        const ProjectedOut po = view_projected(vb, n);
        const int tx = tile_count(cams[v].width, tile), ty = tile_count(cams[v].height, tile);
        BatchView &b = hv[v];
        b.ranges = reinterpret_cast<const uint2 *>(vb + L.ranges_off);
        b.values = reinterpret_cast<const uint32_t *>(vb + L.values_off);
        b.mean2d = po.mean2d;
        b.conic_o = po.conic_o;
        b.rgb = po.rgb;
        b.image = outs[v].image;
        b.t_final = outs[v].t_final;
        b.last = outs[v].last;
        b.n_contrib = outs[v].n_contrib;
        b.W = cams[v].width;
        b.H = cams[v].height;
        b.tiles_x = tx;
        b.tile_begin = total_tiles;
        b.bg[0] = cams[v].bg[0];
        b.bg[1] = cams[v].bg[1];
        b.bg[2] = cams[v].bg[2];
        b.pad_ = 0.0f;
        total_tiles += tx * ty;
    }
    static_assert(sizeof(BatchView) % 4 == 0, "descriptor words");
    const int words = (int)(sizeof(BatchView) * (size_t)V / 4);
    const uint32_t *src = reinterpret_cast<const uint32_t *>(hv.data());
    for (int o = 0; o < words; o += kBlobWords) {
        Blob blob;
        const int cnt = std::min(kBlobWords, words - o);
        std::copy(src + o, src + o + cnt, blob.words);
        launch_k(k_upload, 1, 256, 0, st, reinterpret_cast<uint32_t *>(desc) + o, cnt, blob);
    }
    if (cudaGetLastError() != cudaSuccess) return DARB_ERR_CUDA;

    // fork: every slot stream starts after what is already on the caller's stream
    const int slots = std::min(D, V);
    if (cudaEventRecord(P.fork, st) != cudaSuccess) return DARB_ERR_CUDA;
    for (int s = 0; s < slots; ++s)
        if (cudaStreamWaitEvent(P.side[s], P.fork, 0) != cudaSuccess) return DARB_ERR_CUDA;
    for (int v = 0; v < V; ++v) {
        const int s = v % slots;
        cudaStream_t ss = P.side[s];
        unsigned char *vb = w + L.views + L.per_view * (size_t)v;
        const ProjectedOut po = view_projected(vb, n);
        const Cam cam = make_cam(cams[v]);
        if (launch_preprocess(n, *splats, cam, kparams->psi, tile, kparams->q_max, po, ss) != cudaSuccess)
            return DARB_ERR_CUDA;
        ProjectedIn pin{};
        pin.depth = po.depth;
        pin.radius = po.radius;
        pin.tile_rect = po.tile_rect;
        pin.tiles_touched = po.tiles_touched;
        pin.mean2d = po.mean2d;
        pin.conic_o = po.conic_o;
        pin.tile_runs = po.tile_runs;
        const BinOut bo{nullptr, reinterpret_cast<uint32_t *>(vb + L.values_off),
                        reinterpret_cast<uint32_t *>(vb + L.ranges_off), counts + v, stats + v};
        bool exceeded = false;
        const int tx = tile_count(cams[v].width, tile), ty = tile_count(cams[v].height, tile);
        const SpanCtx sc = make_span_ctx(kparams->q_max, tile, cams[v].width, cams[v].height);
        if (launch_bin_sort(n, pin, tx, ty, sc, bp->capacity, DARB_SORT_DEPTH_THEN_TILE, w + L.slots + L.per_slot * s, bo,
                            nullptr, &exceeded, ss, /*allow_fork=*/false) != cudaSuccess)
            return DARB_ERR_CUDA;
    }
    // join, then one persistent compositing launch over all views
    for (int s = 0; s < slots; ++s) {
        if (cudaEventRecord(P.join[s], P.side[s]) != cudaSuccess) return DARB_ERR_CUDA;
        if (cudaStreamWaitEvent(st, P.join[s], 0) != cudaSuccess) return DARB_ERR_CUDA;
    }
    if (launch_render_fwd_batch(kparams->kind, tile, desc, V, total_tiles, queue, kparams->q_max,
                                kparams->q_max_strict ? 1 : 0, make_spec(*kparams), bp->max_ctas, st) != cudaSuccess)
        return DARB_ERR_CUDA;
    return DARB_OK;
}

}  // extern "C"
