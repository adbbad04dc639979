// Step 4 and its backward: per-pixel front-to-back compositing over each tile's depth-sorted
// splat run (paper Sec. 4.1 "alpha blending ... similar to 3DGS", Eq. HalfCosine and
// Eq. 2DSplattedFunction; forward and backward listings of Sec. B).
//
// One CTA per tile.  Each thread owns PIX pixels of one column of the tile (rows r, r + TILE/PIX,
// ...), so every splat record loaded from shared memory serves PIX pixels and dx is shared.  The
// tile's run is consumed in batches of NT records (NT = threads): each thread gathers one splat's
// record (mean, conic, opacity, colour) into shared memory, then every thread walks the batch.  A
// CTA-wide vote ends the loop once every pixel of the tile has stopped (T < 1e-4) -- the early
// termination of 3DGS.
//
// The support test uses the fixed FP32 sequence conic_q(), and alpha / the kernel value are
// computed by the same inline code in forward and backward, so the backward re-takes exactly
// the forward's decisions when it replays a pixel from its last contributor.
#include "kernels.cuh"

namespace darb {

namespace {

struct Bg {
    float r, g, b;
};

constexpr int kMaxDevicesRender = 64;

#ifndef DARB_FWD_PIX32
#define DARB_FWD_PIX32 4
#endif
template <int TILE>
struct RenderShape {
    static constexpr int PIX = TILE == 32 ? DARB_FWD_PIX32 : (TILE >= 16 ? 2 : 1);  // pixels per thread
    static constexpr int NT = TILE * TILE / PIX;      // threads per CTA = records per batch
    static constexpr int ROWS = TILE / PIX;           // row stride between a thread's pixels
};

// Resident CTAs per SM the compositing kernels may be compiled for (a register budget);
// unset, the compiler chooses.  The backward compiles to 64 registers under a budget of 3 or
// of 4 CTAs per SM (4 stay resident either way), but the schedule it gets for 3 measured
// 0.186 ms against 0.190 for the half-cosine at 3M / 1080p (Gaussian 0.604 against 0.612).
#ifndef DARB_BWD_MIN_CTAS
#define DARB_BWD_MIN_CTAS 3
#endif
#ifdef DARB_FWD_MIN_CTAS
#define DARB_FWD_BOUNDS(nt) __launch_bounds__(nt, DARB_FWD_MIN_CTAS)
#else
#define DARB_FWD_BOUNDS(nt) __launch_bounds__(nt)
#endif
#ifdef DARB_BWD_MIN_CTAS
#define DARB_BWD_BOUNDS(nt) __launch_bounds__(nt, DARB_BWD_MIN_CTAS)
#else
#define DARB_BWD_BOUNDS(nt) __launch_bounds__(nt)
#endif

// The backward's shape: with 32-pixel tiles each thread may take more pixels, so that every
// record read from shared memory and every per-warp reduction serves more pixels.
#ifndef DARB_BWD_PIX32
#define DARB_BWD_PIX32 4
#endif
template <int TILE>
struct BwdShape {
    static constexpr int PIX = TILE == 32 ? DARB_BWD_PIX32 : RenderShape<TILE>::PIX;
    static constexpr int NT = TILE * TILE / PIX;
    static constexpr int ROWS = TILE / PIX;
};

// The forward's per-pair body: branch-free, a pair that does not blend taking weight 0 (1), or
// one branch per failed test (0).  Both give the same bits: C + rgb * 0 = C and T is kept.
// Branch-free measured 0.108 -> 0.103 ms (half-cosine) at 3M splats / 1080p.  The backward
// keeps its branches: there a pair that does not contribute would still pay for F', the
// reciprocal and the nine products (0.204 -> 0.212 ms half-cosine, 0.669 -> 0.736 Gaussian).
// Both passes test the support against support_limit(q_max, strict), taken once per thread:
// with the strictness a kernel argument tested per pair, the forward took 0.103 ms and the
// backward 0.204 ms (half-cosine), against 0.089 and 0.190 ms.
#ifndef DARB_FWD_SELECT
#define DARB_FWD_SELECT 1
#endif

// A batch of staged records: the 9 floats of a splat in two float4s and a float (1), so that a
// thread reads a record in 3 shared-memory loads, or as mean, conic + opacity and colour (0).
// Packed measured 0.0886 -> 0.0846 ms (half-cosine) and 0.306 -> 0.293 ms (Gaussian) at 3M
// splats / 1080p.  Folding a pixel's saturation into the branch-free predicate instead of
// skipping it by a branch was mixed (+2% half-cosine, -2% Gaussian) and is not done.  The
// backward keeps its three arrays: packed, its red and green stay live across the pixel loop
// (65-71 registers, 3 CTAs per SM), 0.187 -> 0.193 ms (half-cosine), 0.603 -> 0.621 (Gaussian).
#ifndef DARB_FWD_PACK
#define DARB_FWD_PACK 1
#endif

// The forward's branch-free body on pairs of a thread's pixels with the packed two-lane FP32
// instructions of sm_100+ (1), or one pixel at a time (0).  The backward keeps one pixel at a
// time: paired (a pair with one contributing lane costing what one pixel does), it needed 80
// registers and 3 CTAs per SM and measured 0.195 against 0.186 ms (half-cosine), also with
// each warp's pixels in 4 consecutive rows so that more pairs have both lanes contributing.
#ifndef DARB_FWD_PAIR
#define DARB_FWD_PAIR 1
#endif

template <int TILE>
struct FwdSmem {
#if DARB_FWD_PACK
    float4 a[RenderShape<TILE>::NT];  // x, y, A, 2B
    float4 b[RenderShape<TILE>::NT];  // C, opacity, red, green
    float c[RenderShape<TILE>::NT];   // blue
#else
    float2 xy[RenderShape<TILE>::NT];
    float4 co[RenderShape<TILE>::NT];  // A, 2B, C, opacity
    float rgb[RenderShape<TILE>::NT][3];
#endif
};

// Where a tile's results go; t_final, last and n_contrib may be null (not written).
struct FwdSink {
    float *image;
    float *t_final;
    uint32_t *last;
    uint32_t *n_contrib;
    Bg bg;
};

// The L1 image loss (Sec. 4.2) taken in the forward's epilogue, where each pixel's colour is
// in registers: dL/dC = sign(C - target) / count per channel, and the block's sum of
// |C - target| / count added to *loss (zeroed by the caller).
struct L1Out {
    const float *target;
    float *dL;
    float *loss;
    float inv_count;
};

// One tile of one view, by the whole CTA.  sink() is called once, after the compositing loop,
// so the output pointers need not stay live in registers across it.  With L1 the epilogue also
// takes the L1 loss of the tile's pixels (every thread of the CTA reaches it).
template <int KIND, int TILE, bool L1 = false, class SinkFn>
__device__ __forceinline__ void render_tile_fwd(int tile, FwdSmem<TILE> &sm, const uint2 *__restrict__ ranges,
                                                const uint32_t *__restrict__ values,
                                                const float2 *__restrict__ mean2d,
                                                const float4 *__restrict__ conic_o, const float *__restrict__ rgb,
                                                int W, int H, int tiles_x, float qmax, int strict,
                                                const KernelSpec &ks, SinkFn sink, const L1Out &l1 = L1Out{},
                                                float *s_l1 = nullptr) {
    using S = RenderShape<TILE>;
    constexpr int NT = S::NT, PIX = S::PIX;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * TILE + (threadIdx.x % TILE);
    const int py0 = ty * TILE + (threadIdx.x / TILE);
    const float fpx = (float)px + 0.5f;
    const uint2 r = ranges[tile];
    const int start = (int)r.x, end = (int)r.y;
    const float qlim = support_limit(qmax, strict);

    float fpy[PIX], T[PIX], C0[PIX], C1[PIX], C2[PIX];
    uint32_t count[PIX], lastp[PIX];
    bool done[PIX];
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int py = py0 + k * S::ROWS;
        fpy[k] = (float)py + 0.5f;
        T[k] = 1.0f;
        C0[k] = C1[k] = C2[k] = 0.0f;
        count[k] = lastp[k] = 0;
        done[k] = !(px < W && py < H);
    }
    // pixels 2p and 2p + 1 as the lanes of one pair (the packed FP32 instructions)
    constexpr bool kPair = DARB_FWD_PAIR && DARB_FWD_SELECT && PIX % 2 == 0;
    constexpr int NPP = PIX / 2 > 0 ? PIX / 2 : 1;
    float2 T2[NPP], C0p[NPP], C1p[NPP], C2p[NPP], nfpy[NPP];
#pragma unroll
    for (int pp = 0; pp < NPP; ++pp) {
        T2[pp] = make_float2(1.0f, 1.0f);
        C0p[pp] = C1p[pp] = C2p[pp] = make_float2(0.0f, 0.0f);
        nfpy[pp] = make_float2(-fpy[(2 * pp) % PIX], -fpy[(2 * pp + 1) % PIX]);
    }
    for (int b0 = start; b0 < end; b0 += NT) {
        bool all_done = true;
#pragma unroll
        for (int k = 0; k < PIX; ++k) all_done &= done[k];
        if (__syncthreads_count(all_done) == NT) break;
        const int idx = b0 + (int)threadIdx.x;
        if (idx < end) {
            const uint32_t id = values[idx];
            const float2 xy = mean2d[id];
            float4 co = conic_o[id];
            co.y = 2.0f * co.y;
            const float c0 = rgb[3 * (size_t)id], c1 = rgb[3 * (size_t)id + 1], c2 = rgb[3 * (size_t)id + 2];
#if DARB_FWD_PACK
            sm.a[threadIdx.x] = make_float4(xy.x, xy.y, co.x, co.y);
            sm.b[threadIdx.x] = make_float4(co.z, co.w, c0, c1);
            sm.c[threadIdx.x] = c2;
#else
            sm.xy[threadIdx.x] = xy;
            sm.co[threadIdx.x] = co;
            sm.rgb[threadIdx.x][0] = c0;
            sm.rgb[threadIdx.x][1] = c1;
            sm.rgb[threadIdx.x][2] = c2;
#endif
        }
        __syncthreads();
        if (all_done) continue;
        const int nb = min(NT, end - b0);
        for (int j = 0; j < nb; ++j) {
#if DARB_FWD_PACK
            const float4 pa = sm.a[j], pb = sm.b[j];
            const float2 xy = make_float2(pa.x, pa.y);
            const float4 co = make_float4(pa.z, pa.w, pb.x, pb.y);
            const float r0 = pb.z, r1 = pb.w, r2 = sm.c[j];
#else
            const float2 xy = sm.xy[j];
            const float4 co = sm.co[j];
            const float r0 = sm.rgb[j][0], r1 = sm.rgb[j][1], r2 = sm.rgb[j][2];
#endif
            const float dx = __fsub_rn(xy.x, fpx);
            bool any_live = false;
            if constexpr (kPair) {
                // the scalar branch-free body below on pairs of pixels: every paired operation
                // rounds per lane as its scalar form (__fmul_rn, __fmaf_rn, 1 - alpha), so the
                // support decisions and the sums are the same bits
                const uint32_t pos = (uint32_t)(b0 - start + j + 1);
                const float2 dx2 = make_float2(dx, dx), y2 = make_float2(xy.y, xy.y);
                const float2 A2 = make_float2(co.x, co.x), B2 = make_float2(co.y, co.y);
                const float2 Cc2 = make_float2(co.z, co.z), o2 = make_float2(co.w, co.w);
                const float2 one2 = make_float2(1.0f, 1.0f);
#pragma unroll
                for (int pp = 0; pp < NPP; ++pp) {
                    const int k0 = 2 * pp, k1 = 2 * pp + 1;
                    if (done[k0] && done[k1]) continue;
                    any_live = true;
                    const float2 dy = __fadd2_rn(y2, nfpy[pp]);
                    const float2 g = __ffma2_rn(A2, dx2, __fmul2_rn(B2, dy));
                    const float2 q = __ffma2_rn(dx2, g, __fmul2_rn(__fmul2_rn(Cc2, dy), dy));
                    const float2 of = __fmul2_rn(o2, make_float2(kernel_F<KIND>(q.x, ks), kernel_F<KIND>(q.y, ks)));
                    const float2 alpha = make_float2(fminf(kAlphaMax, of.x), fminf(kAlphaMax, of.y));
                    const float2 Tn = __fmul2_rn(T2[pp], __fadd2_rn(one2, make_float2(-alpha.x, -alpha.y)));
                    const bool use0 = !done[k0] && in_support_lim(q.x, qlim) && alpha.x >= kAlphaMin;
                    const bool use1 = !done[k1] && in_support_lim(q.y, qlim) && alpha.y >= kAlphaMin;
                    const bool stop0 = Tn.x < kTMin, stop1 = Tn.y < kTMin;
                    if (use0 && stop0) done[k0] = true;
                    if (use1 && stop1) done[k1] = true;
                    const bool blend0 = use0 && !stop0, blend1 = use1 && !stop1;
                    const float2 wp = __fmul2_rn(alpha, T2[pp]);
                    const float2 w = make_float2(blend0 ? wp.x : 0.0f, blend1 ? wp.y : 0.0f);
                    C0p[pp] = __ffma2_rn(make_float2(r0, r0), w, C0p[pp]);
                    C1p[pp] = __ffma2_rn(make_float2(r1, r1), w, C1p[pp]);
                    C2p[pp] = __ffma2_rn(make_float2(r2, r2), w, C2p[pp]);
                    T2[pp] = make_float2(blend0 ? Tn.x : T2[pp].x, blend1 ? Tn.y : T2[pp].y);
                    count[k0] += blend0 ? 1u : 0u;
                    count[k1] += blend1 ? 1u : 0u;
                    lastp[k0] = blend0 ? pos : lastp[k0];
                    lastp[k1] = blend1 ? pos : lastp[k1];
                }
                if (!any_live) break;
                continue;
            }
#if DARB_FWD_SELECT
            const uint32_t pos = (uint32_t)(b0 - start + j + 1);
#pragma unroll
            for (int k = 0; k < PIX; ++k) {
                if (done[k]) continue;
                any_live = true;
                const float dy = __fsub_rn(xy.y, fpy[k]);
                const float q = conic_q(dx, dy, co.x, co.y, co.z);
                const float alpha = fminf(kAlphaMax, __fmul_rn(co.w, kernel_F<KIND>(q, ks)));
                const float Tn = T[k] * (1.0f - alpha);
                const bool use = in_support_lim(q, qlim) && alpha >= kAlphaMin;
                const bool stop = Tn < kTMin;
                if (use && stop) done[k] = true;
                const bool blend = use && !stop;
                const float w = blend ? alpha * T[k] : 0.0f;  // weight 0 leaves C and T exactly as they are
                C0[k] = fmaf(r0, w, C0[k]);
                C1[k] = fmaf(r1, w, C1[k]);
                C2[k] = fmaf(r2, w, C2[k]);
                T[k] = blend ? Tn : T[k];
                count[k] += blend ? 1u : 0u;
                lastp[k] = blend ? pos : lastp[k];
            }
#else
#pragma unroll
            for (int k = 0; k < PIX; ++k) {
                if (done[k]) continue;
                any_live = true;
                const float dy = __fsub_rn(xy.y, fpy[k]);
                const float q = conic_q(dx, dy, co.x, co.y, co.z);
                if (!in_support_lim(q, qlim)) continue;
                const float alpha = fminf(kAlphaMax, __fmul_rn(co.w, kernel_F<KIND>(q, ks)));
                if (alpha < kAlphaMin) continue;
                const float Tn = T[k] * (1.0f - alpha);
                if (Tn < kTMin) {
                    done[k] = true;
                    continue;
                }
                const float w = alpha * T[k];
                C0[k] = fmaf(r0, w, C0[k]);
                C1[k] = fmaf(r1, w, C1[k]);
                C2[k] = fmaf(r2, w, C2[k]);
                T[k] = Tn;
                ++count[k];
                lastp[k] = (uint32_t)(b0 - start + j + 1);
            }
#endif
            if (!any_live) break;
        }
    }
    if constexpr (kPair) {
#pragma unroll
        for (int pp = 0; pp < NPP; ++pp) {
            T[2 * pp] = T2[pp].x;
            T[2 * pp + 1] = T2[pp].y;
            C0[2 * pp] = C0p[pp].x;
            C0[2 * pp + 1] = C0p[pp].y;
            C1[2 * pp] = C1p[pp].x;
            C1[2 * pp + 1] = C1p[pp].y;
            C2[2 * pp] = C2p[pp].x;
            C2[2 * pp + 1] = C2p[pp].y;
        }
    }
    const size_t plane = (size_t)W * H;
    const FwdSink o = sink();
    float acc = 0.0f;  // the pixels' |C - target| (with L1)
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int py = py0 + k * S::ROWS;
        if (!(px < W && py < H)) continue;
        const size_t pix = (size_t)py * W + px;
        const float c[3] = {fmaf(T[k], o.bg.r, C0[k]), fmaf(T[k], o.bg.g, C1[k]), fmaf(T[k], o.bg.b, C2[k])};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            if (o.image) o.image[ch * plane + pix] = c[ch];
            if constexpr (L1) {
                const float d = c[ch] - l1.target[ch * plane + pix];
                l1.dL[ch * plane + pix] = d > 0.0f ? l1.inv_count : (d < 0.0f ? -l1.inv_count : 0.0f);
                acc += fabsf(d);
            }
        }
        if (o.t_final) o.t_final[pix] = T[k];
        if (o.last) o.last[pix] = lastp[k];
        if (o.n_contrib) o.n_contrib[pix] = count[k];
    }
    if constexpr (L1) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if ((threadIdx.x & 31) == 0) s_l1[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            float sum = 0.0f;
            for (int w = 0; w < S::NT / 32; ++w) sum += s_l1[w];
            atomicAdd(l1.loss, sum * l1.inv_count);
        }
    }
}

template <int KIND, int TILE, bool L1>
__global__ void DARB_FWD_BOUNDS(RenderShape<TILE>::NT)
k_render_fwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ values,
             const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o,
             const float *__restrict__ rgb, int W, int H, int tiles_x, float qmax, int strict, KernelSpec ks, Bg bg,
             float *__restrict__ image, float *__restrict__ t_final, uint32_t *__restrict__ last,
             uint32_t *__restrict__ n_contrib, L1Out l1) {
    pdl_entry();
    __shared__ FwdSmem<TILE> sm;
    __shared__ float s_l1[L1 ? RenderShape<TILE>::NT / 32 : 1];
    render_tile_fwd<KIND, TILE, L1>(blockIdx.x, sm, ranges, values, mean2d, conic_o, rgb, W, H, tiles_x, qmax, strict,
                                    ks, [&] { return FwdSink{image, t_final, last, n_contrib, bg}; }, l1, s_l1);
}

// Several views in one persistent launch: CTAs take (view, tile) items from a device counter
// (items numbered view-major; views[v].tile_begin is the first item of view v) until all are
// done, so small and large views share the GPU without per-view launches or tails.
template <int KIND, int TILE>
__global__ void __launch_bounds__(RenderShape<TILE>::NT,
                                  (RenderShape<TILE>::PIX >= 4 ? 1024 : 1536) / RenderShape<TILE>::NT)
k_render_fwd_batch(const BatchView *__restrict__ views, int n_views, int total_tiles, uint32_t *__restrict__ queue,
                   float qmax, int strict, KernelSpec ks) {
    pdl_entry();
    __shared__ FwdSmem<TILE> sm;
    __shared__ int s_item, s_view;
    for (;;) {
        if (threadIdx.x == 0) {
            const int item = (int)atomicAdd(queue, 1u);
            int v = 0;
            if (item < total_tiles) {  // last view whose first item is <= item
                int lo = 0, hi = n_views - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (views[mid].tile_begin <= item) lo = mid; else hi = mid - 1;
                }
                v = lo;
            }
            s_item = item;
            s_view = v;
        }
        __syncthreads();
        const int item = s_item, v = s_view;
        if (item >= total_tiles) break;
        const BatchView &bv = views[v];
        render_tile_fwd<KIND, TILE>(item - bv.tile_begin, sm, bv.ranges, bv.values, bv.mean2d, bv.conic_o, bv.rgb,
                                    bv.W, bv.H, bv.tiles_x, qmax, strict, ks, [&] {
                                        const BatchView &b = views[v];
                                        return FwdSink{b.image, b.t_final, b.last, b.n_contrib,
                                                       Bg{b.bg[0], b.bg[1], b.bg[2]}};
                                    });
        __syncthreads();  // the CTA is done with s_item and the staging arrays
    }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// Warp sums of v[0..7] by halving exchanges (4 + 2 + 1 shuffles move half of the remaining
// values to the partner lane, then 2 more finish the sum): afterwards lane 4i (and its
// neighbours 4i+1..4i+3) holds the sum of v[i].  v[8] is summed by a plain butterfly into r8.
// 14 shuffles for 9 values instead of 45.
__device__ __forceinline__ float warp_sum8(const float (&v)[9], int lane, float &r8) {
    const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
    float a[4], b[2];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const float send = b4 ? v[i] : v[i + 4];
        a[i] = (b4 ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const float send = b3 ? a[i] : a[i + 2];
        b[i] = (b3 ? a[i + 2] : a[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
    float c = (b2 ? b[1] : b[0]) + __shfl_xor_sync(0xffffffffu, b2 ? b[0] : b[1], 4);
    c += __shfl_xor_sync(0xffffffffu, c, 2);
    c += __shfl_xor_sync(0xffffffffu, c, 1);
    r8 = warp_sum(v[8]);
    return c;  // the sum of v[4 b4 + 2 b3 + b2] = v[lane >> 2]
}

// Backward: replay each pixel back to front from its last contributor.  With T_k the
// transmittance in front of splat k and S the colour composited behind it (background
// included), dC/dalpha_k = c_k T_k - S / (1 - alpha_k) and dC/dc_k = alpha_k T_k.  Only the
// projection of S on the pixel's upstream gradient g is needed: g . dC/dalpha_k =
// T_k (g . c_k) - (g . S) / (1 - alpha_k), and g . S grows by (g . c_k) alpha_k T_k per splat,
// so each pixel carries the scalar g . S instead of three colour channels.
// Per splat and tile the contributions of a thread's pixels are added in registers, summed
// over the warp by shuffles, then across warps in shared memory, then added to grad2d with one
// vector atomic per 4 floats.
template <int KIND, int TILE>
__global__ void DARB_BWD_BOUNDS(BwdShape<TILE>::NT)
k_render_bwd(const uint2 *__restrict__ ranges, const uint32_t *__restrict__ values,
             const float2 *__restrict__ mean2d, const float4 *__restrict__ conic_o,
             const float *__restrict__ rgb, int W, int H, int tiles_x, float qmax, int strict, KernelSpec ks, Bg bg,
             const float *__restrict__ t_final, const uint32_t *__restrict__ last,
             const float *__restrict__ dL_dimage, float4 *__restrict__ grad2d) {
    pdl_entry();
    using S = BwdShape<TILE>;
    constexpr int NT = S::NT, PIX = S::PIX;
    constexpr int NW = NT / 32;
    __shared__ float2 s_xy[NT];
    __shared__ float4 s_co[NT];
    __shared__ float s_rgb[NT][3];
    __shared__ uint32_t s_id[NT];
    __shared__ float s_acc[NT][9];
    __shared__ uint32_t s_max[NW];

    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, ty = tile / tiles_x;
    const int px = tx * TILE + (threadIdx.x % TILE);
    const int py0 = ty * TILE + (threadIdx.x / TILE);
    const float fpx = (float)px + 0.5f;
    const uint2 r = ranges[tile];
    const int start = (int)r.x;
    const float qlim = support_limit(qmax, strict);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const size_t plane = (size_t)W * H;

    float fpy[PIX], T[PIX], g0[PIX], g1[PIX], g2[PIX], GS[PIX];
    uint32_t my_last[PIX];
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < PIX; ++k) {
        const int py = py0 + k * S::ROWS;
        fpy[k] = (float)py + 0.5f;
        T[k] = 1.0f;
        g0[k] = g1[k] = g2[k] = 0.0f;
        my_last[k] = 0;
        if (px < W && py < H) {
            const size_t pix = (size_t)py * W + px;
            T[k] = t_final[pix];
            my_last[k] = last[pix];
            g0[k] = dL_dimage[pix];
            g1[k] = dL_dimage[plane + pix];
            g2[k] = dL_dimage[2 * plane + pix];
        }
        GS[k] = T[k] * fmaf(g2[k], bg.b, fmaf(g1[k], bg.g, g0[k] * bg.r));
        m = max(m, my_last[k]);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
    if (lane == 0) s_max[warp] = m;
    for (int i = threadIdx.x; i < NT * 9; i += NT) (&s_acc[0][0])[i] = 0.0f;
    __syncthreads();
    int nlast = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) nlast = max(nlast, (int)s_max[w]);

    for (int bend = nlast; bend > 0; bend -= NT) {
        const int bstart = max(0, bend - NT);
        const int cnt = bend - bstart;
        if ((int)threadIdx.x < cnt) {
            const uint32_t id = values[start + bstart + threadIdx.x];
            s_id[threadIdx.x] = id;
            const float2 xy = mean2d[id];
            float4 co = conic_o[id];
            co.y = 2.0f * co.y;
            const float c0 = rgb[3 * (size_t)id], c1 = rgb[3 * (size_t)id + 1], c2 = rgb[3 * (size_t)id + 2];
            s_xy[threadIdx.x] = xy;
            s_co[threadIdx.x] = co;
            s_rgb[threadIdx.x][0] = c0;
            s_rgb[threadIdx.x][1] = c1;
            s_rgb[threadIdx.x][2] = c2;
        }
        __syncthreads();
        for (int j = cnt - 1; j >= 0; --j) {
            const int pos = bstart + j;
            float v[9];
#pragma unroll
            for (int u = 0; u < 9; ++u) v[u] = 0.0f;
            bool contrib = false;
            const float2 xy = s_xy[j];
            const float4 co = s_co[j];
            const float dx = __fsub_rn(xy.x, fpx);
#pragma unroll
            for (int k = 0; k < PIX; ++k) {
                if (pos >= (int)my_last[k]) continue;
                const float dy = __fsub_rn(xy.y, fpy[k]);
                const float q = conic_q(dx, dy, co.x, co.y, co.z);
                if (!in_support_lim(q, qlim)) continue;
                const float F = kernel_F<KIND>(q, ks);
                const float of = __fmul_rn(co.w, F);
                const float alpha = fminf(kAlphaMax, of);
                if (alpha < kAlphaMin) continue;
                contrib = true;
                const float om = 1.0f - alpha;
                const float iom = __fdividef(1.0f, om);
                const float Tk = T[k] * iom;
                const float c0 = s_rgb[j][0], c1 = s_rgb[j][1], c2 = s_rgb[j][2];
                const float gc = fmaf(g2[k], c2, fmaf(g1[k], c1, g0[k] * c0));
                const float dalpha = fmaf(Tk, gc, -GS[k] * iom);
                const float w = alpha * Tk;
                GS[k] = fmaf(gc, w, GS[k]);
                T[k] = Tk;
                v[6] = fmaf(w, g0[k], v[6]);
                v[7] = fmaf(w, g1[k], v[7]);
                v[8] = fmaf(w, g2[k], v[8]);
                if (!(of > kAlphaMax)) {
                    v[5] = fmaf(F, dalpha, v[5]);
                    const float dq = co.w * kernel_dF<KIND>(q, ks) * dalpha;
                    const float B = 0.5f * co.y;
                    v[0] = fmaf(2.0f * dq, co.x * dx + B * dy, v[0]);
                    v[1] = fmaf(2.0f * dq, B * dx + co.z * dy, v[1]);
                    v[2] = fmaf(dq, dx * dx, v[2]);
                    v[3] = fmaf(2.0f * dq, dx * dy, v[3]);
                    v[4] = fmaf(dq, dy * dy, v[4]);
                }
            }
            const uint32_t who = __ballot_sync(0xffffffffu, contrib);
            if (who != 0) {
                if ((who & (who - 1)) == 0) {  // one contributing lane: it adds its own values
                    if (contrib) {
#pragma unroll
                        for (int u = 0; u < 9; ++u) atomicAdd(&s_acc[j][u], v[u]);
                    }
                } else {
                    float r8;
                    const float r = warp_sum8(v, lane, r8);
                    if ((lane & 3) == 0) atomicAdd(&s_acc[j][lane >> 2], r);
                    if (lane == 1) atomicAdd(&s_acc[j][8], r8);
                }
            }
        }
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            float *a = s_acc[threadIdx.x];
            bool any = false;
#pragma unroll
            for (int u = 0; u < 9; ++u) any |= a[u] != 0.0f;
            if (any) {
                float4 *gp = grad2d + 3 * (size_t)s_id[threadIdx.x];
                atomicAdd(gp, make_float4(a[0], a[1], a[2], a[3]));
                atomicAdd(gp + 1, make_float4(a[4], a[5], a[6], a[7]));
                atomicAdd(reinterpret_cast<float *>(gp + 2), a[8]);
            }
#pragma unroll
            for (int u = 0; u < 9; ++u) a[u] = 0.0f;
        }
        __syncthreads();
    }
}

template <int KIND, int TILE>
cudaError_t fwd_t(int n_tiles, const uint2 *ranges, const uint32_t *values, const float2 *mean2d,
                  const float4 *conic_o, const float *rgb, const Cam &cam, int tiles_x, float qmax, int strict,
                  const KernelSpec &ks, float *image, float *t_final, uint32_t *last, uint32_t *n_contrib,
                  const L1Out &l1, cudaStream_t st) {
    if (l1.target)
        launch_k(k_render_fwd<KIND, TILE, true>, n_tiles, RenderShape<TILE>::NT, 0, st,
                 ranges, values, mean2d, conic_o, rgb, cam.W, cam.H, tiles_x, qmax, strict, ks,
                 Bg{cam.bg[0], cam.bg[1], cam.bg[2]}, image, t_final, last, n_contrib, l1);
    else
        launch_k(k_render_fwd<KIND, TILE, false>, n_tiles, RenderShape<TILE>::NT, 0, st,
                 ranges, values, mean2d, conic_o, rgb, cam.W, cam.H, tiles_x, qmax, strict, ks,
                 Bg{cam.bg[0], cam.bg[1], cam.bg[2]}, image, t_final, last, n_contrib, l1);
    return cudaGetLastError();
}

template <int KIND, int TILE>
cudaError_t bwd_t(int n_tiles, const uint2 *ranges, const uint32_t *values, const float2 *mean2d,
                  const float4 *conic_o, const float *rgb, const Cam &cam, int tiles_x, float qmax, int strict,
                  const KernelSpec &ks, const float *t_final, const uint32_t *last, const float *dL, float *grad2d,
                  cudaStream_t st) {
    launch_k(k_render_bwd<KIND, TILE>, n_tiles, BwdShape<TILE>::NT, 0, st,
             ranges, values, mean2d, conic_o, rgb, cam.W, cam.H, tiles_x, qmax, strict, ks,
             Bg{cam.bg[0], cam.bg[1], cam.bg[2]}, t_final, last, dL, reinterpret_cast<float4 *>(grad2d));
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_fwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict, const KernelSpec &ks,
                              float *image, float *t_final, uint32_t *last, uint32_t *n_contrib,
                              cudaStream_t st, const float *l1_target, float *l1_dL, float *l1_loss) {
    const int n_tiles = tiles_x * tiles_y;
    if (n_tiles == 0) return cudaSuccess;
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
    const L1Out l1{l1_target, l1_dL, l1_loss, 1.0f / (3.0f * (float)cam.W * (float)cam.H)};
#define FWD_ARGS (n_tiles, rg, values, mean2d, conic_o, rgb, cam, tiles_x, qmax, strict, ks, image, t_final, last, n_contrib, l1, st)
#define FWD_CALL(K, T) fwd_t<K, T> FWD_ARGS
    if (tile == 8) {
        switch (kind) {
        case 0: return FWD_CALL(0, 8); case 1: return FWD_CALL(1, 8); case 2: return FWD_CALL(2, 8);
        case 3: return FWD_CALL(3, 8); case 4: return FWD_CALL(4, 8); case 5: return FWD_CALL(5, 8);
        case 6: return FWD_CALL(6, 8); default: return FWD_CALL(7, 8);
        }
    } else if (tile == 16) {
        switch (kind) {
        case 0: return FWD_CALL(0, 16); case 1: return FWD_CALL(1, 16); case 2: return FWD_CALL(2, 16);
        case 3: return FWD_CALL(3, 16); case 4: return FWD_CALL(4, 16); case 5: return FWD_CALL(5, 16);
        case 6: return FWD_CALL(6, 16); default: return FWD_CALL(7, 16);
        }
    } else {
        switch (kind) {
        case 0: return FWD_CALL(0, 32); case 1: return FWD_CALL(1, 32); case 2: return FWD_CALL(2, 32);
        case 3: return FWD_CALL(3, 32); case 4: return FWD_CALL(4, 32); case 5: return FWD_CALL(5, 32);
        case 6: return FWD_CALL(6, 32); default: return FWD_CALL(7, 32);
        }
    }
#undef FWD_CALL
#undef FWD_ARGS
}

namespace {

template <int KIND, int TILE>
cudaError_t fwd_batch_t(const BatchView *views, int n_views, int total_tiles, uint32_t *queue, float qmax, int strict,
                        const KernelSpec &ks, int max_ctas, cudaStream_t st) {
    static int per_sm[kMaxDevicesRender] = {};  // resident CTAs per SM, once per device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int occ = (dev >= 0 && dev < kMaxDevicesRender) ? per_sm[dev] : 0;
    if (occ == 0) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_render_fwd_batch<KIND, TILE>,
                                                          RenderShape<TILE>::NT, 0);
        if (e != cudaSuccess) return e;
        occ = occ > 0 ? occ : 1;
        if (dev >= 0 && dev < kMaxDevicesRender) per_sm[dev] = occ;
    }
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    long long grid = (long long)sms * occ;
    if (max_ctas > 0 && grid > max_ctas) grid = max_ctas;
    if (grid > total_tiles) grid = total_tiles;
    e = launch_zero(st, queue, sizeof(uint32_t));
    if (e != cudaSuccess) return e;
    launch_k(k_render_fwd_batch<KIND, TILE>, (int)grid, RenderShape<TILE>::NT, 0, st, views, n_views, total_tiles, queue,
             qmax, strict, ks);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_render_fwd_batch(int kind, int tile, const BatchView *views, int n_views, int total_tiles,
                                    uint32_t *queue, float qmax, int strict, const KernelSpec &ks, int max_ctas,
                                    cudaStream_t st) {
    if (total_tiles == 0 || n_views == 0) return cudaSuccess;
#define FB_CALL(K, T) fwd_batch_t<K, T>(views, n_views, total_tiles, queue, qmax, strict, ks, max_ctas, st)
    if (tile == 8) {
        switch (kind) {
        case 0: return FB_CALL(0, 8); case 1: return FB_CALL(1, 8); case 2: return FB_CALL(2, 8);
        case 3: return FB_CALL(3, 8); case 4: return FB_CALL(4, 8); case 5: return FB_CALL(5, 8);
        case 6: return FB_CALL(6, 8); default: return FB_CALL(7, 8);
        }
    } else if (tile == 16) {
        switch (kind) {
        case 0: return FB_CALL(0, 16); case 1: return FB_CALL(1, 16); case 2: return FB_CALL(2, 16);
        case 3: return FB_CALL(3, 16); case 4: return FB_CALL(4, 16); case 5: return FB_CALL(5, 16);
        case 6: return FB_CALL(6, 16); default: return FB_CALL(7, 16);
        }
    } else {
        switch (kind) {
        case 0: return FB_CALL(0, 32); case 1: return FB_CALL(1, 32); case 2: return FB_CALL(2, 32);
        case 3: return FB_CALL(3, 32); case 4: return FB_CALL(4, 32); case 5: return FB_CALL(5, 32);
        case 6: return FB_CALL(6, 32); default: return FB_CALL(7, 32);
        }
    }
#undef FB_CALL
}

cudaError_t launch_render_bwd(int kind, int tile, int tiles_x, int tiles_y, const uint32_t *ranges,
                              const uint32_t *values, const float2 *mean2d, const float4 *conic_o,
                              const float *rgb, const Cam &cam, float qmax, int strict, const KernelSpec &ks,
                              const float *t_final, const uint32_t *last, const float *dL_dimage,
                              float *grad2d, cudaStream_t st) {
    const int n_tiles = tiles_x * tiles_y;
    if (n_tiles == 0) return cudaSuccess;
    const uint2 *rg = reinterpret_cast<const uint2 *>(ranges);
#define BWD_ARGS (n_tiles, rg, values, mean2d, conic_o, rgb, cam, tiles_x, qmax, strict, ks, t_final, last, dL_dimage, grad2d, st)
#define BWD_CALL(K, T) bwd_t<K, T> BWD_ARGS
    if (tile == 8) {
        switch (kind) {
        case 0: return BWD_CALL(0, 8); case 1: return BWD_CALL(1, 8); case 2: return BWD_CALL(2, 8);
        case 3: return BWD_CALL(3, 8); case 4: return BWD_CALL(4, 8); case 5: return BWD_CALL(5, 8);
        case 6: return BWD_CALL(6, 8); default: return BWD_CALL(7, 8);
        }
    } else if (tile == 16) {
        switch (kind) {
        case 0: return BWD_CALL(0, 16); case 1: return BWD_CALL(1, 16); case 2: return BWD_CALL(2, 16);
        case 3: return BWD_CALL(3, 16); case 4: return BWD_CALL(4, 16); case 5: return BWD_CALL(5, 16);
        case 6: return BWD_CALL(6, 16); default: return BWD_CALL(7, 16);
        }
    } else {
        switch (kind) {
        case 0: return BWD_CALL(0, 32); case 1: return BWD_CALL(1, 32); case 2: return BWD_CALL(2, 32);
        case 3: return BWD_CALL(3, 32); case 4: return BWD_CALL(4, 32); case 5: return BWD_CALL(5, 32);
        case 6: return BWD_CALL(6, 32); default: return BWD_CALL(7, 32);
        }
    }
#undef BWD_CALL
#undef BWD_ARGS
}

}  // namespace darb
