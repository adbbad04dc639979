// Adaptive density control of the 3DGS optimisation pipeline the paper keeps (Sec. 4 block
// diagram): per-step statistics of the visible splats, then periodically clone, split and prune,
// and the opacity reset.
//
// Statistics (k_densify_stats): the view-space mean gradient in normalised device units
// (pixel gradient x (W/2, H/2)), its norm added to accum, 1 added to count, the largest screen
// radius kept -- for splats with radius > 0.
//
// Densification is a stable three-way stream compaction.  For every splat a fixed float32
// sequence decides: avg = accum / count; grow = avg >= threshold; split = grow and max scale >
// dense_scale; clone = grow and not split; a candidate survives the prune unless its opacity,
// screen radius or world scale crosses a limit (clones and children start with radius 0;
// children carry scales / div).  k_densify_count counts the survivors, kept clones and kept
// split parents of each block, k_densify_offsets scans the block counts, and k_densify_scatter
// writes, in index order within each segment, [survivors | clones | two children per split
// parent].  Survivors keep their Adam moments; clones and children start from zero.  Children's
// means are parent + R(q) (s * z) for the caller's standard-normal draws z.
#include "kernels.cuh"

namespace darb {
namespace {

constexpr int kDenThreads = 256;
constexpr int kDenItems = 8;
constexpr int kDenTile = kDenThreads * kDenItems;

struct DenCfg {
    float thr, dense, min_op, max_screen, max_world, div, log_div;
};

struct Flags {
    bool surv, clone, split;  // survivor, kept clone, split parent with kept children
};

__device__ __forceinline__ bool survives(float opac, float smax, float radius, const DenCfg &c) {
    bool ok = opac >= c.min_op;
    if (c.max_screen > 0.0f) ok = ok && radius <= c.max_screen;
    if (c.max_world > 0.0f) ok = ok && smax <= c.max_world;
    return ok;
}

__device__ __forceinline__ Flags classify(int i, const float *__restrict__ scales, const float *__restrict__ opac,
                                          const float *__restrict__ accum, const float *__restrict__ count,
                                          const int *__restrict__ max_radius, const DenCfg &c) {
    const float cnt = count[i];
    const float avg = cnt > 0.0f ? __fdiv_rn(accum[i], cnt) : 0.0f;
    const float s0 = scales[3 * (size_t)i], s1 = scales[3 * (size_t)i + 1], s2 = scales[3 * (size_t)i + 2];
    const float smax = fmaxf(fmaxf(s0, s1), s2);
    const float o = opac[i];
    const bool grow = avg >= c.thr;
    const bool split = grow && smax > c.dense;
    const bool clone = grow && !split;
    Flags f;
    f.surv = !split && survives(o, smax, (float)max_radius[i], c);
    f.clone = clone && survives(o, smax, 0.0f, c);
    const float cmax = fmaxf(fmaxf(__fdiv_rn(s0, c.div), __fdiv_rn(s1, c.div)), __fdiv_rn(s2, c.div));
    f.split = split && survives(o, cmax, 0.0f, c);
    return f;
}

// 3 counts of up to kDenThreads packed in 10-bit fields of one word
__device__ __forceinline__ uint32_t pack(const Flags &f) {
    return (f.surv ? 1u : 0u) | (f.clone ? 1u << 10 : 0u) | (f.split ? 1u << 20 : 0u);
}

template <int NT>
__device__ __forceinline__ uint32_t block_scan_packed(uint32_t v, uint32_t *s_w, uint32_t &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? s_w[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < NT / 32) s_w[lane] = w;
    }
    __syncthreads();
    const uint32_t excl = (warp > 0 ? s_w[warp - 1] : 0u) + x - v;
    total = s_w[NT / 32 - 1];
    __syncthreads();
    return excl;
}

__global__ void __launch_bounds__(256)
k_densify_stats(const float4 *__restrict__ grad2d, const int *__restrict__ radius, int n, float half_w, float half_h,
                float *__restrict__ accum, float *__restrict__ count, int *__restrict__ max_radius) {
    pdl_entry();
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const int r = radius[i];
    if (r <= 0) return;
    const float4 g = grad2d[3 * (size_t)i];
    const float gx = __fmul_rn(g.x, half_w), gy = __fmul_rn(g.y, half_h);
    const float norm = __fsqrt_rn(__fadd_rn(__fmul_rn(gx, gx), __fmul_rn(gy, gy)));
    accum[i] = __fadd_rn(accum[i], norm);
    count[i] = __fadd_rn(count[i], 1.0f);
    max_radius[i] = max(max_radius[i], r);
}

__global__ void __launch_bounds__(kDenThreads)
k_densify_count(int n, const float *__restrict__ scales, const float *__restrict__ opac,
                const float *__restrict__ accum, const float *__restrict__ count, const int *__restrict__ max_radius,
                DenCfg c, uint32_t *__restrict__ blk) {
    pdl_entry();
    __shared__ uint32_t s_w[kDenThreads / 32];
    uint32_t sum[3] = {0, 0, 0};
    for (int j = 0; j < kDenItems; ++j) {
        const int i = blockIdx.x * kDenTile + j * kDenThreads + threadIdx.x;
        uint32_t v = 0;
        if (i < n) v = pack(classify(i, scales, opac, accum, count, max_radius, c));
        uint32_t tot;
        block_scan_packed<kDenThreads>(v, s_w, tot);
        sum[0] += tot & 1023u;
        sum[1] += (tot >> 10) & 1023u;
        sum[2] += tot >> 20;
    }
    if (threadIdx.x == 0) {
        blk[3 * (size_t)blockIdx.x] = sum[0];
        blk[3 * (size_t)blockIdx.x + 1] = sum[1];
        blk[3 * (size_t)blockIdx.x + 2] = sum[2];
    }
}

// One CTA: exclusive offsets of the three block counts; segment bases; n_out.
__global__ void __launch_bounds__(1024)
k_densify_offsets(int nb, uint32_t *__restrict__ blk, uint32_t *__restrict__ n_out) {
    pdl_entry();
    __shared__ uint32_t s_w[32];
    uint32_t carry[3] = {0, 0, 0};
    for (int f = 0; f < 3; ++f) {
        for (int c0 = 0; c0 < nb; c0 += 1024) {
            const int b = c0 + threadIdx.x;
            const uint32_t v = b < nb ? blk[3 * (size_t)b + f] : 0u;
            uint32_t tot;
            const uint32_t ex = block_scan_packed<1024>(v, s_w, tot);
            if (b < nb) blk[3 * (size_t)b + f] = carry[f] + ex;
            carry[f] += tot;
        }
    }
    if (threadIdx.x == 0) {
        n_out[0] = carry[0] + carry[1] + 2 * carry[2];
        n_out[1] = carry[0];             // clone segment starts here
        n_out[2] = carry[0] + carry[1];  // children start here
    }
}

struct DenIO {
    darb_train_params in, out;
    darb_adam_state sin, sout;
    int k3;  // SH floats per splat
};

__device__ __forceinline__ void copy_row(const float *src, float *dst, int i, int j, int w) {
    for (int e = 0; e < w; ++e) dst[(size_t)j * w + e] = src[(size_t)i * w + e];
}

__device__ __forceinline__ void zero_row(float *dst, int j, int w) {
    for (int e = 0; e < w; ++e) dst[(size_t)j * w + e] = 0.0f;
}

// Copy splat i to row j of the output; moments copied (keep) or zeroed.
__device__ __forceinline__ void emit(const DenIO &io, int i, int j, bool keep_moments) {
    copy_row(io.in.means, io.out.means, i, j, 3);
    copy_row(io.in.log_scales, io.out.log_scales, i, j, 3);
    copy_row(io.in.quats, io.out.quats, i, j, 4);
    copy_row(io.in.opacity_logits, io.out.opacity_logits, i, j, 1);
    copy_row(io.in.sh, io.out.sh, i, j, io.k3);
    copy_row(io.in.scales, io.out.scales, i, j, 3);
    copy_row(io.in.opacities, io.out.opacities, i, j, 1);
    const float *const src[10] = {io.sin.m_means, io.sin.v_means, io.sin.m_scales, io.sin.v_scales, io.sin.m_quats,
                                  io.sin.v_quats, io.sin.m_opac, io.sin.v_opac, io.sin.m_sh, io.sin.v_sh};
    float *const dst[10] = {io.sout.m_means, io.sout.v_means, io.sout.m_scales, io.sout.v_scales, io.sout.m_quats,
                            io.sout.v_quats, io.sout.m_opac, io.sout.v_opac, io.sout.m_sh, io.sout.v_sh};
    const int w[10] = {3, 3, 3, 3, 4, 4, 1, 1, io.k3, io.k3};
    for (int a = 0; a < 10; ++a) {
        if (keep_moments) copy_row(src[a], dst[a], i, j, w[a]);
        else zero_row(dst[a], j, w[a]);
    }
}

__global__ void __launch_bounds__(kDenThreads)
k_densify_scatter(int n, DenIO io, const float *__restrict__ accum, const float *__restrict__ count,
                  const int *__restrict__ max_radius, const float *__restrict__ normals, DenCfg c,
                  const uint32_t *__restrict__ blk, const uint32_t *__restrict__ n_out) {
    pdl_entry();
    __shared__ uint32_t s_w[kDenThreads / 32];
    uint32_t base[3] = {blk[3 * (size_t)blockIdx.x], blk[3 * (size_t)blockIdx.x + 1], blk[3 * (size_t)blockIdx.x + 2]};
    const uint32_t clone0 = n_out[1], child0 = n_out[2];
    for (int j = 0; j < kDenItems; ++j) {
        const int i = blockIdx.x * kDenTile + j * kDenThreads + threadIdx.x;
        Flags f{false, false, false};
        if (i < n) f = classify(i, io.in.scales, io.in.opacities, accum, count, max_radius, c);
        uint32_t tot;
        const uint32_t ex = block_scan_packed<kDenThreads>(pack(f), s_w, tot);
        if (f.surv) emit(io, i, (int)(base[0] + (ex & 1023u)), true);
        if (f.clone) emit(io, i, (int)(clone0 + base[1] + ((ex >> 10) & 1023u)), false);
        if (f.split) {
            const int row = (int)(child0 + 2 * (base[2] + (ex >> 20)));
            // rotation of the normalised quaternion (w, x, y, z)
            const float4 q = reinterpret_cast<const float4 *>(io.in.quats)[i];
            const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
            const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
            const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                                   {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                                   {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
            const float s[3] = {io.in.scales[3 * (size_t)i], io.in.scales[3 * (size_t)i + 1],
                                io.in.scales[3 * (size_t)i + 2]};
            for (int ch = 0; ch < 2; ++ch) {
                const int r = row + ch;
                emit(io, i, r, false);
                const float *zz = normals + (size_t)6 * i + 3 * ch;
                const float v[3] = {s[0] * zz[0], s[1] * zz[1], s[2] * zz[2]};
                for (int a = 0; a < 3; ++a) {
                    io.out.means[3 * (size_t)r + a] =
                        io.in.means[3 * (size_t)i + a] + (R[a][0] * v[0] + R[a][1] * v[1] + R[a][2] * v[2]);
                    const float ls = __fsub_rn(io.in.log_scales[3 * (size_t)i + a], c.log_div);
                    io.out.log_scales[3 * (size_t)r + a] = ls;
                    io.out.scales[3 * (size_t)r + a] = expf(ls);
                }
            }
        }
        base[0] += tot & 1023u;
        base[1] += (tot >> 10) & 1023u;
        base[2] += tot >> 20;
    }
}

__global__ void __launch_bounds__(256)
k_reset_opacity(int n, float cap, float *__restrict__ logits, float *__restrict__ opac) {
    pdl_entry();
    const int i = blockIdx.x * 256 + threadIdx.x;
    if (i >= n) return;
    const float l = fminf(logits[i], cap);
    logits[i] = l;
    opac[i] = 1.0f / (1.0f + expf(-l));
}

}  // namespace

size_t densify_workspace_bytes(int n) {
    const size_t nb = ((size_t)n + kDenTile - 1) / kDenTile;
    return 256 + ((3 * nb * 4 + 255) & ~(size_t)255) + 256;
}

cudaError_t launch_densify_stats(const float *grad2d, const int *radius, int n, int W, int H, float *accum,
                                 float *count, int *max_radius, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    launch_k(k_densify_stats, (n + 255) / 256, 256, 0, st, reinterpret_cast<const float4 *>(grad2d), radius, n, 0.5f * W,
             0.5f * H, accum, count, max_radius);
    return cudaGetLastError();
}

cudaError_t launch_densify(const darb_train_params &in, const darb_adam_state &sin, const float *accum,
                           const float *count, const int *max_radius, const float *normals,
                           const darb_densify_cfg &cfg, void *workspace, const darb_train_params &out,
                           const darb_adam_state &sout, uint32_t *n_out, cudaStream_t st) {
    const int n = in.n;
    unsigned char *w = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(workspace) + 255) &
                                                         ~(uintptr_t)255);
    uint32_t *blk = reinterpret_cast<uint32_t *>(w + 256);
    const int nb = (n + kDenTile - 1) / kDenTile;
    DenCfg c{cfg.grad_threshold, cfg.dense_scale, cfg.min_opacity, cfg.max_screen_radius, cfg.max_world_scale,
             cfg.split_scale_div, (float)std::log((double)cfg.split_scale_div)};
    if (nb == 0) return cudaMemsetAsync(n_out, 0, 3 * sizeof(uint32_t), st);
    launch_k(k_densify_count, nb, kDenThreads, 0, st, n, in.scales, in.opacities, accum, count, max_radius, c, blk);
    launch_k(k_densify_offsets, 1, 1024, 0, st, nb, blk, n_out);
    DenIO io{in, out, sin, sout, 3 * (in.sh_degree + 1) * (in.sh_degree + 1)};
    launch_k(k_densify_scatter, nb, kDenThreads, 0, st, n, io, accum, count, max_radius, normals, c, blk, n_out);
    return cudaGetLastError();
}

cudaError_t launch_reset_opacity(const darb_train_params &p, float max_opacity, cudaStream_t st) {
    if (p.n == 0) return cudaSuccess;
    const float cap = (float)std::log((double)max_opacity / (1.0 - (double)max_opacity));
    launch_k(k_reset_opacity, (p.n + 255) / 256, 256, 0, st, p.n, cap, p.opacity_logits, p.opacities);
    return cudaGetLastError();
}

}  // namespace darb
