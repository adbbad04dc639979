// The paper's image loss (Sec. 4.2): L = (1 - lambda) L1 + lambda (1 - SSIM), with the SSIM of
// the 3DGS work it builds on -- per channel, an 11 x 11 Gaussian window (sigma 1.5, normalised)
// over zero-padded images, C1 = 0.01^2, C2 = 0.03^2 -- averaged over channels and pixels.
//
// Two tiled kernels, each CTA one 32 x 32 output tile of one channel with a 5-pixel halo; every
// separable blur pass gives each thread 4 consecutive outputs, so an input value is read from
// shared memory once for all the outputs it reaches:
//   k_ssim_fwd  stages x and y, blurs the five moments (x, y, x^2, y^2, xy) with separable
//               passes in shared memory, and writes per pixel the partial derivatives of SSIM
//               w.r.t. the local moments m_x, s_xx, s_xy, plus the block sums of SSIM and |x - y|;
//   k_ssim_bwd  blurs those three maps (the window is symmetric, so the blur is its own adjoint)
//               and forms dL/dx = (1 - lambda) sign(x - y) / N - lambda (G*d_m + 2x G*d_sxx +
//               y G*d_sxy) / N, N = 3HW; its first CTA also writes the loss.
// With A1 = 2 m_x m_y + C1, A2 = 2 (s_xy - m_x m_y) + C2, B1 = m_x^2 + m_y^2 + C1,
// B2 = s_xx - m_x^2 + s_yy - m_y^2 + C2 and SSIM = A1 A2 / (B1 B2):
//   d_m = 2 m_y (A2 - A1) / (B1 B2) - 2 m_x SSIM (1/B1 - 1/B2),  d_sxx = -SSIM / B2,
//   d_sxy = 2 A1 / (B1 B2).
#include "kernels.cuh"

namespace darb {
namespace {

constexpr int kSsimR = 5;
constexpr int kSsimTs = 32;
constexpr int kSsimIn = kSsimTs + 2 * kSsimR;  // 42
constexpr int kSsimThreads = 256;
constexpr int kSsimRb = 4;  // outputs per thread along the blur direction (register blocking)
constexpr int kSsimTaps = 2 * kSsimR + 1;
constexpr float kSsimC1 = 0.01f * 0.01f;
constexpr float kSsimC2 = 0.03f * 0.03f;
constexpr int kStage = (kSsimIn * kSsimIn + kSsimThreads - 1) / kSsimThreads;  // halo elements per thread
// Resident CTAs per SM both kernels are compiled for (0: the compiler's register count).
#ifndef DARB_SSIM_MIN_CTAS
#define DARB_SSIM_MIN_CTAS 0
#endif
#if DARB_SSIM_MIN_CTAS > 0
#define DARB_SSIM_BOUNDS __launch_bounds__(kSsimThreads, DARB_SSIM_MIN_CTAS)
#else
#define DARB_SSIM_BOUNDS __launch_bounds__(kSsimThreads)
#endif
static_assert(kSsimTs % kSsimRb == 0 && (kSsimTs / kSsimRb) * kSsimTs == kSsimThreads, "one vertical group per thread");

struct Window {
    float g[kSsimTaps];
};

Window make_window() {
    Window w;
    double sum = 0.0, v[kSsimTaps];
    for (int k = -kSsimR; k <= kSsimR; ++k) {
        v[k + kSsimR] = std::exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
        sum += v[k + kSsimR];
    }
    for (int k = 0; k < kSsimTaps; ++k) w.g[k] = (float)(v[k] / sum);
    return w;
}

__device__ __forceinline__ float block_sum(float v, float *s_w) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
    __syncthreads();
    float t = 0.0f;
    if (threadIdx.x == 0)
        for (int i = 0; i < kSsimThreads / 32; ++i) t += s_w[i];
    return t;  // valid on thread 0
}

// Blurs along a row: out[i] = sum_k g[k] in[c0 + i + k] for kSsimRb consecutive outputs, each
// sum taken in tap order (the same order as one output at a time).
template <int NQ, class In>
__device__ __forceinline__ void hblur(const Window &win, In in, float (&out)[NQ][kSsimRb]) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
        for (int i = 0; i < kSsimRb; ++i) out[q][i] = 0.0f;
#pragma unroll
    for (int t = 0; t < kSsimRb + kSsimTaps - 1; ++t) {  // each input once, into every output it reaches
        float val[NQ];
        in(t, val);
#pragma unroll
        for (int i = 0; i < kSsimRb; ++i) {
            const int k = t - i;
            if (k >= 0 && k < kSsimTaps)
#pragma unroll
                for (int q = 0; q < NQ; ++q) out[q][i] = fmaf(win.g[k], val[q], out[q][i]);
        }
    }
}

// Forward: the five local moments by separable blurs (x along rows, then y along columns, each
// thread kSsimRb consecutive outputs), then the derivative maps and the block sums.
__global__ void DARB_SSIM_BOUNDS
k_ssim_fwd(const float *__restrict__ x, const float *__restrict__ y, int W, int H, Window win,
           float *__restrict__ d_m, float *__restrict__ d_sxx, float *__restrict__ d_sxy, double *__restrict__ sums) {
    pdl_entry();
    __shared__ float sx[kSsimIn][kSsimIn + 1], sy[kSsimIn][kSsimIn + 1];
    __shared__ float h[5][kSsimIn][kSsimTs + 1];  // padded: a warp's row-pass stores hit 32 banks
    __shared__ float s_w[kSsimThreads / 32];
    const int x0 = blockIdx.x * kSsimTs, y0 = blockIdx.y * kSsimTs;
    const size_t plane = (size_t)W * H, off = (size_t)blockIdx.z * plane;
    {  // every load of the halo tile issued before the first store
        float vx[kStage], vy[kStage];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int i = threadIdx.x + u * kSsimThreads;
            const int r = i / kSsimIn, c = i - r * kSsimIn;
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
            const bool in = i < kSsimIn * kSsimIn && gx >= 0 && gx < W && gy >= 0 && gy < H;
            vx[u] = in ? x[off + (size_t)gy * W + gx] : 0.0f;
            vy[u] = in ? y[off + (size_t)gy * W + gx] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int i = threadIdx.x + u * kSsimThreads;
            if (i < kSsimIn * kSsimIn) {
                const int r = i / kSsimIn, c = i - r * kSsimIn;
                sx[r][c] = vx[u];
                sy[r][c] = vy[u];
            }
        }
    }
    __syncthreads();
    // along x: item = (row, group of kSsimRb columns)
    constexpr int kGroups = kSsimTs / kSsimRb;
    for (int item = threadIdx.x; item < kSsimIn * kGroups; item += kSsimThreads) {
        const int r = item / kGroups, c0 = (item - r * kGroups) * kSsimRb;
        float o[5][kSsimRb];
        hblur<5>(win, [&](int t, float (&val)[5]) {
            const float u = sx[r][c0 + t], v = sy[r][c0 + t];
            val[0] = u;
            val[1] = v;
            val[2] = u * u;
            val[3] = v * v;
            val[4] = u * v;
        }, o);
#pragma unroll
        for (int q = 0; q < 5; ++q)
#pragma unroll
            for (int i = 0; i < kSsimRb; ++i) h[q][r][c0 + i] = o[q][i];
    }
    __syncthreads();
    // along y: thread = (column, group of kSsimRb rows)
    const int c = threadIdx.x % kSsimTs, r0 = (threadIdx.x / kSsimTs) * kSsimRb;
    float m[5][kSsimRb];
    hblur<5>(win, [&](int t, float (&val)[5]) {
#pragma unroll
        for (int q = 0; q < 5; ++q) val[q] = h[q][r0 + t][c];
    }, m);
    float ssim_sum = 0.0f, l1_sum = 0.0f;
#pragma unroll
    for (int i = 0; i < kSsimRb; ++i) {
        const int r = r0 + i, gy = y0 + r, gx = x0 + c;
        if (gx >= W || gy >= H) continue;
        const float mx = m[0][i], my = m[1][i];
        const float A1 = 2.0f * mx * my + kSsimC1;
        const float A2 = 2.0f * (m[4][i] - mx * my) + kSsimC2;
        const float B1 = mx * mx + my * my + kSsimC1;
        const float B2 = (m[2][i] - mx * mx) + (m[3][i] - my * my) + kSsimC2;
        const float iB1 = __frcp_rn(B1), iB2 = __frcp_rn(B2);  // two reciprocals, no division
        const float iB = iB1 * iB2;
        const float sv = A1 * A2 * iB;
        const size_t p = off + (size_t)gy * W + gx;
        d_m[p] = 2.0f * my * (A2 - A1) * iB - 2.0f * mx * sv * (iB1 - iB2);
        d_sxx[p] = -sv * iB2;
        d_sxy[p] = 2.0f * A1 * iB;
        ssim_sum += sv;
        l1_sum += fabsf(sx[r + kSsimR][c + kSsimR] - sy[r + kSsimR][c + kSsimR]);
    }
    const float ts = block_sum(ssim_sum, s_w);
    __syncthreads();
    const float tl = block_sum(l1_sum, s_w);
    if (threadIdx.x == 0) {
        atomicAdd(&sums[0], (double)ts);
        atomicAdd(&sums[1], (double)tl);
    }
}

// Backward: blurs the three derivative maps (the window is symmetric, so the blur is its own
// adjoint) with the same blocking, then forms dL/dx.
__global__ void DARB_SSIM_BOUNDS
k_ssim_bwd(const float *__restrict__ x, const float *__restrict__ y, int W, int H, Window win,
           const float *__restrict__ d_m, const float *__restrict__ d_sxx, const float *__restrict__ d_sxy,
           float lam, const double *__restrict__ sums, float *__restrict__ dL, float *__restrict__ loss) {
    pdl_entry();
    __shared__ float sa[3][kSsimIn][kSsimIn + 1];
    __shared__ float h[3][kSsimIn][kSsimTs + 1];
    const int x0 = blockIdx.x * kSsimTs, y0 = blockIdx.y * kSsimTs;
    const size_t plane = (size_t)W * H, off = (size_t)blockIdx.z * plane;
    const double n = 3.0 * (double)plane;
    const float inv_n = (float)(1.0 / n);
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0) {
        const double ssim = sums[0] / n, l1 = sums[1] / n;
        loss[0] = (float)((1.0 - lam) * l1 + lam * (1.0 - ssim));
        loss[1] = (float)ssim;
    }
    {  // every load of the three halo tiles issued before the first store
        float va[kStage][3];
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int i = threadIdx.x + u * kSsimThreads;
            const int r = i / kSsimIn, c = i - r * kSsimIn;
            const int gy = y0 - kSsimR + r, gx = x0 - kSsimR + c;
            const bool in = i < kSsimIn * kSsimIn && gx >= 0 && gx < W && gy >= 0 && gy < H;
            const size_t p = off + (size_t)gy * W + gx;
            va[u][0] = in ? d_m[p] : 0.0f;
            va[u][1] = in ? d_sxx[p] : 0.0f;
            va[u][2] = in ? d_sxy[p] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kStage; ++u) {
            const int i = threadIdx.x + u * kSsimThreads;
            if (i < kSsimIn * kSsimIn) {
                const int r = i / kSsimIn, c = i - r * kSsimIn;
#pragma unroll
                for (int q = 0; q < 3; ++q) sa[q][r][c] = va[u][q];
            }
        }
    }
    __syncthreads();
    constexpr int kGroups = kSsimTs / kSsimRb;
    for (int item = threadIdx.x; item < kSsimIn * kGroups; item += kSsimThreads) {
        const int r = item / kGroups, c0 = (item - r * kGroups) * kSsimRb;
        float o[3][kSsimRb];
        hblur<3>(win, [&](int t, float (&val)[3]) {
#pragma unroll
            for (int q = 0; q < 3; ++q) val[q] = sa[q][r][c0 + t];
        }, o);
#pragma unroll
        for (int q = 0; q < 3; ++q)
#pragma unroll
            for (int i = 0; i < kSsimRb; ++i) h[q][r][c0 + i] = o[q][i];
    }
    __syncthreads();
    const int c = threadIdx.x % kSsimTs, r0 = (threadIdx.x / kSsimTs) * kSsimRb;
    float b[3][kSsimRb];
    hblur<3>(win, [&](int t, float (&val)[3]) {
#pragma unroll
        for (int q = 0; q < 3; ++q) val[q] = h[q][r0 + t][c];
    }, b);
#pragma unroll
    for (int i = 0; i < kSsimRb; ++i) {
        const int gy = y0 + r0 + i, gx = x0 + c;
        if (gx >= W || gy >= H) continue;
        const size_t p = off + (size_t)gy * W + gx;
        const float xv = x[p], yv = y[p], d = xv - yv;
        const float sgn = d > 0.0f ? 1.0f : (d < 0.0f ? -1.0f : 0.0f);
        const float dssim = (b[0][i] + 2.0f * xv * b[1][i] + yv * b[2][i]) * inv_n;
        dL[p] = (1.0f - lam) * sgn * inv_n - lam * dssim;
    }
}

}  // namespace

size_t l1_dssim_workspace_bytes(int W, int H) {
    const size_t maps = 3 * (size_t)3 * W * H * sizeof(float);
    return 256 + ((maps + 255) & ~(size_t)255) + 256;
}

cudaError_t launch_l1_dssim(const float *image, const float *target, int W, int H, float lam, void *workspace,
                            float *dL, float *loss, cudaStream_t st) {
    unsigned char *w = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(workspace) + 255) &
                                                         ~(uintptr_t)255);
    double *sums = reinterpret_cast<double *>(w);
    float *maps = reinterpret_cast<float *>(w + 256);
    const size_t n = (size_t)3 * W * H;
    cudaError_t e = launch_zero(st, sums, 2 * sizeof(double));
    if (e != cudaSuccess) return e;
    static const Window win = make_window();
    const dim3 grid((W + kSsimTs - 1) / kSsimTs, (H + kSsimTs - 1) / kSsimTs, 3);
    launch_k(k_ssim_fwd, grid, kSsimThreads, 0, st, image, target, W, H, win, maps, maps + n, maps + 2 * n, sums);
    launch_k(k_ssim_bwd, grid, kSsimThreads, 0, st, image, target, W, H, win, maps, maps + n, maps + 2 * n, lam, sums, dL,
             loss);
    return cudaGetLastError();
}

}  // namespace darb
