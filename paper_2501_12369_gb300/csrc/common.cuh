// Shared device helpers of libdarb.so (GB300, sm_103a).
#pragma once

#include <cmath>
#include <cstdint>
#include <cuda_runtime.h>

#include "darb.h"

namespace darb {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  Every kernel of the library is launched through launch_k,
// which lets it be scheduled while its predecessor in the stream drains, and starts with
// pdl_entry(): wait until the predecessor grid has completed and its writes are visible (a
// no-op without a programmatic predecessor), then allow the successor to be scheduled.  Only
// the launch latency and the CTA start-up overlap; no kernel touches memory before the wait.
// DARB_PDL=0 in the environment launches without the attribute.
__device__ __forceinline__ void pdl_entry() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

bool pdl_enabled();  // read once from DARB_PDL (default on)

template <typename... P, typename... A>
inline void launch_k(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    // a launch error is also left for cudaGetLastError, which every caller checks
    (void)cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}

// SMs of a GB300 (2 dies x 76): the cap of the grid-stride launches is a multiple of it.
constexpr int kGridSms = 152;

constexpr float kAlphaMax = 0.99f;          // 3DGS alpha clamp (listings: min(0.99f, ...))
constexpr float kAlphaMin = 1.0f / 255.0f;  // 3DGS: skip alpha < 1/255
constexpr float kTMin = 0.0001f;            // 3DGS: stop before T (1 - alpha) < 1e-4
constexpr float kDilation = 0.3f;           // low-pass filter added to the 2D covariance
constexpr float kGuardBand = 1.3f;          // Jacobian clamp at 1.3 tan(fov/2)
constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;

constexpr int kNumKernels = 8;  // the seven fixed kernels and DARB_GENERIC

// Camera as passed by value to kernels.
struct Cam {
    float V[16];
    float fx, fy, cx, cy, near_plane;
    int W, H;
    float bg[3];
    float campos[3];  // -R^T t, for the SH viewing direction
    // the Jacobian's guard band, kGuardBand * W / (2 fx) and * H / (2 fy): the same FP32
    // operations a splat would take, done once per camera
    float limx, limy;
};

inline Cam make_cam(const darb_camera &c) {
    Cam k;
    for (int i = 0; i < 16; ++i) k.V[i] = c.viewmat[i];
    k.fx = c.fx; k.fy = c.fy; k.cx = c.cx; k.cy = c.cy; k.near_plane = c.near_plane;
    k.W = c.width; k.H = c.height;
    for (int i = 0; i < 3; ++i) k.bg[i] = c.bg[i];
    for (int j = 0; j < 3; ++j) {
        double s = 0.0;
        for (int r = 0; r < 3; ++r) s -= (double)c.viewmat[4 * r + j] * (double)c.viewmat[4 * r + 3];
        k.campos[j] = (float)s;
    }
    // IEEE FP32 on the host as on the device: 2 fx is exact, then one rounded division and one
    // rounded product (no contraction applies)
    const float tx2 = 2.0f * c.fx, ty2 = 2.0f * c.fy;
    const float qx = (float)c.width / tx2, qy = (float)c.height / ty2;
    k.limx = kGuardBand * qx;
    k.limy = kGuardBand * qy;
    return k;
}

// ---------------------------------------------------------------------------
// Kernel profiles F(q) and dF/dq in FP32 (Table 1 with the xi of Table 2 in the forms the
// Sec. B listings evaluate).  Every main-lobe argument is bounded (cos on [0, pi/2] or
// [0, pi], exp on [-4.5, 0]), so the hardware approximations (__cosf, __expf, __sincosf:
// absolute error below 4e-7 there) are accurate enough; the sinc uses its Taylor series in
// x^2 to the x^14 term (truncation error below 3e-7 on [0, pi]).
// kernel_F is written with explicit intrinsics so that its rounding never depends on how the
// compiler contracts the surrounding code: forward and backward must get the same alpha.

// Parameters of the generic member (kind DARB_GENERIC): F = base(u), u = q^(beta/2) / xi.
struct KernelSpec {
    int base;         // 0 exp(-u), 1 cos u, 2 1/2 + 1/2 cos u, 3 |sin u| / u, 4 (u + 1)^(-1/2), 5 1 - u
    float inv_xi;     // 1 / xi
    float half_beta;  // beta / 2
};

inline KernelSpec make_spec(const darb_kernel_params &k) {
    KernelSpec s;
    s.base = k.base;
    s.inv_xi = k.xi > 0.0f ? 1.0f / k.xi : 0.0f;
    s.half_beta = 0.5f * k.beta;
    return s;
}

template <int K> __device__ __forceinline__ float kernel_F(float q, const KernelSpec &ks);
template <int K> __device__ __forceinline__ float kernel_dF(float q, const KernelSpec &ks);

// sin(x)/x = 1 - u/3! + u^2/5! - ... - u^7/15! with u = x^2, evaluated by Horner as
// 1 - u (1/3! - u (1/5! - u (1/7! - u (1/9! - u (1/11! - u (1/13! - u/15!)))))).
__device__ __forceinline__ float sinc_series(float u) {
    float r = __fmaf_rn(u, 1.0f / 1307674368000.0f, -1.0f / 6227020800.0f);  // -(1/13! - u/15!)
    r = __fmaf_rn(r, u, 1.0f / 39916800.0f);   // 1/11! - u(...)
    r = __fmaf_rn(r, u, -1.0f / 362880.0f);    // -(1/9! - u(...))
    r = __fmaf_rn(r, u, 1.0f / 5040.0f);       // 1/7! - u(...)
    r = __fmaf_rn(r, u, -1.0f / 120.0f);       // -(1/5! - u(...))
    r = __fmaf_rn(r, u, 1.0f / 6.0f);          // 1/3! - u(...)
    return __fmaf_rn(r, -u, 1.0f);
}

template <> __device__ __forceinline__ float kernel_F<DARB_GAUSSIAN>(float q, const KernelSpec &) {
    return __expf(__fmul_rn(-0.5f, q));
}
template <> __device__ __forceinline__ float kernel_dF<DARB_GAUSSIAN>(float q, const KernelSpec &) { return -0.5f * __expf(-0.5f * q); }

template <> __device__ __forceinline__ float kernel_F<DARB_HALF_COSINE>(float q, const KernelSpec &) {
    return __cosf(__fmul_rn(q, kPi / 18.0f));
}
template <> __device__ __forceinline__ float kernel_dF<DARB_HALF_COSINE>(float q, const KernelSpec &) {
    return -(kPi / 18.0f) * __sinf(q * (kPi / 18.0f));
}

template <> __device__ __forceinline__ float kernel_F<DARB_RAISED_COSINE>(float q, const KernelSpec &) {
    return __fmaf_rn(0.5f, __cosf(__fmul_rn(__fsqrt_rn(q), kPi / 2.5f)), 0.5f);
}
template <> __device__ __forceinline__ float kernel_dF<DARB_RAISED_COSINE>(float q, const KernelSpec &) {
    // -(k/4) sin(k sqrt q) / sqrt q, k = pi/2.5; limit -k^2/4 at q = 0.
    constexpr float k = kPi / 2.5f;
    if (q < 1e-6f) return -0.25f * k * k + (k * k * k * k / 24.0f) * q;
    const float r = sqrtf(q);
    return -0.25f * k * __sinf(k * r) / r;
}

template <> __device__ __forceinline__ float kernel_F<DARB_MOD_SINC>(float q, const KernelSpec &) {
    // x = pi sqrt(q) / 3, so x^2 = (pi^2 / 9) q; sin(x)/x >= 0 on the main lobe
    return fmaxf(sinc_series(__fmul_rn(q, kPi * kPi / 9.0f)), 0.0f);
}
template <> __device__ __forceinline__ float kernel_dF<DARB_MOD_SINC>(float q, const KernelSpec &) {
    // (x cos x - sin x) / (2 q x), x = pi sqrt(q)/3; series below x = 0.3.
    const float x = sqrtf(q) * (kPi / 3.0f);
    if (x < 0.3f) {
        constexpr float a = kPi * kPi / 9.0f;  // x^2 = a q
        return -a / 6.0f + (a * a / 60.0f) * q - (a * a * a / 1680.0f) * q * q +
               (a * a * a * a / 90720.0f) * q * q * q;
    }
    float s, c;
    __sincosf(x, &s, &c);
    return (x * c - s) / (2.0f * q * x);
}

template <> __device__ __forceinline__ float kernel_F<DARB_INV_QUADRIC>(float q, const KernelSpec &) {
    return __fdividef(1.0f, __fadd_rn(1.0f, q));
}
template <> __device__ __forceinline__ float kernel_dF<DARB_INV_QUADRIC>(float q, const KernelSpec &) {
    const float r = __fdividef(1.0f, 1.0f + q);
    return -r * r;
}

template <> __device__ __forceinline__ float kernel_F<DARB_INV_MULTIQUADRIC>(float q, const KernelSpec &) {
    return rsqrtf(__fadd_rn(1.0f, q));
}
template <> __device__ __forceinline__ float kernel_dF<DARB_INV_MULTIQUADRIC>(float q, const KernelSpec &) {
    const float r = rsqrtf(1.0f + q);
    return -0.5f * r * r * r;
}

template <> __device__ __forceinline__ float kernel_F<DARB_PARABOLA>(float q, const KernelSpec &) {
    return __fmaf_rn(q, -1.0f / 9.0f, 1.0f);
}
template <> __device__ __forceinline__ float kernel_dF<DARB_PARABOLA>(float, const KernelSpec &) { return -1.0f / 9.0f; }

// The generic member.  u = q / xi exactly when beta = 2, sqrt(q) / xi when beta = 1, else
// __powf (a few ulp).  The cosines use the hardware approximation on the main lobe and the
// accurate routine beyond pi; the sinc its series on [0, pi].
__device__ __forceinline__ float generic_u(float q, const KernelSpec &ks) {
    if (ks.half_beta == 1.0f) return __fmul_rn(q, ks.inv_xi);
    if (!(q > 0.0f)) return 0.0f;
    if (ks.half_beta == 0.5f) return __fmul_rn(__fsqrt_rn(q), ks.inv_xi);
    return __fmul_rn(__powf(q, ks.half_beta), ks.inv_xi);
}

__device__ __forceinline__ float generic_base(int base, float u) {
    switch (base) {
    case 0: return __expf(-u);
    case 1: return __cosf(u);
    case 2: return __fmaf_rn(0.5f, u <= kPi ? __cosf(u) : cosf(u), 0.5f);
    case 3: return u <= kPi ? fmaxf(sinc_series(__fmul_rn(u, u)), 0.0f) : fabsf(sinf(u)) / u;
    case 4: return rsqrtf(__fadd_rn(u, 1.0f));
    default: return __fadd_rn(1.0f, -u);
    }
}

__device__ __forceinline__ float generic_base_du(int base, float u) {
    switch (base) {
    case 0: return -__expf(-u);
    case 1: return -__sinf(u);
    case 2: return -0.5f * (u <= kPi ? __sinf(u) : sinf(u));
    case 3: {
        if (u < 1e-3f) return -u * (1.0f / 3.0f);
        float sn, cs;
        if (u <= kPi) __sincosf(u, &sn, &cs);
        else sincosf(u, &sn, &cs);
        const float d = (u * cs - sn) / (u * u);
        return sn < 0.0f ? -d : d;
    }
    case 4: {
        const float r = rsqrtf(u + 1.0f);
        return -0.5f * r * r * r;
    }
    default: return -1.0f;
    }
}

template <> __device__ __forceinline__ float kernel_F<DARB_GENERIC>(float q, const KernelSpec &ks) {
    return generic_base(ks.base, generic_u(q, ks));
}
template <> __device__ __forceinline__ float kernel_dF<DARB_GENERIC>(float q, const KernelSpec &ks) {
    if (ks.half_beta == 1.0f) return generic_base_du(ks.base, q * ks.inv_xi) * ks.inv_xi;
    const float qq = fmaxf(q, 1e-30f);  // one-sided limit at the centre (finite for beta >= 1 on cosines)
    const float u = generic_u(qq, ks);
    return generic_base_du(ks.base, u) * ks.half_beta * u / qq;
}

// ---------------------------------------------------------------------------
// Tile membership: per row of tiles, the run [c0, c1] that the x-extent of the splat's ellipse
// {q <= q_max} over the row's band of pixel-centre heights reaches -- the ellipse's leftmost and
// rightmost points clamped to the band -- inside the rectangle r.  Every pixel centre with
// q <= q_max lies in a member tile.  Fixed IEEE FP32 sequence (no contraction): the oracle
// takes the same operations, so both sides build the same lists.
struct SpanCtx {
    float qmax;
    int tile, W, H;
    int shift;  // log2(tile): tiles are 8, 16 or 32 pixels
};

__host__ __device__ inline SpanCtx make_span_ctx(float qmax, int tile, int W, int H) {
    int shift = 0;
    while ((1 << shift) < tile) ++shift;
    return SpanCtx{qmax, tile, W, H, shift};
}

// Per-splat part of the sequence: the ellipse's extents, 1/A and its leftmost / rightmost x
// offsets at the unclamped extreme heights (rows whose band contains an extreme reuse them).
// At the height dyR0 = -B xm / C of its rightmost point the ellipse's x-extent is exactly xm
// (substitute dyR0 into the root below), so rR = xm and rL = -xm.
struct SpanSplat {
    float u0, u1, nB, det, ym, dyR0, dyL0, aq, invA, rR, rL;
    bool ok;
};

__device__ __forceinline__ SpanSplat span_prepare(float u0, float u1, float A, float B, float C, float qm) {
    SpanSplat p;
    p.u0 = u0;
    p.u1 = u1;
    p.det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    p.ok = p.det > 0.0f;
    const float xm = __fsqrt_rn(__fdiv_rn(__fmul_rn(qm, C), p.det));
    p.ym = __fsqrt_rn(__fdiv_rn(__fmul_rn(qm, A), p.det));
    p.nB = -B;
    p.dyR0 = __fdiv_rn(__fmul_rn(p.nB, xm), C);
    p.dyL0 = -p.dyR0;
    p.aq = __fmul_rn(A, qm);
    p.invA = __fdiv_rn(1.0f, A);
    p.rR = xm;
    p.rL = -xm;
    return p;
}

__device__ __forceinline__ bool span_row(const SpanSplat &p, const SpanCtx &sc, const int4 &r, int ty, int &c0,
                                         int &c1) {
    if (!p.ok) return false;
    const float ya = __fadd_rn((float)(ty << sc.shift), 0.5f);
    const float yb = fminf(__fsub_rn((float)((ty + 1) << sc.shift), 0.5f), __fsub_rn((float)sc.H, 0.5f));
    const float ea = fmaxf(__fsub_rn(ya, p.u1), -p.ym), eb = fminf(__fsub_rn(yb, p.u1), p.ym);
    if (!(ea <= eb)) return false;
    const float dyR = fminf(fmaxf(p.dyR0, ea), eb), dyL = fminf(fmaxf(p.dyL0, ea), eb);
    const float right =
        dyR == p.dyR0
            ? p.rR
            : __fmul_rn(__fadd_rn(__fmul_rn(p.nB, dyR),
                                  __fsqrt_rn(fmaxf(__fsub_rn(p.aq, __fmul_rn(p.det, __fmul_rn(dyR, dyR))), 0.0f))),
                        p.invA);
    const float left =
        dyL == p.dyL0
            ? p.rL
            : __fmul_rn(__fsub_rn(__fmul_rn(p.nB, dyL),
                                  __fsqrt_rn(fmaxf(__fsub_rn(p.aq, __fmul_rn(p.det, __fmul_rn(dyL, dyL))), 0.0f))),
                        p.invA);
    const float i0 = fmaxf(ceilf(__fsub_rn(__fadd_rn(p.u0, left), 0.5f)), 0.0f);
    const float i1 = fminf(floorf(__fsub_rn(__fadd_rn(p.u0, right), 0.5f)), (float)(sc.W - 1));
    if (!(i0 <= i1)) return false;
    c0 = max((int)i0 >> sc.shift, r.x);  // i0, i1 >= 0
    c1 = min((int)i1 >> sc.shift, r.z);
    return c0 <= c1;
}

// The runs packed per splat (tile_runs): for a rectangle of at most 8 rows and 15 columns,
// byte k holds row r.y + k's run as (c1 - r.x) << 4 | (c0 - r.x), 0x0F for a row without
// member tiles (c0 > c1 once unpacked); kRunsUnpacked otherwise.
constexpr uint64_t kRunsUnpacked = ~0ull;
constexpr uint64_t kRunsNone = 0x0f0f0f0f0f0f0f0full;  // eight empty rows
constexpr int kRunsRows = 8;

__device__ __forceinline__ bool runs_packable(const int4 &r) { return r.w - r.y < kRunsRows && r.z - r.x < 15; }

__device__ __forceinline__ uint64_t runs_put(uint64_t pk, const int4 &r, int ty, int c0, int c1) {
    const int sh = 8 * (ty - r.y);
    return (pk & ~(0xffull << sh)) | ((uint64_t)((c1 - r.x) << 4 | (c0 - r.x)) << sh);
}

// Calls f(ty, c0, c1) for the run of every tile row of r that has member tiles, top to bottom,
// until f returns false, from the packed word pk (not kRunsUnpacked).
template <typename F>
__device__ __forceinline__ void for_each_packed_run(uint64_t pk, const int4 &r, F &&f) {
    for (int ty = r.y; ty <= r.w; ++ty) {
        const uint32_t b = (uint32_t)(pk >> (8 * (ty - r.y))) & 0xffu;
        const int c0 = r.x + (int)(b & 15u), c1 = r.x + (int)(b >> 4);
        if (c0 <= c1 && !f(ty, c0, c1)) return;
    }
}

// Calls f(ty, c0, c1) for the run of every tile row of r that has member tiles, top to bottom,
// until f returns false: unpacked from pk, or computed from splat id's ellipse when pk is
// kRunsUnpacked.
template <typename F>
__device__ __forceinline__ void for_each_run(uint64_t pk, const float2 *__restrict__ mean2d,
                                             const float4 *__restrict__ conic_o, uint32_t id, const int4 &r,
                                             const SpanCtx &sc, F &&f) {
    if (pk != kRunsUnpacked) {
        for_each_packed_run(pk, r, f);
        return;
    }
    const float2 mu = __ldg(mean2d + id);
    const float4 co = __ldg(conic_o + id);
    const SpanSplat p = span_prepare(mu.x, mu.y, co.x, co.y, co.z, sc.qmax);
    for (int ty = r.y; ty <= r.w; ++ty) {
        int c0, c1;
        if (span_row(p, sc, r, ty, c0, c1) && !f(ty, c0, c1)) return;
    }
}

// The runs of one splat computed by the whole warp (every lane passes the same splat): lane l
// takes rows r.y + l, r.y + l + 32, ... and calls f(ty, c0, c1, before) for its row when the
// row has member tiles, `before` being the member tiles of the splat's rows above it.  Returns
// the splat's member-tile count to every lane.
template <typename F>
__device__ __forceinline__ uint32_t warp_runs(float u0, float u1, float A, float B, float C, const int4 &r,
                                              const SpanCtx &sc, F &&f) {
    const int lane = threadIdx.x & 31;
    const SpanSplat p = span_prepare(u0, u1, A, B, C, sc.qmax);
    uint32_t carry = 0;
    for (int ty0 = r.y; ty0 <= r.w; ty0 += 32) {
        const int ty = ty0 + lane;
        int c0 = 0, c1 = -1;
        const bool has = ty <= r.w && span_row(p, sc, r, ty, c0, c1);
        const uint32_t w = has ? (uint32_t)(c1 - c0 + 1) : 0u;
        uint32_t x = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (has) f(ty, c0, c1, carry + x - w);
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    return carry;
}

// Member tiles of a splat in row-major order: the tile of its l-th instance (l below its count).
__device__ __forceinline__ uint32_t instance_tile_p(const SpanSplat &p, const int4 &r, uint32_t l, int tiles_x,
                                                    const SpanCtx &sc) {
    for (int ty = r.y; ty <= r.w; ++ty) {
        int c0, c1;
        if (!span_row(p, sc, r, ty, c0, c1)) continue;
        const uint32_t w = (uint32_t)(c1 - c0 + 1);
        if (l < w) return (uint32_t)(ty * tiles_x + c0) + l;
        l -= w;
    }
    return 0xffffffffu;  // unreachable for l below the count
}

__device__ __forceinline__ uint32_t instance_tile(float2 mu, float4 co, const int4 &r, uint32_t l, int tiles_x,
                                                  const SpanCtx &sc) {
    return instance_tile_p(span_prepare(mu.x, mu.y, co.x, co.y, co.z, sc.qmax), r, l, tiles_x, sc);
}

// The support test on q: 0 <= q <= q_max (q < q_max when strict).
__device__ __forceinline__ bool in_support(float q, float qmax, bool strict) {
    return q >= 0.0f && (strict ? q < qmax : q <= qmax);
}

// The same test with the strictness folded into the limit once: for floats, q < q_max exactly
// when q <= the float just below q_max, so in_support(q, qmax, strict) equals
// in_support_lim(q, support_limit(qmax, strict)) for every q (q_max positive and finite, as
// the boundary checks).
__device__ __forceinline__ float support_limit(float qmax, bool strict) {
    return strict ? __uint_as_float(__float_as_uint(qmax) - 1u) : qmax;
}
__device__ __forceinline__ bool in_support_lim(float q, float qlim) { return q >= 0.0f && q <= qlim; }

// q = dx (A dx + 2B dy) + (C dy) dy as a fixed FP32 sequence (no contraction beyond the
// two explicit fused multiply-adds), shared by forward and backward so both take the
// same support decision.  B2 = 2B (exact).
__device__ __forceinline__ float conic_q(float dx, float dy, float A, float B2, float C) {
    const float e = __fmul_rn(B2, dy);
    const float g = __fmaf_rn(A, dx, e);
    const float h = __fmul_rn(__fmul_rn(C, dy), dy);
    return __fmaf_rn(dx, g, h);
}

// ---------------------------------------------------------------------------
// Adam (Kingma & Ba) on one element: m, v moments; bias corrections as reciprocals.

struct AdamConsts {
    float lr_means, lr_scales, lr_quats, lr_opacities, lr_sh_dc, lr_sh_rest;
    float b1, b2, eps, ibc1, ibc2;
};

// The step divides by sqrt(v_hat) + eps with the hardware's approximate square root and
// divide (PTX sqrt.approx.f32, within 2^-23 relative, subnormals kept; __fdividef, 2 ulp for
// divisors below 2^126): a few ulp on an update of order lr, against the IEEE sequences'
// many instructions per element.
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ void adam_apply(float &p, float g, float &m, float &v, float lr, const AdamConsts &c) {
    m = fmaf(c.b1, m, (1.0f - c.b1) * g);
    v = fmaf(c.b2, v, (1.0f - c.b2) * g * g);
    p -= lr * __fdividef(m * c.ibc1, sqrt_approx(v * c.ibc2) + c.eps);
}

inline AdamConsts make_adam_consts(const darb_adam_config &c) {
    AdamConsts a;
    a.lr_means = c.lr_means; a.lr_scales = c.lr_scales; a.lr_quats = c.lr_quats;
    a.lr_opacities = c.lr_opacities; a.lr_sh_dc = c.lr_sh_dc; a.lr_sh_rest = c.lr_sh_rest;
    a.b1 = c.beta1; a.b2 = c.beta2; a.eps = c.eps;
    // bias corrections on the host in double: 1 - beta^t loses digits for beta near 1
    a.ibc1 = (float)(1.0 / (1.0 - std::pow((double)c.beta1, (double)c.step)));
    a.ibc2 = (float)(1.0 / (1.0 - std::pow((double)c.beta2, (double)c.step)));
    return a;
}

// ---------------------------------------------------------------------------
// Host-side helpers.

#define DARB_CUDA_TRY(expr)                                   \
    do {                                                      \
        cudaError_t _e = (expr);                              \
        if (_e != cudaSuccess) return DARB_ERR_CUDA;          \
    } while (0)

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline int tile_count(int extent, int tile) { return (extent + tile - 1) / tile; }

inline int log2_ceil(uint32_t v) {
    int b = 0;
    while ((1ull << b) < v) ++b;
    return b;
}

}  // namespace darb
