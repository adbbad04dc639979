// Step 1 and its backward: per-splat preprocessing (paper Sec. 4.1 "DARB Projection",
// Eq. 2x2covProjection, Table 2; the "cov *= correctionFactor" lines of the Sec. B
// listings).  One thread per splat; HBM-bound.
//
// The geometry (everything that later decides culling, radius, tile rectangle, depth
// order and the per-pixel support test) follows a fixed IEEE FP32 operation sequence
// written with __f*_rn intrinsics, which the compiler neither contracts nor reorders,
// so its results are bit-reproducible.  SH colour and the backward use ordinary FP32.
#include "common.cuh"
#include "kernels.cuh"

namespace darb {

// Real SH basis to degree 3 (3DGS ordering m = -l..l, Condon-Shortley phase).
// Constants: 1/(2 sqrt pi), sqrt(3)/(2 sqrt pi), sqrt(15)/(2 sqrt pi), sqrt(5)/(4 sqrt pi),
// sqrt(15)/(4 sqrt pi), sqrt(35/(2pi))/4, sqrt(105/pi)/2, sqrt(21/(2pi))/4, sqrt(7/pi)/4,
// sqrt(105/pi)/4.
struct SH {
    static constexpr float c0 = 0.28209479177387814f;
    static constexpr float c1 = 0.4886025119029199f;
    static constexpr float c2a = 1.0925484305920792f;
    static constexpr float c2b = 0.31539156525252005f;
    static constexpr float c2c = 0.5462742152960396f;
    static constexpr float c3a = 0.5900435899266435f;
    static constexpr float c3b = 2.890611442640554f;
    static constexpr float c3c = 0.4570457994644658f;
    static constexpr float c3d = 0.3731763325901154f;
    static constexpr float c3e = 1.445305721320277f;
};

template <int DEG>
__device__ __forceinline__ void sh_eval_basis(float x, float y, float z, float *Y) {
    Y[0] = SH::c0;
    if (DEG >= 1) {
        Y[1] = -SH::c1 * y;
        Y[2] = SH::c1 * z;
        Y[3] = -SH::c1 * x;
    }
    if (DEG >= 2) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[4] = SH::c2a * x * y;
        Y[5] = -SH::c2a * y * z;
        Y[6] = SH::c2b * (2.0f * zz - xx - yy);
        Y[7] = -SH::c2a * x * z;
        Y[8] = SH::c2c * (xx - yy);
    }
    if (DEG >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        Y[9] = -SH::c3a * y * (3.0f * xx - yy);
        Y[10] = SH::c3b * x * y * z;
        Y[11] = -SH::c3c * y * (4.0f * zz - xx - yy);
        Y[12] = SH::c3d * z * (2.0f * zz - 3.0f * xx - 3.0f * yy);
        Y[13] = -SH::c3c * x * (4.0f * zz - xx - yy);
        Y[14] = SH::c3e * z * (xx - yy);
        Y[15] = -SH::c3a * x * (xx - 3.0f * yy);
    }
}

// Gradient of sum_k w_k Y_k(x, y, z) w.r.t. (x, y, z), treating them as independent.
template <int DEG>
__device__ __forceinline__ void sh_basis_vjp(float x, float y, float z, const float *w, float *g) {
    g[0] = g[1] = g[2] = 0.0f;
    if (DEG >= 1) {
        g[1] += -SH::c1 * w[1];
        g[2] += SH::c1 * w[2];
        g[0] += -SH::c1 * w[3];
    }
    if (DEG >= 2) {
        g[0] += SH::c2a * y * w[4];
        g[1] += SH::c2a * x * w[4];
        g[1] += -SH::c2a * z * w[5];
        g[2] += -SH::c2a * y * w[5];
        g[0] += -2.0f * SH::c2b * x * w[6];
        g[1] += -2.0f * SH::c2b * y * w[6];
        g[2] += 4.0f * SH::c2b * z * w[6];
        g[0] += -SH::c2a * z * w[7];
        g[2] += -SH::c2a * x * w[7];
        g[0] += 2.0f * SH::c2c * x * w[8];
        g[1] += -2.0f * SH::c2c * y * w[8];
    }
    if (DEG >= 3) {
        const float xx = x * x, yy = y * y, zz = z * z;
        g[0] += -SH::c3a * 6.0f * x * y * w[9];
        g[1] += -SH::c3a * (3.0f * xx - 3.0f * yy) * w[9];
        g[0] += SH::c3b * y * z * w[10];
        g[1] += SH::c3b * x * z * w[10];
        g[2] += SH::c3b * x * y * w[10];
        g[0] += SH::c3c * 2.0f * x * y * w[11];
        g[1] += -SH::c3c * (4.0f * zz - xx - 3.0f * yy) * w[11];
        g[2] += -SH::c3c * 8.0f * y * z * w[11];
        g[0] += -SH::c3d * 6.0f * x * z * w[12];
        g[1] += -SH::c3d * 6.0f * y * z * w[12];
        g[2] += SH::c3d * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12];
        g[0] += -SH::c3c * (4.0f * zz - 3.0f * xx - yy) * w[13];
        g[1] += SH::c3c * 2.0f * x * y * w[13];
        g[2] += -SH::c3c * 8.0f * x * z * w[13];
        g[0] += SH::c3e * 2.0f * x * z * w[14];
        g[1] += -SH::c3e * 2.0f * y * z * w[14];
        g[2] += SH::c3e * (xx - yy) * w[14];
        g[0] += -SH::c3a * (3.0f * xx - 3.0f * yy) * w[15];
        g[1] += SH::c3a * 6.0f * x * y * w[15];
    }
}

template <int DEG>
__device__ __forceinline__ void load_sh(const float *__restrict__ sh, int i, float (*c)[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    if constexpr ((K * 3) % 4 == 0) {
        const float4 *p = reinterpret_cast<const float4 *>(sh + (size_t)i * K * 3);
        float buf[K * 3];
#pragma unroll
        for (int j = 0; j < K * 3 / 4; ++j) {
            const float4 v = __ldg(p + j);
            buf[4 * j] = v.x; buf[4 * j + 1] = v.y; buf[4 * j + 2] = v.z; buf[4 * j + 3] = v.w;
        }
#pragma unroll
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) c[k][ch] = buf[3 * k + ch];
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) c[k][ch] = __ldg(sh + ((size_t)i * K + k) * 3 + ch);
    }
}

template <int DEG>
__device__ __forceinline__ void store_sh(float *__restrict__ dsh, int i, const float (*c)[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    if constexpr ((K * 3) % 4 == 0) {
        float4 *p = reinterpret_cast<float4 *>(dsh + (size_t)i * K * 3);
        float buf[K * 3];
#pragma unroll
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) buf[3 * k + ch] = c[k][ch];
#pragma unroll
        for (int j = 0; j < K * 3 / 4; ++j) p[j] = make_float4(buf[4 * j], buf[4 * j + 1], buf[4 * j + 2], buf[4 * j + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) dsh[((size_t)i * K + k) * 3 + ch] = c[k][ch];
    }
}

// The fixed FP32 projection sequence.  Returns false when the splat is culled.
struct Geom {
    float t[3];
    float A, B, C;
    float u0, u1;
    int rect[4];
    int radius;
};

__device__ __forceinline__ bool project_fixed(const float m[3], const float s[3], const float4 qr,
                                              const Cam &cam, float psi, int tile, Geom &g) {
    const float *V = cam.V;
    float t[3];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        t[r] = __fmaf_rn(V[4 * r + 2], m[2], __fmaf_rn(V[4 * r + 1], m[1], __fmaf_rn(V[4 * r], m[0], V[4 * r + 3])));
    const float tz = t[2];
    if (!(tz > cam.near_plane)) return false;

    const float n2 = __fmaf_rn(qr.w, qr.w, __fmaf_rn(qr.z, qr.z, __fmaf_rn(qr.y, qr.y, __fmul_rn(qr.x, qr.x))));
    if (!(n2 > 0.0f) || !isfinite(n2)) return false;
    const float inv = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    // quats are stored (w, x, y, z) = (qr.x, qr.y, qr.z, qr.w)
    const float w = __fmul_rn(qr.x, inv), x = __fmul_rn(qr.y, inv), y = __fmul_rn(qr.z, inv), z = __fmul_rn(qr.w, inv);
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    float R[3][3];
    R[0][0] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(yy, zz)));
    R[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    R[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    R[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    R[1][1] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, zz)));
    R[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    R[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    R[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    R[2][2] = __fsub_rn(1.0f, __fmul_rn(2.0f, __fadd_rn(xx, yy)));

    float M[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[j][k] = __fmul_rn(R[j][k], s[k]);
    float S[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int l = j; l < 3; ++l) {
            S[j][l] = __fmaf_rn(M[j][2], M[l][2], __fmaf_rn(M[j][1], M[l][1], __fmul_rn(M[j][0], M[l][0])));
            S[l][j] = S[j][l];
        }

    const float fx = cam.fx, fy = cam.fy;
    const float txtz = __fdiv_rn(t[0], tz), tytz = __fdiv_rn(t[1], tz);
    const float limx = cam.limx, limy = cam.limy;
    const float txc = __fmul_rn(fminf(limx, fmaxf(-limx, txtz)), tz);
    const float tyc = __fmul_rn(fminf(limy, fmaxf(-limy, tytz)), tz);
    const float tz2 = __fmul_rn(tz, tz);
    const float J00 = __fdiv_rn(fx, tz), J02 = __fdiv_rn(-__fmul_rn(fx, txc), tz2);
    const float J11 = __fdiv_rn(fy, tz), J12 = __fdiv_rn(-__fmul_rn(fy, tyc), tz2);

    float T0[3], T1[3], U0[3], U1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = __fmaf_rn(J02, V[8 + k], __fmul_rn(J00, V[k]));
        T1[k] = __fmaf_rn(J12, V[8 + k], __fmul_rn(J11, V[4 + k]));
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        U0[k] = __fmaf_rn(T0[2], S[2][k], __fmaf_rn(T0[1], S[1][k], __fmul_rn(T0[0], S[0][k])));
        U1[k] = __fmaf_rn(T1[2], S[2][k], __fmaf_rn(T1[1], S[1][k], __fmul_rn(T1[0], S[0][k])));
    }
    const float s00 = __fmaf_rn(U0[2], T0[2], __fmaf_rn(U0[1], T0[1], __fmul_rn(U0[0], T0[0])));
    const float s01 = __fmaf_rn(U0[2], T1[2], __fmaf_rn(U0[1], T1[1], __fmul_rn(U0[0], T1[0])));
    const float s11 = __fmaf_rn(U1[2], T1[2], __fmaf_rn(U1[1], T1[1], __fmul_rn(U1[0], T1[0])));

    const float a = __fadd_rn(__fmul_rn(psi, s00), kDilation);
    const float b = __fmul_rn(psi, s01);
    const float c = __fadd_rn(__fmul_rn(psi, s11), kDilation);
    const float det = __fmaf_rn(a, c, -__fmul_rn(b, b));
    if (!(det > 0.0f)) return false;
    g.A = __fdiv_rn(c, det);
    g.B = __fdiv_rn(-b, det);
    g.C = __fdiv_rn(a, det);

    const float mid = __fmul_rn(0.5f, __fadd_rn(a, c));
    const float disc = __fmaf_rn(mid, mid, -det);
    const float lam = __fadd_rn(mid, __fsqrt_rn(fmaxf(disc, 0.0f)));
    const float Rf = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));

    const float u0 = __fmaf_rn(fx, txtz, cam.cx), u1 = __fmaf_rn(fy, tytz, cam.cy);
    if (!isfinite(u0) || !isfinite(u1) || !isfinite(Rf)) return false;
    const float x0 = fmaxf(ceilf(__fsub_rn(__fsub_rn(u0, Rf), 0.5f)), 0.0f);
    const float x1 = fminf(floorf(__fsub_rn(__fadd_rn(u0, Rf), 0.5f)), (float)(cam.W - 1));
    const float y0 = fmaxf(ceilf(__fsub_rn(__fsub_rn(u1, Rf), 0.5f)), 0.0f);
    const float y1 = fminf(floorf(__fsub_rn(__fadd_rn(u1, Rf), 0.5f)), (float)(cam.H - 1));
    if (!(x0 <= x1) || !(y0 <= y1)) return false;
    const int tsh = __ffs(tile) - 1;  // tile is 8, 16 or 32 and the bounds are >= 0: a shift divides
    g.rect[0] = (int)x0 >> tsh;
    g.rect[1] = (int)y0 >> tsh;
    g.rect[2] = (int)x1 >> tsh;
    g.rect[3] = (int)y1 >> tsh;
    g.radius = (int)fminf(Rf, 16777216.0f);
    g.u0 = u0;
    g.u1 = u1;
    g.t[0] = t[0]; g.t[1] = t[1]; g.t[2] = tz;
    return true;
}

// One CTA takes kPreThreads consecutive splats in two phases.  Phase 1: every thread projects
// its splat (the decision track) and either writes the culled record or queues the splat, with
// its projected geometry, in shared memory.  Phase 2: the threads take the queued (visible)
// splats densely and do the heavy part -- member tiles by row runs, SH colour, the records --
// so that whole warps, not 38% of each warp's lanes, run it.
constexpr int kPreThreads = 256;

// L2 prefetch of a queued splat's SH row in phase 1 (1), or none (0).
#ifndef DARB_PRE_SH_PREFETCH
#define DARB_PRE_SH_PREFETCH 1
#endif
// A culled splat's record: radius 0, no member tiles, unpacked runs.  Its other fields are not
// read by any later step and are left as they were (1), or zeroed as well (0).
#ifndef DARB_PRE_CULLED_MIN
#define DARB_PRE_CULLED_MIN 1
#endif

__device__ __forceinline__ void write_culled(const ProjectedOut &out, int i) {
    out.radius[i] = 0;
    out.tiles_touched[i] = 0;
    out.tile_runs[i] = kRunsUnpacked;
#if !DARB_PRE_CULLED_MIN
    out.tile_rect[i] = make_int4(0, 0, 0, 0);
    out.depth[i] = 0.0f;
#endif
}

struct PreGeom {
    float tz, A, B, C, u0, u1;
    int rect[4];
    int radius, idx;
};

// Compiled for 5 resident CTAs per SM (48 registers, 1280 threads, each with DARB_PRE_SPT = 2
// splats): the projection is latency-bound, and a register cap raised occupancy from the
// compiler's choice (0.172 -> 0.153 ms at 3M splats / 1080p with 8 CTAs of one splat per thread).
// With two splats per thread, 5 CTAs measure 0.136 ms against 0.145 at 6 (40 registers, which
// spill) and 0.142 at 4; one splat per thread at 6 CTAs: 0.145.  DARB_PRE_MIN_CTAS=0 leaves the
// register count to the compiler.
#ifndef DARB_PRE_MIN_CTAS
#define DARB_PRE_MIN_CTAS 5
#endif
// Splats per thread of k_preprocess: with 2, a thread issues both splats' loads before it
// projects the first.
#ifndef DARB_PRE_SPT
#define DARB_PRE_SPT 2
#endif
#if DARB_PRE_MIN_CTAS > 0
#define DARB_PRE_BOUNDS __launch_bounds__(kPreThreads, DARB_PRE_MIN_CTAS)
#else
#define DARB_PRE_BOUNDS __launch_bounds__(kPreThreads)
#endif

// Phase 2 of k_preprocess for one queued (projected, not culled) splat: member tiles by row
// runs, the records, the SH colour.
template <int DEG>
__device__ __forceinline__ void preprocess_queued(const PreGeom &g, const float *__restrict__ means,
                                                  const float *__restrict__ opac, const float *__restrict__ sh,
                                                  const Cam &cam, int tile, float qmax, const ProjectedOut &out) {
    const int i = g.idx;
    const SpanCtx sc = make_span_ctx(qmax, tile, cam.W, cam.H);
    const int4 r = make_int4(g.rect[0], g.rect[1], g.rect[2], g.rect[3]);
    uint32_t cnt = 0;  // member tiles: the ellipse's run in every row of the rectangle
    const bool pack = runs_packable(r);
    uint64_t runs = pack ? kRunsNone : kRunsUnpacked;
    const SpanSplat sp = span_prepare(g.u0, g.u1, g.A, g.B, g.C, qmax);
    for (int ty = r.y; ty <= r.w; ++ty) {
        int c0, c1;
        if (span_row(sp, sc, r, ty, c0, c1)) {
            cnt += (uint32_t)(c1 - c0 + 1);
            if (pack) runs = runs_put(runs, r, ty, c0, c1);
        }
    }
    if (cnt == 0) {  // an ellipse that reaches no tile: culled
        write_culled(out, i);
        return;
    }
    out.depth[i] = g.tz;
    out.radius[i] = g.radius;
    out.tile_rect[i] = r;
    out.tiles_touched[i] = cnt;
    out.tile_runs[i] = runs;
    out.mean2d[i] = make_float2(g.u0, g.u1);
    out.conic_o[i] = make_float4(g.A, g.B, g.C, __ldg(opac + i));

    // SH colour (value track, ordinary FP32)
    constexpr int K = (DEG + 1) * (DEG + 1);
    float coef[K][3];
    load_sh<DEG>(sh, i, coef);
    float d0 = __ldg(means + 3 * (size_t)i) - cam.campos[0], d1 = __ldg(means + 3 * (size_t)i + 1) - cam.campos[1],
          d2 = __ldg(means + 3 * (size_t)i + 2) - cam.campos[2];
    const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    d0 *= il; d1 *= il; d2 *= il;
    float Y[K];
    sh_eval_basis<DEG>(d0, d1, d2, Y);
    uint8_t cl = 0;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float v = 0.5f;
#pragma unroll
        for (int k = 0; k < K; ++k) v = fmaf(Y[k], coef[k][ch], v);
        if (v < 0.0f) {
            v = 0.0f;
            cl |= (uint8_t)(1u << ch);
        }
        out.rgb[3 * (size_t)i + ch] = v;
    }
    out.clamped[i] = cl;
}

template <int DEG>
__global__ void DARB_PRE_BOUNDS
k_preprocess(int n, const float *__restrict__ means, const float *__restrict__ scales,
             const float4 *__restrict__ quats, const float *__restrict__ opac,
             const float *__restrict__ sh, Cam cam, float psi, int tile, float qmax, ProjectedOut out) {
    pdl_entry();
    constexpr int SPT = DARB_PRE_SPT;
    __shared__ PreGeom s_q[kPreThreads * SPT];
    __shared__ int s_n;
    if (threadIdx.x == 0) s_n = 0;
    __syncthreads();
    {
        // the loads of every splat of the thread first, so that the later splats' loads are in
        // flight while the first is projected
        const int i0 = blockIdx.x * kPreThreads * SPT + (int)threadIdx.x;
        float m[SPT][3], sc3[SPT][3];
        float4 qr[SPT];
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
            const int i = i0 + u * kPreThreads;
            if (i < n) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    m[u][c] = __ldg(means + 3 * (size_t)i + c);
                    sc3[u][c] = __ldg(scales + 3 * (size_t)i + c);
                }
                qr[u] = __ldg(quats + i);
            }
        }
#pragma unroll
        for (int u = 0; u < SPT; ++u) {
            const int i = i0 + u * kPreThreads;
            bool vis = false;
            Geom g;
            if (i < n) vis = project_fixed(m[u], sc3[u], qr[u], cam, psi, tile, g);
            const uint32_t vm = __ballot_sync(0xffffffffu, vis);
            int base = 0;
            if ((threadIdx.x & 31) == 0 && vm) base = atomicAdd(&s_n, __popc(vm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (vis) {
                PreGeom &q = s_q[base + __popc(vm & ((1u << (threadIdx.x & 31)) - 1u))];
                q.tz = g.t[2];
                q.A = g.A;
                q.B = g.B;
                q.C = g.C;
                q.u0 = g.u0;
                q.u1 = g.u1;
#pragma unroll
                for (int k = 0; k < 4; ++k) q.rect[k] = g.rect[k];
                q.radius = g.radius;
                q.idx = i;
            } else if (i < n) {
                write_culled(out, i);
            }
#if DARB_PRE_SH_PREFETCH
            if (vis) {  // start the SH row of a queued splat on its way to L2 during the projection of the rest
                const char *row = reinterpret_cast<const char *>(sh + (size_t)i * 3 * (DEG + 1) * (DEG + 1));
                constexpr int kRowBytes = 12 * (DEG + 1) * (DEG + 1);
#pragma unroll
                for (int o = 0; o < kRowBytes + 127; o += 128)
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(row + min(o, kRowBytes - 1)));
            }
#endif
        }
    }
    __syncthreads();
    const int nq = s_n;
    for (int e = threadIdx.x; e < nq; e += kPreThreads) preprocess_queued<DEG>(s_q[e], means, opac, sh, cam, tile, qmax,
                                                                               out);
}


// ---------------------------------------------------------------------------
// Backward of the preprocessing.  Recomputes the forward quantities in FP32 and
// applies the chain rule: conic -> Sigma2 (dSigma2 = -K G K), Sigma2 = psi Sigma' + 0.3 I,
// Sigma' = T Sigma T^T with T = J W, J(t) with the guard band, mu'(t), t = W m + w,
// Sigma = M M^T with M = R(q/|q|) diag(s), and the SH colour (coefficients and viewing
// direction).

template <int DEG, class LoadCoef>
__device__ __forceinline__ void splat_backward(int i, const float *__restrict__ means, const float *__restrict__ scales,
                                               const float4 *__restrict__ quats, LoadCoef load_coef,
                                               const Cam &cam, float psi, uint8_t cl,
                                               const float4 *__restrict__ grad2d, float *dm, float *ds, float *dq,
                                               float &dop, float (*dcoef)[3]) {
    constexpr int K = (DEG + 1) * (DEG + 1);
    const float4 g0 = grad2d[3 * (size_t)i], g1 = grad2d[3 * (size_t)i + 1], g2 = grad2d[3 * (size_t)i + 2];
    const float dmx = g0.x, dmy = g0.y, dA = g0.z, dB = g0.w, dC = g1.x, dO = g1.y;
    const float drgb[3] = {g1.z, g1.w, g2.x};
    dop = dO;

    const float *V = cam.V;
    const float m[3] = {means[3 * (size_t)i], means[3 * (size_t)i + 1], means[3 * (size_t)i + 2]};
    float t[3];
    for (int r = 0; r < 3; ++r) t[r] = V[4 * r] * m[0] + V[4 * r + 1] * m[1] + V[4 * r + 2] * m[2] + V[4 * r + 3];
    const float tx = t[0], ty = t[1], tz = t[2];

    const float4 qr = quats[i];
    const float qn = sqrtf(qr.x * qr.x + qr.y * qr.y + qr.z * qr.z + qr.w * qr.w);
    const float w = qr.x / qn, x = qr.y / qn, y = qr.z / qn, z = qr.w / qn;
    const float R[3][3] = {{1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y)},
                           {2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x)},
                           {2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)}};
    const float s[3] = {scales[3 * (size_t)i], scales[3 * (size_t)i + 1], scales[3 * (size_t)i + 2]};
    float M[3][3], Sig[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) M[j][l] = R[j][l] * s[l];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) Sig[j][l] = M[j][0] * M[l][0] + M[j][1] * M[l][1] + M[j][2] * M[l][2];

    // Jacobian; the guard-band decision repeats the forward's FP32 sequence
    const float fx = cam.fx, fy = cam.fy;
    const float txtz = __fdiv_rn(tx, tz), tytz = __fdiv_rn(ty, tz);
    const float limx = cam.limx, limy = cam.limy;
    const bool clx = (txtz < -limx) || (txtz > limx), cly = (tytz < -limy) || (tytz > limy);
    const float Lx = txtz < 0.f ? -limx : limx, Ly = tytz < 0.f ? -limy : limy;
    const float txc = clx ? Lx * tz : tx, tyc = cly ? Ly * tz : ty;
    const float iz = 1.0f / tz, iz2 = iz * iz;
    const float J00 = fx * iz, J02 = -fx * txc * iz2, J11 = fy * iz, J12 = -fy * tyc * iz2;
    float Tm[2][3];
    for (int k = 0; k < 3; ++k) {
        Tm[0][k] = J00 * V[k] + J02 * V[8 + k];
        Tm[1][k] = J11 * V[4 + k] + J12 * V[8 + k];
    }
    float TS[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) TS[r][k] = Tm[r][0] * Sig[0][k] + Tm[r][1] * Sig[1][k] + Tm[r][2] * Sig[2][k];
    const float s00 = TS[0][0] * Tm[0][0] + TS[0][1] * Tm[0][1] + TS[0][2] * Tm[0][2];
    const float s01 = TS[0][0] * Tm[1][0] + TS[0][1] * Tm[1][1] + TS[0][2] * Tm[1][2];
    const float s11 = TS[1][0] * Tm[1][0] + TS[1][1] * Tm[1][1] + TS[1][2] * Tm[1][2];
    const float a = psi * s00 + kDilation, b = psi * s01, c = psi * s11 + kDilation;
    const float idet = 1.0f / (a * c - b * b);
    const float K00 = c * idet, K01 = -b * idet, K11 = a * idet;

    // dSigma2 = -K G K with G = [[dA, dB/2], [dB/2, dC]]; then x psi
    const float G01 = 0.5f * dB;
    const float KG00 = K00 * dA + K01 * G01, KG01 = K00 * G01 + K01 * dC;
    const float KG10 = K01 * dA + K11 * G01, KG11 = K01 * G01 + K11 * dC;
    const float d00 = -psi * (KG00 * K00 + KG01 * K01);
    const float d01 = -psi * (KG00 * K01 + KG01 * K11);
    const float d11 = -psi * (KG10 * K01 + KG11 * K11);
    const float dsp[2][2] = {{d00, d01}, {d01, d11}};

    // Sigma' = Tm Sig Tm^T: dSig = Tm^T dsp Tm, dTm = 2 dsp Tm Sig
    float dSig[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) {
            float v = 0.f;
            for (int r = 0; r < 2; ++r)
                for (int u = 0; u < 2; ++u) v += Tm[r][j] * dsp[r][u] * Tm[u][l];
            dSig[j][l] = v;
        }
    float dTm[2][3];
    for (int r = 0; r < 2; ++r)
        for (int k = 0; k < 3; ++k) dTm[r][k] = 2.f * (dsp[r][0] * TS[0][k] + dsp[r][1] * TS[1][k]);
    float dJ00 = 0.f, dJ02 = 0.f, dJ11 = 0.f, dJ12 = 0.f;
    for (int k = 0; k < 3; ++k) {
        dJ00 += dTm[0][k] * V[k];
        dJ02 += dTm[0][k] * V[8 + k];
        dJ11 += dTm[1][k] * V[4 + k];
        dJ12 += dTm[1][k] * V[8 + k];
    }
    float dt[3] = {0.f, 0.f, 0.f};
    dt[2] += -(dJ00 * fx + dJ11 * fy) * iz2;
    if (!clx) {
        dt[0] += -dJ02 * fx * iz2;
        dt[2] += dJ02 * 2.f * fx * tx * iz2 * iz;
    } else {
        dt[2] += dJ02 * fx * Lx * iz2;
    }
    if (!cly) {
        dt[1] += -dJ12 * fy * iz2;
        dt[2] += dJ12 * 2.f * fy * ty * iz2 * iz;
    } else {
        dt[2] += dJ12 * fy * Ly * iz2;
    }
    dt[0] += dmx * fx * iz;
    dt[1] += dmy * fy * iz;
    dt[2] += -(dmx * fx * tx + dmy * fy * ty) * iz2;
    float gm[3];
    for (int j = 0; j < 3; ++j) gm[j] = V[j] * dt[0] + V[4 + j] * dt[1] + V[8 + j] * dt[2];

    // Sigma = M M^T, M = R diag(s)
    float dM[3][3], dR[3][3];
    for (int j = 0; j < 3; ++j)
        for (int l = 0; l < 3; ++l) dM[j][l] = 2.f * (dSig[j][0] * M[0][l] + dSig[j][1] * M[1][l] + dSig[j][2] * M[2][l]);
    for (int l = 0; l < 3; ++l) {
        ds[l] = dM[0][l] * R[0][l] + dM[1][l] * R[1][l] + dM[2][l] * R[2][l];
        for (int j = 0; j < 3; ++j) dR[j][l] = dM[j][l] * s[l];
    }
    // R(w, x, y, z): partial derivatives of the nine entries
    const float gw = 2.f * (-z * dR[0][1] + y * dR[0][2] + z * dR[1][0] - x * dR[1][2] - y * dR[2][0] + x * dR[2][1]);
    const float gx = 2.f * (y * dR[0][1] + z * dR[0][2] + y * dR[1][0] - 2.f * x * dR[1][1] - w * dR[1][2] +
                            z * dR[2][0] + w * dR[2][1] - 2.f * x * dR[2][2]);
    const float gy = 2.f * (-2.f * y * dR[0][0] + x * dR[0][1] + w * dR[0][2] + x * dR[1][0] + z * dR[1][2] -
                            w * dR[2][0] + z * dR[2][1] - 2.f * y * dR[2][2]);
    const float gz = 2.f * (-2.f * z * dR[0][0] - w * dR[0][1] + x * dR[0][2] + w * dR[1][0] - 2.f * z * dR[1][1] +
                            y * dR[1][2] + x * dR[2][0] + y * dR[2][1]);
    const float nd = w * gw + x * gx + y * gy + z * gz;
    const float iqn = 1.0f / qn;
    dq[0] = (gw - w * nd) * iqn;
    dq[1] = (gx - x * nd) * iqn;
    dq[2] = (gy - y * nd) * iqn;
    dq[3] = (gz - z * nd) * iqn;

    // SH: coefficients and the viewing direction
    float v0 = m[0] - cam.campos[0], v1 = m[1] - cam.campos[1], v2 = m[2] - cam.campos[2];
    const float len = sqrtf(v0 * v0 + v1 * v1 + v2 * v2);
    const float dir[3] = {v0 / len, v1 / len, v2 / len};
    float Y[K];
    sh_eval_basis<DEG>(dir[0], dir[1], dir[2], Y);
    float gr[3];
    for (int ch = 0; ch < 3; ++ch) gr[ch] = ((cl >> ch) & 1) ? 0.f : drgb[ch];
    float coef[K][3];
    load_coef(coef);
    float wsum[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
        float acc = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            dcoef[k][ch] = Y[k] * gr[ch];
            acc += gr[ch] * coef[k][ch];
        }
        wsum[k] = acc;
    }
    float gd[3];
    sh_basis_vjp<DEG>(dir[0], dir[1], dir[2], wsum, gd);
    const float dd = dir[0] * gd[0] + dir[1] * gd[1] + dir[2] * gd[2];
    for (int j = 0; j < 3; ++j) dm[j] = gm[j] + (gd[j] - dir[j] * dd) / len;
}


template <int DEG>
__global__ void __launch_bounds__(256)
k_preprocess_bwd(int n, const float *__restrict__ means, const float *__restrict__ scales,
                 const float4 *__restrict__ quats, const float *__restrict__ sh, Cam cam, float psi,
                 const int *__restrict__ radius, const uint8_t *__restrict__ clamped,
                 const float4 *__restrict__ grad2d, GradOut out) {
    pdl_entry();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    constexpr int K = (DEG + 1) * (DEG + 1);
    float dm[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, dop = 0.f;
    float dcoef[K][3];
#pragma unroll
    for (int k = 0; k < K; ++k) dcoef[k][0] = dcoef[k][1] = dcoef[k][2] = 0.0f;
    if (radius[i] != 0)
        splat_backward<DEG>(
            i, means, scales, quats, [&](float(*c)[3]) { load_sh<DEG>(sh, i, c); }, cam, psi, clamped[i], grad2d, dm,
            ds, dq, dop, dcoef);
    for (int j = 0; j < 3; ++j) {
        out.dmeans[3 * (size_t)i + j] = dm[j];
        out.dscales[3 * (size_t)i + j] = ds[j];
    }
    reinterpret_cast<float4 *>(out.dquats)[i] = make_float4(dq[0], dq[1], dq[2], dq[3]);
    out.dopacities[i] = dop;
    store_sh<DEG>(out.dsh, i, dcoef);
}

// The same gradients applied at once by Adam to the raw parameters (log-scales, opacity
// logits), refreshing the activated copies; no gradient goes through HBM.
//
// Two phases per block of kBwdAdamThreads splats.  (1) Each thread runs its splat's chain
// rule and leaves the gradients w.r.t. the raw parameters in shared memory, one segment per
// parameter group laid out as in HBM.  (2) The block walks each group's contiguous HBM
// segment (its splats' rows) with consecutive lanes on consecutive float4s, several in
// flight per thread, and applies Adam: parameters and both moments are read and written
// once, coalesced, as in a flat optimiser pass.
template <int DEG>
struct BwdAdamStage {
    static constexpr int K = (DEG + 1) * (DEG + 1);
    static constexpr int ROW = 3 * K;  // SH floats per splat
    // SH rows of an even number of float4s are padded by one float4: the per-splat float4
    // stores of a quarter-warp then fall in distinct banks
    static constexpr int PAD = (ROW % 4 == 0 && (ROW / 4) % 2 == 0) ? ROW + 4 : ROW;
};

constexpr int kBwdAdamThreads = 128;

// float4s in flight per thread and array in the Adam walk, and whether its parameter / moment
// traffic uses the streaming (evict-first) cache hints.
#ifndef DARB_ADAM_UNROLL
#define DARB_ADAM_UNROLL 4
#endif
#ifndef DARB_ADAM_STREAMING
#define DARB_ADAM_STREAMING 0
#endif
__device__ __forceinline__ float4 adam_ld(const float4 *p) {
#if DARB_ADAM_STREAMING
    return __ldcs(p);
#else
    return *p;
#endif
}
__device__ __forceinline__ void adam_st(float4 *p, float4 v) {
#if DARB_ADAM_STREAMING
    __stcs(p, v);
#else
    *p = v;
#endif
}

// One parameter group of the block: count floats from p/m/v (HBM, 16-byte aligned) with
// gradients grad4(j) for float4 j; ACT 1 refreshes act = exp(p), ACT 2 act = sigmoid(p).
template <int ACT, class Grad4, class LrOf>
__device__ __forceinline__ void block_adam(int count, float *__restrict__ p, float *__restrict__ m,
                                           float *__restrict__ v, float *__restrict__ act, Grad4 grad4, LrOf lr_of,
                                           const AdamConsts &ac) {
    constexpr int NT = kBwdAdamThreads, U = DARB_ADAM_UNROLL;
    const int n4 = count >> 2;
    float4 *p4 = reinterpret_cast<float4 *>(p), *m4 = reinterpret_cast<float4 *>(m), *v4 = reinterpret_cast<float4 *>(v);
    for (int b = threadIdx.x; b < n4; b += NT * U) {
        float4 P[U], M[U], V[U], G[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = b + u * NT;
            if (j < n4) {
                P[u] = adam_ld(p4 + j);
                M[u] = adam_ld(m4 + j);
                V[u] = adam_ld(v4 + j);
                G[u] = grad4(j);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = b + u * NT;
            if (j < n4) {
                adam_apply(P[u].x, G[u].x, M[u].x, V[u].x, lr_of(4 * j + 0), ac);
                adam_apply(P[u].y, G[u].y, M[u].y, V[u].y, lr_of(4 * j + 1), ac);
                adam_apply(P[u].z, G[u].z, M[u].z, V[u].z, lr_of(4 * j + 2), ac);
                adam_apply(P[u].w, G[u].w, M[u].w, V[u].w, lr_of(4 * j + 3), ac);
                adam_st(p4 + j, P[u]);
                adam_st(m4 + j, M[u]);
                adam_st(v4 + j, V[u]);
                if (ACT == 1)
                    reinterpret_cast<float4 *>(act)[j] =
                        make_float4(expf(P[u].x), expf(P[u].y), expf(P[u].z), expf(P[u].w));
                if (ACT == 2)
                    reinterpret_cast<float4 *>(act)[j] =
                        make_float4(1.0f / (1.0f + expf(-P[u].x)), 1.0f / (1.0f + expf(-P[u].y)),
                                    1.0f / (1.0f + expf(-P[u].z)), 1.0f / (1.0f + expf(-P[u].w)));
            }
        }
    }
    // the last block's ragged end: count % 4 floats
    const int f = (n4 << 2) + (int)threadIdx.x;
    if (f < count) {
        const float4 g = grad4(f >> 2);
        const float gs[4] = {g.x, g.y, g.z, g.w};
        float pp = p[f], mm = m[f], vv = v[f];
        adam_apply(pp, gs[f & 3], mm, vv, lr_of(f), ac);
        p[f] = pp;
        m[f] = mm;
        v[f] = vv;
        if (ACT == 1) act[f] = expf(pp);
        if (ACT == 2) act[f] = 1.0f / (1.0f + expf(-pp));
    }
}

#ifndef DARB_BWD_ADAM_MIN_CTAS
#define DARB_BWD_ADAM_MIN_CTAS 6
#endif
template <int DEG>
__global__ void __launch_bounds__(kBwdAdamThreads, DEG == 2 ? 4 : DARB_BWD_ADAM_MIN_CTAS)
k_preprocess_bwd_adam(int n, darb_train_params P, darb_adam_state A, AdamConsts ac, Cam cam, float psi,
                      const int *__restrict__ radius, const uint8_t *__restrict__ clamped,
                      const float4 *__restrict__ grad2d) {
    pdl_entry();
    using S = BwdAdamStage<DEG>;
    constexpr int K = S::K, ROW = S::ROW, PAD = S::PAD, NT = kBwdAdamThreads;
    // gradient segments; the tail of each is read as float4 up to a multiple of 4 floats
    __shared__ __align__(16) float s_means[NT * 3];
    __shared__ __align__(16) float s_lsc[NT * 3];
    __shared__ __align__(16) float s_quat[NT * 4];
    __shared__ __align__(16) float s_logit[NT];
    __shared__ __align__(16) float s_sh[NT * PAD];
    const int t = threadIdx.x;
    const int i0 = blockIdx.x * NT;
    const int i = i0 + t;
    const int cnt = min(NT, n - i0);
    if (i < n) {
        float dm[3] = {0.f, 0.f, 0.f}, ds[3] = {0.f, 0.f, 0.f}, dq[4] = {0.f, 0.f, 0.f, 0.f}, dop = 0.f;
        float dcoef[K][3];
#pragma unroll
        for (int k = 0; k < K; ++k) dcoef[k][0] = dcoef[k][1] = dcoef[k][2] = 0.0f;
        if (radius[i] != 0)
            splat_backward<DEG>(
                i, P.means, P.scales, reinterpret_cast<const float4 *>(P.quats),
                [&](float(*c)[3]) { load_sh<DEG>(P.sh, i, c); }, cam, psi, clamped[i], grad2d, dm, ds, dq, dop, dcoef);
        // gradients w.r.t. the raw parameters: d scale / d log-scale = scale, d sigmoid = o (1 - o)
        const size_t i3 = 3 * (size_t)i;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            s_means[3 * t + j] = dm[j];
            s_lsc[3 * t + j] = ds[j] * P.scales[i3 + j];
        }
        *reinterpret_cast<float4 *>(&s_quat[4 * t]) = make_float4(dq[0], dq[1], dq[2], dq[3]);
        const float o = P.opacities[i];
        s_logit[t] = dop * (o * (1.0f - o));
        const float *dc = &dcoef[0][0];
        if constexpr (ROW % 4 == 0) {
#pragma unroll
            for (int u = 0; u < ROW / 4; ++u)
                *reinterpret_cast<float4 *>(&s_sh[t * PAD + 4 * u]) =
                    make_float4(dc[4 * u], dc[4 * u + 1], dc[4 * u + 2], dc[4 * u + 3]);
        } else {
#pragma unroll
            for (int u = 0; u < ROW; ++u) s_sh[t * PAD + u] = dc[u];
        }
    }
    __syncthreads();
    // Block segments start at row i0 (a multiple of 128), so each is 16-byte aligned in HBM
    // (the arrays are) and in shared memory.
    const size_t r3 = 3 * (size_t)i0;
    auto flat = [](const float *s) { return [s](int j) { return reinterpret_cast<const float4 *>(s)[j]; }; };
    auto lr_const = [](float lr) { return [lr](int) { return lr; }; };
    block_adam<0>(3 * cnt, P.means + r3, A.m_means + r3, A.v_means + r3, nullptr, flat(s_means),
                  lr_const(ac.lr_means), ac);
    block_adam<1>(3 * cnt, P.log_scales + r3, A.m_scales + r3, A.v_scales + r3, P.scales + r3, flat(s_lsc),
                  lr_const(ac.lr_scales), ac);
    block_adam<0>(4 * cnt, P.quats + 4 * (size_t)i0, A.m_quats + 4 * (size_t)i0, A.v_quats + 4 * (size_t)i0, nullptr,
                  flat(s_quat), lr_const(ac.lr_quats), ac);
    block_adam<2>(cnt, P.opacity_logits + i0, A.m_opac + i0, A.v_opac + i0, P.opacities + i0, flat(s_logit),
                  lr_const(ac.lr_opacities), ac);
    const size_t rs = (size_t)i0 * ROW;
    const float lr_dc = ac.lr_sh_dc, lr_rest = ac.lr_sh_rest;
    auto lr_sh = [=](int f) { return f % ROW < 3 ? lr_dc : lr_rest; };  // the DC term: first 3 floats of a row
    if constexpr (PAD == ROW) {
        block_adam<0>(ROW * cnt, P.sh + rs, A.m_sh + rs, A.v_sh + rs, nullptr, flat(s_sh), lr_sh, ac);
    } else {
        auto padded = [&](int j) {
            const int r = j / (ROW / 4), col = 4 * (j - r * (ROW / 4));
            return *reinterpret_cast<const float4 *>(&s_sh[r * PAD + col]);
        };
        block_adam<0>(ROW * cnt, P.sh + rs, A.m_sh + rs, A.v_sh + rs, nullptr, padded, lr_sh, ac);
    }
}

// ---------------------------------------------------------------------------

cudaError_t launch_preprocess(int n, const darb_splats &sp, const Cam &cam, float psi, int tile, float qmax,
                              const ProjectedOut &out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = kPreThreads, blocks = (n + threads * DARB_PRE_SPT - 1) / (threads * DARB_PRE_SPT);
    const float4 *q = reinterpret_cast<const float4 *>(sp.quats);
    switch (sp.sh_degree) {
    case 0: launch_k(k_preprocess<0>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.opacities, sp.sh,
                     cam, psi, tile, qmax, out); break;
    case 1: launch_k(k_preprocess<1>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.opacities, sp.sh,
                     cam, psi, tile, qmax, out); break;
    case 2: launch_k(k_preprocess<2>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.opacities, sp.sh,
                     cam, psi, tile, qmax, out); break;
    default: launch_k(k_preprocess<3>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.opacities, sp.sh,
                      cam, psi, tile, qmax, out); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd(int n, const darb_splats &sp, const Cam &cam, float psi,
                                  const int *radius, const uint8_t *clamped, const float *grad2d,
                                  const GradOut &out, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const int threads = 256, blocks = (n + threads - 1) / threads;
    const float4 *q = reinterpret_cast<const float4 *>(sp.quats);
    const float4 *g = reinterpret_cast<const float4 *>(grad2d);
    switch (sp.sh_degree) {
    case 0: launch_k(k_preprocess_bwd<0>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.sh, cam, psi, radius, clamped, g, out); break;
    case 1: launch_k(k_preprocess_bwd<1>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.sh, cam, psi, radius, clamped, g, out); break;
    case 2: launch_k(k_preprocess_bwd<2>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.sh, cam, psi, radius, clamped, g, out); break;
    default: launch_k(k_preprocess_bwd<3>, blocks, threads, 0, st, n, sp.means, sp.scales, q, sp.sh, cam, psi, radius, clamped, g, out); break;
    }
    return cudaGetLastError();
}

template <int DEG>
cudaError_t launch_bwd_adam_deg(int n, const darb_train_params &p, const darb_adam_state &s, const AdamConsts &ac,
                                const Cam &cam, float psi, const int *radius, const uint8_t *clamped,
                                const float4 *g, cudaStream_t st) {
    const int blocks = (n + kBwdAdamThreads - 1) / kBwdAdamThreads;
    launch_k(k_preprocess_bwd_adam<DEG>, blocks, kBwdAdamThreads, 0, st, n, p, s, ac, cam, psi, radius, clamped, g);
    return cudaGetLastError();
}

cudaError_t launch_preprocess_bwd_adam(int n, int sh_degree, const darb_train_params &p, const darb_adam_state &s,
                                       const AdamConsts &ac, const Cam &cam, float psi, const int *radius,
                                       const uint8_t *clamped, const float *grad2d, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    const float4 *g = reinterpret_cast<const float4 *>(grad2d);
    switch (sh_degree) {
    case 0: return launch_bwd_adam_deg<0>(n, p, s, ac, cam, psi, radius, clamped, g, st);
    case 1: return launch_bwd_adam_deg<1>(n, p, s, ac, cam, psi, radius, clamped, g, st);
    case 2: return launch_bwd_adam_deg<2>(n, p, s, ac, cam, psi, radius, clamped, g, st);
    default: return launch_bwd_adam_deg<3>(n, p, s, ac, cam, psi, radius, clamped, g, st);
    }
}

}  // namespace darb
