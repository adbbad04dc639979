// Training-step kernels: the L1 photometric loss term (paper Sec. 4.2) and the Adam update of
// the 3DGS optimiser (Sec. 5: original 3DGS hyper-parameters, opacity learning rate 0.02).
// Both are elementwise and HBM-bound; float4 accesses where the layout allows.
#include <algorithm>

#include "kernels.cuh"

namespace darb {

namespace {

__global__ void __launch_bounds__(256)
k_l1_loss(const float *__restrict__ image, const float *__restrict__ target, int count, float inv_count,
          float *__restrict__ dL, float *__restrict__ loss) {
    pdl_entry();
    __shared__ float s_warp[8];
    float acc = 0.0f;
    auto sgn = [inv_count](float d) { return d > 0.0f ? inv_count : (d < 0.0f ? -inv_count : 0.0f); };
    const int tid = blockIdx.x * 256 + threadIdx.x, stride = gridDim.x * 256;
    // float4 lanes when all three buffers are 16-byte aligned, then the ragged end one by one
    const bool vec = ((reinterpret_cast<uintptr_t>(image) | reinterpret_cast<uintptr_t>(target) |
                       reinterpret_cast<uintptr_t>(dL)) & 15) == 0;
    const int n4 = vec ? count >> 2 : 0;
    for (int i = tid; i < n4; i += stride) {
        const float4 a = reinterpret_cast<const float4 *>(image)[i], b = reinterpret_cast<const float4 *>(target)[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        reinterpret_cast<float4 *>(dL)[i] = make_float4(sgn(d0), sgn(d1), sgn(d2), sgn(d3));
        acc += (fabsf(d0) + fabsf(d1)) + (fabsf(d2) + fabsf(d3));
    }
    for (int i = 4 * n4 + tid; i < count; i += stride) {
        const float d = image[i] - target[i];
        dL[i] = sgn(d);
        acc += fabsf(d);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += s_warp[w];
        atomicAdd(loss, s * inv_count);
    }
}

// act: 0 = identity, 1 = exp (log-scale -> scale), 2 = sigmoid (logit -> opacity).
// For act != 0 the incoming gradient is w.r.t. the activated value and `activated` holds that
// value; the raw gradient is g * d(act)/d(raw), and `activated` is refreshed after the step.
template <int ACT>
__device__ __forceinline__ void adam_elem(float &p, float g, float &m, float &v, float lr, float b1, float b2,
                                          float eps, float ibc1, float ibc2, float *act_val) {
    if (ACT == 1) g *= *act_val;
    if (ACT == 2) g *= *act_val * (1.0f - *act_val);
    AdamConsts c;
    c.b1 = b1; c.b2 = b2; c.eps = eps; c.ibc1 = ibc1; c.ibc2 = ibc2;
    adam_apply(p, g, m, v, lr, c);
    if (ACT == 1) *act_val = expf(p);
    if (ACT == 2) *act_val = 1.0f / (1.0f + expf(-p));
}

// Flat parameter group, float4 lanes; `row`/`split` select lr2 for the elements whose index
// within a row of ROW floats is >= SPLIT (the SH coefficients after the DC term).  ROW is a
// multiple of 4 (or 0 for a single learning rate), so no float4 straddles two rows.
template <int ACT, int ROW, int SPLIT>
__global__ void __launch_bounds__(256)
k_adam4(long long count, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
        float *__restrict__ v, float lr, float lr2, float b1, float b2, float eps, float ibc1, float ibc2,
        float *__restrict__ activated) {
    pdl_entry();
    const long long n4 = count >> 2;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n4; j += stride) {
        float4 P = reinterpret_cast<float4 *>(p)[j];
        const float4 G = reinterpret_cast<const float4 *>(g)[j];
        float4 Mm = reinterpret_cast<float4 *>(m)[j];
        float4 V = reinterpret_cast<float4 *>(v)[j];
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
        if (ACT) A = reinterpret_cast<float4 *>(activated)[j];
        float lrs[4] = {lr, lr, lr, lr};
        if (ROW > 0) {
            const int pos = (int)((j * 4) % (ROW > 0 ? ROW : 1));  // ROW is a compile-time constant
#pragma unroll
            for (int u = 0; u < 4; ++u) lrs[u] = (pos + u >= SPLIT) ? lr2 : lr;
        }
        adam_elem<ACT>(P.x, G.x, Mm.x, V.x, lrs[0], b1, b2, eps, ibc1, ibc2, &A.x);
        adam_elem<ACT>(P.y, G.y, Mm.y, V.y, lrs[1], b1, b2, eps, ibc1, ibc2, &A.y);
        adam_elem<ACT>(P.z, G.z, Mm.z, V.z, lrs[2], b1, b2, eps, ibc1, ibc2, &A.z);
        adam_elem<ACT>(P.w, G.w, Mm.w, V.w, lrs[3], b1, b2, eps, ibc1, ibc2, &A.w);
        reinterpret_cast<float4 *>(p)[j] = P;
        reinterpret_cast<float4 *>(m)[j] = Mm;
        reinterpret_cast<float4 *>(v)[j] = V;
        if (ACT) reinterpret_cast<float4 *>(activated)[j] = A;
    }
    // scalar tail (count % 4 elements)
    if (blockIdx.x == 0 && threadIdx.x < (count & 3)) {
        const long long i = (n4 << 2) + threadIdx.x;
        float pp = p[i], mm = m[i], vv = v[i];
        float a = ACT ? activated[i] : 0.f;
        const float l = (ROW > 0 && (int)(i % (ROW > 0 ? ROW : 1)) >= SPLIT) ? lr2 : lr;
        adam_elem<ACT>(pp, g[i], mm, vv, l, b1, b2, eps, ibc1, ibc2, &a);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
        if (ACT) activated[i] = a;
    }
}

// Rows whose length is not a multiple of 4 (SH degrees 0 and 2): scalar lanes.
template <int ROW, int SPLIT>
__global__ void __launch_bounds__(256)
k_adam_rows(long long count, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
            float *__restrict__ v, float lr, float lr2, float b1, float b2, float eps, float ibc1, float ibc2) {
    pdl_entry();
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        float pp = p[i], mm = m[i], vv = v[i];
        const float l = (int)(i % ROW) >= SPLIT ? lr2 : lr;
        adam_elem<0>(pp, g[i], mm, vv, l, b1, b2, eps, ibc1, ibc2, nullptr);
        p[i] = pp;
        m[i] = mm;
        v[i] = vv;
    }
}

int grid_for(long long count) {
    long long b = (count + 255) / 256;
    return (int)(b < kGridSms * 16 ? (b > 0 ? b : 1) : kGridSms * 16);
}

}  // namespace

namespace {

struct ZeroRegion {
    void *p;
    size_t bytes;
};

__global__ void __launch_bounds__(256) k_zero(ZeroRegion r0, ZeroRegion r1, ZeroRegion r2) {
    pdl_entry();
    const size_t tid = (size_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (size_t)gridDim.x * blockDim.x;
    const ZeroRegion rs[3] = {r0, r1, r2};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const ZeroRegion r = rs[k];
        if (!r.p || r.bytes == 0) continue;
        if ((reinterpret_cast<uintptr_t>(r.p) & 15) == 0 && (r.bytes & 15) == 0) {
            uint4 *q = reinterpret_cast<uint4 *>(r.p);
            for (size_t i = tid; i < r.bytes / 16; i += stride) q[i] = make_uint4(0, 0, 0, 0);
        } else {
            uint32_t *q = reinterpret_cast<uint32_t *>(r.p);
            for (size_t i = tid; i < r.bytes / 4; i += stride) q[i] = 0u;
        }
    }
}

}  // namespace

cudaError_t launch_zero(cudaStream_t st, void *p0, size_t b0, void *p1, size_t b1, void *p2, size_t b2) {
    const size_t words = (b0 + b1 + b2) / 16 + 1;
    const int blocks = (int)std::min<size_t>((words + 255) / 256, kGridSms * 8);
    launch_k(k_zero, blocks, 256, 0, st, ZeroRegion{p0, b0}, ZeroRegion{p1, b1}, ZeroRegion{p2, b2});
    return cudaGetLastError();
}

cudaError_t launch_l1_loss(const float *image, const float *target, int count, float *dL, float *loss,
                           cudaStream_t st) {
    cudaError_t e = launch_zero(st, loss, sizeof(float));
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    launch_k(k_l1_loss, grid_for((count + 3) / 4), 256, 0, st, image, target, count, 1.0f / (float)count, dL, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(const darb_train_params &p, const darb_splat_grads &g, const darb_adam_state &s,
                        const darb_adam_config &c, cudaStream_t st) {
    const long long n = p.n;
    if (n == 0) return cudaSuccess;
    const AdamConsts ac = make_adam_consts(c);
    const float ibc1 = ac.ibc1, ibc2 = ac.ibc2;
    const float b1 = c.beta1, b2 = c.beta2, eps = c.eps;
    const long long K = (long long)(p.sh_degree + 1) * (p.sh_degree + 1);
    auto g4 = [](long long count) { return grid_for((count + 3) / 4); };
    launch_k(k_adam4<0, 0, 0>, g4(3 * n), 256, 0, st, 3 * n, p.means, g.dmeans, s.m_means, s.v_means, c.lr_means,
             c.lr_means, b1, b2, eps, ibc1, ibc2, nullptr);
    launch_k(k_adam4<1, 0, 0>, g4(3 * n), 256, 0, st, 3 * n, p.log_scales, g.dscales, s.m_scales, s.v_scales, c.lr_scales,
             c.lr_scales, b1, b2, eps, ibc1, ibc2, p.scales);
    launch_k(k_adam4<0, 0, 0>, g4(4 * n), 256, 0, st, 4 * n, p.quats, g.dquats, s.m_quats, s.v_quats, c.lr_quats,
             c.lr_quats, b1, b2, eps, ibc1, ibc2, nullptr);
    launch_k(k_adam4<2, 0, 0>, g4(n), 256, 0, st, n, p.opacity_logits, g.dopacities, s.m_opac, s.v_opac, c.lr_opacities,
             c.lr_opacities, b1, b2, eps, ibc1, ibc2, p.opacities);
    const long long cs = 3 * K * n;
    switch (p.sh_degree) {
    case 0:
        launch_k(k_adam_rows<3, 3>, grid_for(cs), 256, 0, st, cs, p.sh, g.dsh, s.m_sh, s.v_sh, c.lr_sh_dc, c.lr_sh_rest, b1,
                 b2, eps, ibc1, ibc2);
        break;
    case 1:
        launch_k(k_adam4<0, 12, 3>, g4(cs), 256, 0, st, cs, p.sh, g.dsh, s.m_sh, s.v_sh, c.lr_sh_dc, c.lr_sh_rest, b1, b2,
                 eps, ibc1, ibc2, nullptr);
        break;
    case 2:
        launch_k(k_adam_rows<27, 3>, grid_for(cs), 256, 0, st, cs, p.sh, g.dsh, s.m_sh, s.v_sh, c.lr_sh_dc, c.lr_sh_rest, b1,
                 b2, eps, ibc1, ibc2);
        break;
    default:
        launch_k(k_adam4<0, 48, 3>, g4(cs), 256, 0, st, cs, p.sh, g.dsh, s.m_sh, s.v_sh, c.lr_sh_dc, c.lr_sh_rest, b1, b2,
                 eps, ibc1, ibc2, nullptr);
        break;
    }
    return cudaGetLastError();
}

}  // namespace darb
