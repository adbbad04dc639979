// Training-step kernels: the L1 photometric loss term (paper Sec. 4.2) and the Adam update of
// the 3DGS optimiser (Sec. 5: original 3DGS hyper-parameters, opacity learning rate 0.02).
// Both are elementwise and HBM-bound; float4 accesses where the layout allows.
#include "kernels.cuh"

namespace darb {

namespace {

__global__ void __launch_bounds__(256)
k_l1_loss(const float *__restrict__ image, const float *__restrict__ target, int count, float inv_count,
          float *__restrict__ dL, float *__restrict__ loss) {
    __shared__ float s_warp[8];
    float acc = 0.0f;
    for (int i = blockIdx.x * 256 + threadIdx.x; i < count; i += gridDim.x * 256) {
        const float d = image[i] - target[i];
        dL[i] = d > 0.0f ? inv_count : (d < 0.0f ? -inv_count : 0.0f);
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
// lr2 applies to the elements whose index within a row of `row` floats is >= split (SH rest).
__global__ void __launch_bounds__(256)
k_adam(long long count, float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
       float *__restrict__ v, float lr, float lr2, int row, int split, float b1, float b2, float eps,
       float bc1, float bc2, int act, float *__restrict__ activated) {
    for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < count; i += (long long)gridDim.x * 256) {
        float grad = g[i];
        if (act == 1) grad *= activated[i];
        else if (act == 2) {
            const float o = activated[i];
            grad *= o * (1.0f - o);
        }
        const float mi = b1 * m[i] + (1.0f - b1) * grad;
        const float vi = b2 * v[i] + (1.0f - b2) * grad * grad;
        m[i] = mi;
        v[i] = vi;
        const float step = (row > 0 && (int)(i % row) >= split) ? lr2 : lr;
        const float pi = p[i] - step * (mi / bc1) / (sqrtf(vi / bc2) + eps);
        p[i] = pi;
        if (act == 1) activated[i] = expf(pi);
        else if (act == 2) activated[i] = 1.0f / (1.0f + expf(-pi));
    }
}

int grid_for(long long count) {
    long long b = (count + 255) / 256;
    return (int)(b < 152 * 16 ? (b > 0 ? b : 1) : 152 * 16);
}

}  // namespace

cudaError_t launch_l1_loss(const float *image, const float *target, int count, float *dL, float *loss,
                           cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), st);
    if (e != cudaSuccess) return e;
    if (count == 0) return cudaSuccess;
    k_l1_loss<<<grid_for(count), 256, 0, st>>>(image, target, count, 1.0f / (float)count, dL, loss);
    return cudaGetLastError();
}

cudaError_t launch_adam(const darb_train_params &p, const darb_splat_grads &g, const darb_adam_state &s,
                        const darb_adam_config &c, cudaStream_t st) {
    const long long n = p.n;
    if (n == 0) return cudaSuccess;
    const float bc1 = 1.0f - powf(c.beta1, (float)c.step);
    const float bc2 = 1.0f - powf(c.beta2, (float)c.step);
    const long long K = (long long)(p.sh_degree + 1) * (p.sh_degree + 1);
    struct Group {
        long long count;
        float *p;
        const float *g;
        float *m, *v;
        float lr, lr2;
        int row, split, act;
        float *activated;
    } groups[5] = {
        {3 * n, p.means, g.dmeans, s.m_means, s.v_means, c.lr_means, c.lr_means, 0, 0, 0, nullptr},
        {3 * n, p.log_scales, g.dscales, s.m_scales, s.v_scales, c.lr_scales, c.lr_scales, 0, 0, 1, p.scales},
        {4 * n, p.quats, g.dquats, s.m_quats, s.v_quats, c.lr_quats, c.lr_quats, 0, 0, 0, nullptr},
        {n, p.opacity_logits, g.dopacities, s.m_opac, s.v_opac, c.lr_opacities, c.lr_opacities, 0, 0, 2, p.opacities},
        {3 * K * n, p.sh, g.dsh, s.m_sh, s.v_sh, c.lr_sh_dc, c.lr_sh_rest, (int)(3 * K), 3, 0, nullptr},
    };
    for (const Group &gr : groups) {
        k_adam<<<grid_for(gr.count), 256, 0, st>>>(gr.count, gr.p, gr.g, gr.m, gr.v, gr.lr, gr.lr2, gr.row, gr.split,
                                                   c.beta1, c.beta2, c.eps, bc1, bc2, gr.act, gr.activated);
    }
    return cudaGetLastError();
}

}  // namespace darb
