// psi by the moment integral (Sec. A.2): for a kernel F of q = d_M^2, the projected 2D
// density of the truncated 3D kernel with covariance Sigma has covariance psi times the EWA
// block, psi being the per-axis second moment of F(|x|^2) on its support,
//     psi = (1/3) int_0^R r^4 F(r^2) dr / int_0^R r^2 F(r^2) dr,   R = sqrt(q_max).
// The two integrals are sums over 2^22 midpoints, evaluated in FP64 (one-off, so the FP64
// rate does not matter) and reduced per block, then across blocks with double atomics.
#include "kernels.cuh"

namespace darb {
namespace {

constexpr long long kPsiSamples = 1ll << 22;
constexpr int kPsiThreads = 256;

struct PsiKernel {
    int kind, base;
    double xi, beta;
};

__device__ double F64(const PsiKernel &k, double q) {
    const double pi = kPiD;
    switch (k.kind) {
    case DARB_GAUSSIAN: return exp(-0.5 * q);
    case DARB_HALF_COSINE: return cos(pi * q / 18.0);
    case DARB_RAISED_COSINE: return 0.5 + 0.5 * cos(pi * sqrt(q) / 2.5);
    case DARB_MOD_SINC: {
        const double x = pi * sqrt(q) / 3.0;
        return x == 0.0 ? 1.0 : fabs(sin(x)) / x;
    }
    case DARB_INV_QUADRIC: return 1.0 / (1.0 + q);
    case DARB_INV_MULTIQUADRIC: return 1.0 / sqrt(1.0 + q);
    case DARB_PARABOLA: return 1.0 - q / 9.0;
    default: {
        const double u = q > 0.0 ? pow(q, 0.5 * k.beta) / k.xi : 0.0;
        switch (k.base) {
        case 0: return exp(-u);
        case 1: return cos(u);
        case 2: return 0.5 + 0.5 * cos(u);
        case 3: return u == 0.0 ? 1.0 : fabs(sin(u)) / u;
        case 4: return 1.0 / sqrt(u + 1.0);
        default: return 1.0 - u;
        }
    }
    }
}

__global__ void __launch_bounds__(kPsiThreads)
k_psi_moment(PsiKernel k, double rmax, double *__restrict__ sums) {
    pdl_entry();
    __shared__ double s4[kPsiThreads / 32], s2[kPsiThreads / 32];
    const double h = rmax / (double)kPsiSamples;
    double a4 = 0.0, a2 = 0.0;
    for (long long i = (long long)blockIdx.x * kPsiThreads + threadIdx.x; i < kPsiSamples;
         i += (long long)gridDim.x * kPsiThreads) {
        const double r = ((double)i + 0.5) * h, r2 = r * r;
        const double f = F64(k, r2) * r2;
        a2 += f;
        a4 += f * r2;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a4 += __shfl_xor_sync(0xffffffffu, a4, o);
        a2 += __shfl_xor_sync(0xffffffffu, a2, o);
    }
    if ((threadIdx.x & 31) == 0) {
        s4[threadIdx.x >> 5] = a4;
        s2[threadIdx.x >> 5] = a2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t4 = 0.0, t2 = 0.0;
        for (int w = 0; w < kPsiThreads / 32; ++w) {
            t4 += s4[w];
            t2 += s2[w];
        }
        atomicAdd(&sums[0], t4 * h);
        atomicAdd(&sums[1], t2 * h);
    }
}

}  // namespace

cudaError_t launch_psi_moment(const darb_kernel_params &kp, double *sums, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(sums, 0, 2 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const PsiKernel k{kp.kind, kp.base, (double)kp.xi, (double)kp.beta};
    launch_k(k_psi_moment, kGridSms * 4, kPsiThreads, 0, st, k, std::sqrt((double)kp.q_max), sums);
    return cudaGetLastError();
}

}  // namespace darb
