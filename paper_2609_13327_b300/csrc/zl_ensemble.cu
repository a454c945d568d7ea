// Standardized forecast ensemble (the application of Sec. 2.2): the forecast
// perturbations (e_j - mean) / sqrt(K_f - 1) mapped by the left inverse Zh^-
// (the standardized variables transform of Sec. 2.1, with Zh^- standing for
// (P^c)^{-1/2}).  Their outer products sum to the standardized ensemble
// covariance P~^e = (P^c)^{-1/2} P^e (P^c)^{-1/2 T} that the suggested Hybrid
// of Sec. 2.2 localizes.
//
// Zh^- is linear, so the members are mapped first (the left inverse with the
// K_f members as right-hand sides, whichever kernels the plan uses) and the
// centring and scaling are done afterwards on the K_f x K x L coefficients by
// one small kernel: no buffer beyond the caller's output is needed.

#include "zl_internal.cuh"

#include <cmath>

namespace {

// xt[j][e] <- (xt[j][e] - mean_j xt[j][e]) * scale for e < n (mean over the K_f rows,
// accumulated in FP64); one thread per coefficient e, rows read coalesced.
template <typename T>
__global__ void center_scale_kernel(T* __restrict__ xt, int Kf, long long n, double scale) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        double mean = 0.0;
        for (int j = 0; j < Kf; ++j) mean += (double)xt[(long long)j * n + e];
        mean /= Kf;
        for (int j = 0; j < Kf; ++j) xt[(long long)j * n + e] = (T)(((double)xt[(long long)j * n + e] - mean) * scale);
    }
}

}  // namespace

extern "C" zl_status zl_standardize_ensemble(zl_plan p, const void* members, void* xt, int Kf, void* stream) {
    if (p == nullptr || members == nullptr || xt == nullptr || Kf < 2 || members == xt) return ZL_ERR_ARG;
    const zl_status st = zl_apply_left_inverse(p, members, xt, Kf, stream);
    if (st != ZL_OK) return st;
    const long long n = (long long)p->d.K * p->L;
    const double scale = 1.0 / std::sqrt((double)(Kf - 1));
    const int threads = 256;
    const long long want = (n + threads - 1) / threads;
    const int blocks = (int)(want < 4096 ? want : 4096);
    cudaStream_t s = (cudaStream_t)stream;
    if (p->d.prec == ZL_FP64)
        center_scale_kernel<double><<<blocks, threads, 0, s>>>(static_cast<double*>(xt), Kf, n, scale);
    else
        center_scale_kernel<float><<<blocks, threads, 0, s>>>(static_cast<float*>(xt), Kf, n, scale);
    return cudaGetLastError() == cudaSuccess ? ZL_OK : ZL_ERR_CUDA;
}
