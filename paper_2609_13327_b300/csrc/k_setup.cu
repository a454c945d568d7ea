// Setup: the per-column pseudo-inverse A_m^+ in FP64 (one CTA per grid column).
//
// The paper factorises every column matrix A_m (n_w x K, A_m[l][k] = Z[k][l][m],
// Sec. 3.9) by an SVD and applies A_m^{-1} = F_m Lambda_m^{-1} E_m^T in step V1
// (Sec. 3.10).  Here the same operator is formed once per column as a dense
// K x n_w matrix P_m = A_m^+ so that every apply is a single product:
//
//   1. Gram     G_m = A_m A_m^T (n_w <= K)  or  A_m^T A_m (n_w > K), g = min(n_w, K)
//   2. Cholesky G_m = L_m L_m^T; a pivot <= rank_eps * trace(G_m) marks column m
//               rank-deficient (rank(A) = sum_m rank(A_m), supporting info S2)
//   3. solve    P0 = A_m^T G_m^{-1}  (n_w <= K)   or   G_m^{-1} A_m^T  (n_w > K)
//   4. refine   one Newton step with the residual in FP64:
//               E = A_m P0 - I,  P = P0 - P0 E    (n_w <= K)
//               E = P0 A_m - I,  P = P0 - E P0    (n_w > K)
//               The Gram route alone loses cond(A_m)^2 * eps; after the step
//               the error is back at the cond(A_m) * eps of the paper's SVD.
//
// FP64 on the B300 is slow, but this runs once per plan: O(n_w K g) flops per column.

#include "zl_internal.cuh"

#include <climits>

namespace zl {

namespace {

constexpr double kRankEps = 1e-13;
constexpr int kSetupThreads = 128;

__device__ __forceinline__ double load_as_double(const double* p) { return *p; }
__device__ __forceinline__ double load_as_double(const float* p) { return (double)*p; }
__device__ __forceinline__ void store_from_double(double* p, double v) { *p = v; }
__device__ __forceinline__ void store_from_double(float* p, double v) { *p = (float)v; }

// Shared-memory layout (doubles): A [nw][K] (later overwritten by P^T), G [g][g]
// (later E), PT [nw][K] (P0^T: PT[l][k] = P0[k][l]).
template <typename TZ>
__global__ void __launch_bounds__(kSetupThreads)
setup_columns_kernel(const TZ* __restrict__ Z, TZ* __restrict__ P, int K, int nw, long long nh,
                     int* __restrict__ status) {
    extern __shared__ double sm[];
    const int g = nw <= K ? nw : K;
    double* A = sm;
    double* G = A + (size_t)nw * K;
    double* PT = G + (size_t)g * g;
    __shared__ double s_trace;
    __shared__ int s_bad;

    const long long m = blockIdx.x;
    const int tid = threadIdx.x, nt = blockDim.x;

    for (int i = tid; i < nw * K; i += nt) {
        const int l = i / K, k = i - l * K;
        A[i] = load_as_double(Z + ((long long)k * nw + l) * nh + m);
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();

    // 1. Gram (lower triangle)
    for (int e = tid; e < g * g; e += nt) {
        const int i = e / g, j = e - i * g;
        if (j > i) continue;
        double acc = 0.0;
        if (nw <= K) {
            for (int k = 0; k < K; ++k) acc = fma(A[i * K + k], A[j * K + k], acc);
        } else {
            for (int l = 0; l < nw; ++l) acc = fma(A[l * K + i], A[l * K + j], acc);
        }
        G[i * g + j] = acc;
    }
    __syncthreads();
    if (tid == 0) {
        double tr = 0.0;
        for (int i = 0; i < g; ++i) tr += G[i * g + i];
        s_trace = tr;
    }
    __syncthreads();

    // 2. left-looking Cholesky, in place in the lower triangle of G
    for (int j = 0; j < g; ++j) {
        if (tid == 0) {
            double d = G[j * g + j];
            for (int p = 0; p < j; ++p) d = fma(-G[j * g + p], G[j * g + p], d);
            if (!(d > kRankEps * s_trace)) {
                s_bad = 1;
                d = 1.0;
            }
            G[j * g + j] = sqrt(d);
        }
        __syncthreads();
        if (s_bad) break;
        const double piv = G[j * g + j];
        for (int i = j + 1 + tid; i < g; i += nt) {
            double v = G[i * g + j];
            for (int p = 0; p < j; ++p) v = fma(-G[i * g + p], G[j * g + p], v);
            G[i * g + j] = v / piv;
        }
        __syncthreads();
    }
    if (s_bad) {
        if (tid == 0) atomicMin(status, (int)m);
        return;
    }

    // 3. P0 by forward/back substitution, one right-hand side per thread
    if (nw <= K) {
        // G Y = A_m, Y is nw x K: column k of Y is row k of P0, stored PT[l][k]
        for (int k = tid; k < K; k += nt) {
            for (int i = 0; i < g; ++i) {
                double v = A[i * K + k];
                for (int p = 0; p < i; ++p) v = fma(-G[i * g + p], PT[p * K + k], v);
                PT[i * K + k] = v / G[i * g + i];
            }
            for (int i = g - 1; i >= 0; --i) {
                double v = PT[i * K + k];
                for (int p = i + 1; p < g; ++p) v = fma(-G[p * g + i], PT[p * K + k], v);
                PT[i * K + k] = v / G[i * g + i];
            }
        }
    } else {
        // G Y = A_m^T, Y is K x nw: column l of Y is column l of P0, stored PT[l][k]
        for (int l = tid; l < nw; l += nt) {
            double* y = PT + (size_t)l * K;
            for (int i = 0; i < g; ++i) {
                double v = A[l * K + i];
                for (int p = 0; p < i; ++p) v = fma(-G[i * g + p], y[p], v);
                y[i] = v / G[i * g + i];
            }
            for (int i = g - 1; i >= 0; --i) {
                double v = y[i];
                for (int p = i + 1; p < g; ++p) v = fma(-G[p * g + i], y[p], v);
                y[i] = v / G[i * g + i];
            }
        }
    }
    __syncthreads();

    // 4. one Newton step; E (g x g) overwrites G, the refined P^T overwrites A
    if (nw <= K) {
        for (int e = tid; e < g * g; e += nt) {
            const int i = e / g, j = e - i * g;    // E[i][j] = sum_k A[i][k] P0[k][j] - delta_ij
            double acc = (i == j) ? -1.0 : 0.0;
            for (int k = 0; k < K; ++k) acc = fma(A[i * K + k], PT[j * K + k], acc);
            G[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < nw * K; e += nt) {
            const int j = e / K, k = e - j * K;    // P[k][j] = P0[k][j] - sum_i P0[k][i] E[i][j]
            double acc = PT[j * K + k];
            for (int i = 0; i < nw; ++i) acc = fma(-PT[i * K + k], G[i * g + j], acc);
            A[e] = acc;
        }
    } else {
        for (int e = tid; e < g * g; e += nt) {
            const int i = e / g, j = e - i * g;    // E[i][j] = sum_l P0[i][l] A[l][j] - delta_ij
            double acc = (i == j) ? -1.0 : 0.0;
            for (int l = 0; l < nw; ++l) acc = fma(PT[l * K + i], A[l * K + j], acc);
            G[e] = acc;
        }
        __syncthreads();
        for (int e = tid; e < nw * K; e += nt) {
            const int l = e / K, i = e - l * K;    // P[i][l] = P0[i][l] - sum_j E[i][j] P0[j][l]
            double acc = PT[l * K + i];
            for (int j = 0; j < K; ++j) acc = fma(-G[i * g + j], PT[l * K + j], acc);
            A[e] = acc;
        }
    }
    __syncthreads();

    for (int e = tid; e < nw * K; e += nt) {
        const int l = e / K, k = e - l * K;
        store_from_double(P + ((long long)k * nw + l) * nh + m, A[e]);
    }
}

}  // namespace

size_t setup_smem_bytes(int nw, int K) {
    const size_t g = nw <= K ? nw : K;
    return (2 * (size_t)nw * K + g * g) * sizeof(double);
}

cudaError_t launch_setup_columns(const zl_desc& d, long long nh, const void* Z, void* P, int* d_status,
                                 cudaStream_t s) {
    const size_t smem = setup_smem_bytes(d.nw, d.K);
    cudaError_t e;
    if (d.prec == ZL_FP64) {
        e = cudaFuncSetAttribute(setup_columns_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        setup_columns_kernel<double><<<(unsigned)nh, kSetupThreads, smem, s>>>(
            (const double*)Z, (double*)P, d.K, d.nw, nh, d_status);
    } else {
        e = cudaFuncSetAttribute(setup_columns_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        setup_columns_kernel<float><<<(unsigned)nh, kSetupThreads, smem, s>>>(
            (const float*)Z, (float*)P, d.K, d.nw, nh, d_status);
    }
    return cudaGetLastError();
}

}  // namespace zl
