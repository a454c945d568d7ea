// Matrix-form diagnostics of the paper's experiment, on the GPU:
//
//   column_svd   the per-column singular value decomposition A_m = E_m Lambda_m F_m^T
//                (Eq. svdOfAm, Sec. 3.9) of every grid column's n_w x K matrix, in FP64,
//                by one-sided (Hestenes) Jacobi rotations;
//   xi           the matrix-form accuracy indicators of Sec. 4.8: Xi = I - M M^T for
//                M = Zh^- Zh (Eq. MatrixDifferenceSwiftAlgorithm with Ph = Zh Zh^T),
//                reduced to ||Xi||_F and max |Xi_ij|;
//   delta        the vector-form indicator of Sec. 4.9: d = x~ - Zh^- Zh x~ and ||d||_2
//                per right-hand side (Eq. vectorDifferencedelta, RMSEdelta).
//
// One-sided Jacobi.  With B the p x q matrix whose q columns are to be made orthogonal
// (B = A_m when n_w >= K, B = A_m^T otherwise, so q = min(n_w, K) = g), each rotation of a
// column pair (i, j) zeroes b_i . b_j; the product of the rotations V (q x q) gives
// B V = U Sigma with orthogonal columns.  Sigma holds the column norms, U the normalised
// columns.  For B = A_m: E_m = U, F_m = V; for B = A_m^T: E_m = V, F_m = U.  A warp owns
// one grid column; a sweep visits every pair once in the round-robin order, q / 2
// disjoint pairs per step (one per lane), so a lane's rotation never touches another
// lane's columns.  Sweeps stop when no pair needed a rotation or after kMaxSweeps.
// The singular values are returned in descending order, and each singular pair's sign is
// fixed so that the entry of largest magnitude of F_m's column is positive.

#include "zl_internal.cuh"

#include <algorithm>

namespace zl {

namespace {

constexpr int kMaxSweeps = 40;
constexpr int kSvdMaxQ = 64;          // g = min(n_w, K) <= 64 (two columns per lane)

__device__ __forceinline__ void rr_pair(int step, int slot, int qe, int& i, int& j) {
    // round-robin tournament on qe (even) players: player qe - 1 stays, the others rotate
    const int n = qe - 1;
    if (slot == 0) {
        i = n;
        j = step % n;
    } else {
        i = (step + slot) % n;
        j = (step - slot + n) % n;
    }
    if (i > j) {
        const int t = i;
        i = j;
        j = t;
    }
}

template <typename T>
__global__ void column_svd_kernel(const T* __restrict__ Z, int K, int nw, long long nh, int wpc,
                                  double* __restrict__ E, double* __restrict__ Lam, double* __restrict__ F) {
    extern __shared__ double sm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long m = (long long)blockIdx.x * wpc + warp;
    const bool tall = nw >= K;                 // B = A_m (p = n_w, q = K) or A_m^T (p = K, q = n_w)
    const int p = tall ? nw : K, q = tall ? K : nw;
    const int qe = q + (q & 1);                // even number of players (a dummy column when q is odd)
    double* B = sm + (size_t)warp * ((size_t)p * qe + (size_t)qe * qe);   // [p][qe], row-major
    double* V = B + (size_t)p * qe;                                       // [qe][qe]
    if (m >= nh) return;
    // load: B[r][c] = A_m[r][c] (tall) or A_m[c][r]; A_m[l][k] = Z[k][l][m]
    for (int e = lane; e < p * qe; e += 32) {
        const int r = e / qe, c = e - r * qe;
        double v = 0.0;
        if (c < q) v = tall ? (double)Z[((long long)c * nw + r) * nh + m] : (double)Z[((long long)r * nw + c) * nh + m];
        B[e] = v;
    }
    for (int e = lane; e < qe * qe; e += 32) V[e] = (e / qe == e % qe) ? 1.0 : 0.0;
    __syncwarp();
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        int rotated = 0;
        for (int step = 0; step < qe - 1; ++step) {
            for (int slot = lane; slot < qe / 2; slot += 32) {
                int i, j;
                rr_pair(step, slot, qe, i, j);
                if (j >= q) continue;          // the dummy column
                double a = 0.0, b = 0.0, g = 0.0;
                for (int r = 0; r < p; ++r) {
                    const double x = B[r * qe + i], y = B[r * qe + j];
                    a = fma(x, x, a);
                    b = fma(y, y, b);
                    g = fma(x, y, g);
                }
                if (g == 0.0 || fabs(g) <= 1e-15 * sqrt(a * b)) continue;
                const double zeta = (b - a) / (2.0 * g);
                const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int r = 0; r < p; ++r) {
                    const double x = B[r * qe + i], y = B[r * qe + j];
                    B[r * qe + i] = c * x - s * y;
                    B[r * qe + j] = s * x + c * y;
                }
                for (int r = 0; r < q; ++r) {
                    const double x = V[r * qe + i], y = V[r * qe + j];
                    V[r * qe + i] = c * x - s * y;
                    V[r * qe + j] = s * x + c * y;
                }
                rotated = 1;
            }
            __syncwarp();
        }
        if (!__any_sync(0xffffffffu, rotated)) break;
    }
    // singular values (column norms), their descending rank, and the sign of each pair
    const int g = q;
    double sig[2] = {0.0, 0.0};
    int rank[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c < g) {
            double a = 0.0;
            for (int r = 0; r < p; ++r) a = fma(B[r * qe + c], B[r * qe + c], a);
            sig[h] = sqrt(a);
        }
    }
    // rank of column c = number of columns with a larger norm (ties broken by index)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        int rk = 0;
        for (int o = 0; o < g; ++o) {
            const double so = __shfl_sync(0xffffffffu, sig[o >> 5], o & 31);
            if (c < g && (so > sig[h] || (so == sig[h] && o < c))) ++rk;
        }
        rank[h] = rk;
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int c = lane + 32 * h;
        if (c >= g) continue;
        const int o = rank[h];
        const double sv = sig[h];
        const double inv = sv > 0.0 ? 1.0 / sv : 0.0;
        // F column: tall -> V[:, c] (length K); wide -> B[:, c] / sigma (length K)
        double fmax = 0.0, fsgn = 1.0;
        for (int k = 0; k < K; ++k) {
            const double v = tall ? V[k * qe + c] : B[k * qe + c] * inv;
            if (fabs(v) > fmax) {
                fmax = fabs(v);
                fsgn = v < 0.0 ? -1.0 : 1.0;
            }
        }
        Lam[m * g + o] = sv;
        for (int k = 0; k < K; ++k) {
            const double v = tall ? V[k * qe + c] : B[k * qe + c] * inv;
            F[(m * K + k) * g + o] = fsgn * v;
        }
        for (int l = 0; l < nw; ++l) {
            const double v = tall ? B[l * qe + c] * inv : V[l * qe + c];
            E[(m * nw + l) * g + o] = fsgn * v;
        }
    }
}

// Xi = I - M M^T (n x n, M row-major): each block forms a 32 x 32 tile of Xi and folds
// its squares and absolute values into acc[0] (sum) and acc[1] (max, as ordered bits).
constexpr int kXiTile = 32;

__global__ void xi_kernel(const double* __restrict__ M, int n, double* __restrict__ acc) {
    __shared__ double a[kXiTile][kXiTile + 1], b[kXiTile][kXiTile + 1];
    __shared__ double red_s[8], red_m[8];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads, 4 rows each
    const int i0 = blockIdx.y * kXiTile, j0 = blockIdx.x * kXiTile;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int k0 = 0; k0 < n; k0 += kXiTile) {
        for (int r = ty; r < kXiTile; r += 8) {
            a[r][tx] = (i0 + r < n && k0 + tx < n) ? M[(long long)(i0 + r) * n + k0 + tx] : 0.0;
            b[r][tx] = (j0 + r < n && k0 + tx < n) ? M[(long long)(j0 + r) * n + k0 + tx] : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < kXiTile; ++k) {
            const double bv = b[tx][k];
#pragma unroll
            for (int u = 0; u < 4; ++u) s[u] = fma(a[ty + 8 * u][k], bv, s[u]);
        }
        __syncthreads();
    }
    double sq = 0.0, mx = 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int i = i0 + ty + 8 * u, j = j0 + tx;
        if (i < n && j < n) {
            const double xi = (i == j ? 1.0 : 0.0) - s[u];
            sq = fma(xi, xi, sq);
            mx = fmax(mx, fabs(xi));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        sq += __shfl_xor_sync(0xffffffffu, sq, o);
        mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (tx == 0) {
        red_s[ty] = sq;
        red_m[ty] = mx;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double ts = 0.0, tm = 0.0;
        for (int w = 0; w < 8; ++w) {
            ts += red_s[w];
            tm = fmax(tm, red_m[w]);
        }
        atomicAdd(&acc[0], ts);
        // non-negative doubles order like their bit patterns
        atomicMax(reinterpret_cast<unsigned long long*>(&acc[1]), (unsigned long long)__double_as_longlong(tm));
    }
}

// d = xt - back per element and ||d_r||_2 per right-hand side (one block per right-hand side)
template <typename T>
__global__ void delta_kernel(const T* __restrict__ xt, const T* __restrict__ back, T* __restrict__ d,
                             double* __restrict__ norms, long long len) {
    __shared__ double red[32];
    const long long base = (long long)blockIdx.x * len;
    double s = 0.0;
    for (long long i = threadIdx.x; i < len; i += blockDim.x) {
        const T v = xt[base + i] - back[base + i];
        d[base + i] = v;
        s = fma((double)v, (double)v, s);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        norms[blockIdx.x] = sqrt(t);
    }
}

// xt[row][j] = partial[row][j] * scale[j] (rows = (rhs, member) pairs); in place allowed
template <typename T>
__global__ void scale_modes_kernel(const T* partial, const T* __restrict__ scale, T* xt, long long rows, int L) {
    const long long total = rows * L;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x)
        xt[i] = partial[i] * scale[i % L];
}

}  // namespace

template <typename T>
cudaError_t launch_scale_modes(const T* partial, const T* scale, T* xt, long long rows, int L, cudaStream_t s) {
    const long long total = rows * L;
    const int grid = (int)std::min<long long>((total + 255) / 256, 148 * 16);
    scale_modes_kernel<T><<<grid, 256, 0, s>>>(partial, scale, xt, rows, L);
    return cudaGetLastError();
}

template cudaError_t launch_scale_modes<double>(const double*, const double*, double*, long long, int, cudaStream_t);
template cudaError_t launch_scale_modes<float>(const float*, const float*, float*, long long, int, cudaStream_t);

size_t column_svd_smem_per_warp(int nw, int K) {
    const int p = std::max(nw, K), q = std::min(nw, K);
    const int qe = q + (q & 1);
    return ((size_t)p * qe + (size_t)qe * qe) * sizeof(double);
}

cudaError_t launch_column_svd(const zl_plan_s& p, double* E, double* Lam, double* F, cudaStream_t s) {
    if (std::min(p.d.nw, p.d.K) > kSvdMaxQ) return cudaErrorInvalidValue;
    const size_t per = column_svd_smem_per_warp(p.d.nw, p.d.K);
    int wpc = (int)std::min<size_t>(8, (200 * 1024) / per);
    if (wpc < 1) return cudaErrorInvalidValue;
    const size_t smem = per * wpc;
    const int grid = (int)((p.nh + wpc - 1) / wpc);
    cudaError_t e;
    if (p.d.prec == ZL_FP64) {
        e = cudaFuncSetAttribute(column_svd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        column_svd_kernel<double><<<grid, 32 * wpc, smem, s>>>(reinterpret_cast<const double*>(p.Zc), p.d.K, p.d.nw,
                                                                p.nh, wpc, E, Lam, F);
    } else {
        e = cudaFuncSetAttribute(column_svd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        column_svd_kernel<float><<<grid, 32 * wpc, smem, s>>>(reinterpret_cast<const float*>(p.Zc), p.d.K, p.d.nw,
                                                               p.nh, wpc, E, Lam, F);
    }
    return cudaGetLastError();
}

cudaError_t launch_xi(const double* M, int n, double* acc, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc, 0, 2 * sizeof(double), s);
    if (e != cudaSuccess) return e;
    const int t = (n + kXiTile - 1) / kXiTile;
    xi_kernel<<<dim3(t, t), 256, 0, s>>>(M, n, acc);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_delta(const T* xt, const T* back, T* d, double* norms, long long len, int R, cudaStream_t s) {
    delta_kernel<T><<<R, 256, 0, s>>>(xt, back, d, norms, len);
    return cudaGetLastError();
}

template cudaError_t launch_delta<double>(const double*, const double*, double*, double*, long long, int, cudaStream_t);
template cudaError_t launch_delta<float>(const float*, const float*, float*, double*, long long, int, cudaStream_t);

}  // namespace zl
