// CUDA-core kernels of the four operators, templated on the element type
// (double: the plain FP64 GPU form of the algorithm; float: the FP32 path).
//
// All four operators share two shapes.  With M a member matrix stored
// [K][n_w][n_h] (the ensemble Z, or the per-column pseudo-inverse P) and a
// per-mode scale (Delta_b^{-1/2} or Delta_b^{1/2}):
//
//   forward  out[r][k][j] = scale_j * (V_b^T w_k)_{s_j},  w_k[m] = sum_l M[k][l][m] x[r][l][m]
//            left inverse (M = P, Delta^{-1/2}): steps V1-V5 of Sec. 3.10
//            Zh^T         (M = Z, Delta^{+1/2})
//   inverse  out[r][l][m] = sum_k M[k][l][m] y_k[m],  y_k = V_b (scale (.) c_k)
//            square root  (M = Z, Delta^{+1/2}): A V Delta^{1/2} (Sec. 3.9)
//            adjoint      (M = P, Delta^{-1/2}): (A^+)^T V Delta^{-1/2}
//
// V_b^T is applied separably: an x-pass per grid row that keeps only the Px
// x-frequencies that occur among the kept modes (intermediate t1 [R][K][ny][Px]
// in HBM), then a y-pass that forms each kept mode (p_y, p_x) and scales it.
// The x-pass is fused with the per-column product: a CTA owns one grid row, so
// the regrouping of w^(m) into member segments (steps V2-V3, the paper's
// inter-processor exchange) never leaves shared memory.
//
// For FP32 data the TMA-fed persistent column kernels of k_f32.cu take the forward
// and inverse column passes wherever their tiles apply (dispatch in launch_fwd and
// inverse_plain); the kernels here serve FP64 and the remaining FP32 shapes, and the
// FP32 y-passes (fwd_ypass_sgemm, inv_ypass_dense) serve both.

#include "zl_internal.cuh"

#include <algorithm>

namespace zl {

namespace {

constexpr int kThreads = 256;
constexpr int KC = 8;                    // members per CTA in the forward pass
constexpr size_t kRowSmemBudget = 72 * 1024;

// ---------------------------------------------------------------------------
// forward, pass 1: per-column product + x-pass, CTA = (grid row y, RC rhs, KC members)
// ---------------------------------------------------------------------------
template <typename T, int RC>
__global__ void __launch_bounds__(kThreads)
fwd_column_xpass(const T* __restrict__ x, const T* __restrict__ M, const T* __restrict__ bx, T* __restrict__ t1,
                 int R, int nw, int K, int nx, int ny, int Px, int y0, long long nh_m) {
    extern __shared__ unsigned char smem_raw[];
    T* W = reinterpret_cast<T*>(smem_raw);   // [KC][RC][ldw]
    const int ldw = nx + 1;
    // member chunk fastest, then rhs chunk, then grid row: the CTAs that share a
    // row's x and M tiles run back to back and find them in L2.  x holds the ny rows
    // y0 .. y0 + ny - 1 of the grid (all of it when y0 = 0 and ny is the grid's), M the
    // whole grid (nh_m columns); t1 rows are relative to y0.
    const int k0 = blockIdx.x * KC;
    const int r0 = blockIdx.y * RC;
    const int y = blockIdx.z;
    const long long nh = (long long)nx * ny;

    for (int xc = threadIdx.x; xc < nx; xc += blockDim.x) {
        const long long m = (long long)y * nx + xc;
        const long long mm = (long long)(y0 + y) * nx + xc;
        T acc[RC][KC];
#pragma unroll
        for (int r = 0; r < RC; ++r)
#pragma unroll
            for (int k = 0; k < KC; ++k) acc[r][k] = T(0);
        for (int l = 0; l < nw; ++l) {
            T xv[RC];
#pragma unroll
            for (int r = 0; r < RC; ++r)
                xv[r] = (r0 + r < R) ? x[((long long)(r0 + r) * nw + l) * nh + m] : T(0);
#pragma unroll
            for (int k = 0; k < KC; ++k) {
                const T pv = (k0 + k < K) ? M[((long long)(k0 + k) * nw + l) * nh_m + mm] : T(0);
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[r][k] = fma(pv, xv[r], acc[r][k]);
            }
        }
#pragma unroll
        for (int k = 0; k < KC; ++k)
#pragma unroll
            for (int r = 0; r < RC; ++r) W[((size_t)k * RC + r) * ldw + xc] = acc[r][k];
    }
    __syncthreads();

    // x-pass, a small GEMM per CTA: t1[r][k][y][jx] = sum_x W[k][r][x] * bx[jx][x].
    // Thread (rg, cg) of a 16 x 16 layout owns rows rg + 16 i (i < 4) and
    // x-frequencies c0 + cg + 16 j (j < 3); W rows are padded to ldw = nx + 1
    // words so the 16 rows a warp reads sit in distinct banks, and the basis
    // rows are read from L1 with two distinct addresses per warp.
    const int rows = KC * RC;
    const int rg = threadIdx.x & 15, cg = threadIdx.x >> 4;
    for (int c0 = 0; c0 < Px; c0 += 48) {
        T acc[4][3][2];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) acc[i][j][0] = acc[i][j][1] = T(0);
        const T* wrow[4];
        const T* brow[3];
#pragma unroll
        for (int i = 0; i < 4; ++i) wrow[i] = W + (size_t)min(rg + 16 * i, rows - 1) * ldw;
#pragma unroll
        for (int j = 0; j < 3; ++j) brow[j] = bx + (size_t)min(c0 + cg + 16 * j, Px - 1) * nx;
        auto step = [&](int xc, int h) {
            T wv[4], bv[3];
#pragma unroll
            for (int i = 0; i < 4; ++i) wv[i] = wrow[i][xc];
#pragma unroll
            for (int j = 0; j < 3; ++j) bv[j] = __ldg(brow[j] + xc);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 3; ++j) acc[i][j][h] = fma(wv[i], bv[j], acc[i][j][h]);
        };
        int xc = 0;
        for (; xc + 1 < nx; xc += 2) {
            step(xc, 0);
            step(xc + 1, 1);
        }
        if (xc < nx) step(xc, 0);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int row = rg + 16 * i;
            const int k = row / RC, r = row - k * RC;
            if (row >= rows || r0 + r >= R || k0 + k >= K) continue;
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int jx = c0 + cg + 16 * j;
                if (jx < Px)
                    t1[(((long long)y * R + r0 + r) * K + k0 + k) * Px + jx] = acc[i][j][0] + acc[i][j][1];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// forward, pass 2: y-pass + scale + compaction, CTA = (member k, rhs r)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
fwd_ypass(const T* __restrict__ t1, const T* __restrict__ by, const int* __restrict__ m_py,
          const int* __restrict__ m_jx, const T* __restrict__ scale, T* __restrict__ out,
          int R, int K, int ny, int Px, int ldp, int L, int ychunk, int by_ld, int y_off) {
    extern __shared__ unsigned char smem_raw[];
    T* acc = reinterpret_cast<T*>(smem_raw);   // [L]
    T* tile = acc + L;                         // [Px][ychunk + 1]: odd stride, conflict-free rows
    const int ldt = ychunk + 1;
    const int k = blockIdx.x, r = blockIdx.y;
    const T* src = t1 + ((long long)r * K + k) * ldp;
    const long long ystride = (long long)R * K * ldp;
    for (int j = threadIdx.x; j < L; j += blockDim.x) acc[j] = T(0);
    for (int y0 = 0; y0 < ny; y0 += ychunk) {
        const int yn = min(ychunk, ny - y0);
        __syncthreads();
        for (int e = threadIdx.x; e < yn * Px; e += blockDim.x) {
            const int yy = e / Px, jx = e - yy * Px;
            tile[jx * ldt + yy] = src[(long long)(y0 + yy) * ystride + jx];
        }
        __syncthreads();
        for (int j = threadIdx.x; j < L; j += blockDim.x) {
            const T* b = by + (size_t)m_py[j] * by_ld + y_off + y0;
            const T* t = tile + (size_t)m_jx[j] * ldt;
            T s0 = 0, s1 = 0;
            int yy = 0;
            for (; yy + 1 < yn; yy += 2) {
                s0 = fma(b[yy], t[yy], s0);
                s1 = fma(b[yy + 1], t[yy + 1], s1);
            }
            if (yy < yn) s0 = fma(b[yy], t[yy], s0);
            acc[j] += s0 + s1;
        }
    }
    __syncthreads();
    T* o = out + ((long long)r * K + k) * L;
    for (int j = threadIdx.x; j < L; j += blockDim.x) o[j] = scale ? acc[j] * scale[j] : acc[j];
}

// ---------------------------------------------------------------------------
// inverse, pass 1: scale + inverse y-pass, CTA = (member k, rhs r)
//   u[r][k][y][jx] = sum_{j in group(jx)} by[py_j][y] * scale_j * c[r][k][j]
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
inv_ypass(const T* __restrict__ c, const T* __restrict__ by, const int* __restrict__ m_py,
          const int* __restrict__ grp_start, const int* __restrict__ grp_modes, const T* __restrict__ scale,
          T* __restrict__ u, int K, int ny, int Px, int L) {
    extern __shared__ unsigned char smem_raw[];
    T* cs = reinterpret_cast<T*>(smem_raw);   // [L]
    const int k = blockIdx.x, r = blockIdx.y;
    const T* src = c + ((long long)r * K + k) * L;
    for (int j = threadIdx.x; j < L; j += blockDim.x) cs[j] = src[j] * scale[j];
    __syncthreads();
    T* dst = u + ((long long)r * K + k) * ny * Px;
    for (int e = threadIdx.x; e < ny * Px; e += blockDim.x) {
        const int yy = e / Px, jx = e - yy * Px;
        T s = 0;
        for (int q = grp_start[jx]; q < grp_start[jx + 1]; ++q) {
            const int j = grp_modes[q];
            s = fma(by[(size_t)m_py[j] * ny + yy], cs[j], s);
        }
        dst[e] = s;
    }
}


// ---------------------------------------------------------------------------
// inverse, pass 1 as a small dense GEMM per (member k, rhs r):
//   u[r][k][y][jx] = sum_i byk[y][i] C[i][jx],  C[i][jx] = scale_j c[r][k][j] for the kept
//   mode j = (i-th kept y-frequency, jx-th kept x-frequency), 0 for the others.
// C is built in shared memory with its columns grouped as [i][jx % 4][jx / 4] so that a
// thread's QJ x-frequencies (jx = g + 4 q, g = its group) are QJ consecutive words; the
// kept y-basis is staged 64 MY rows at a time; thread (rows yy + 64 m for m < MY, group g)
// accumulates its MY x QJ outputs with MY basis loads and QJ / 4 vector loads of C per
// kept y-frequency, and the output tile leaves through shared memory with coalesced
// stores.
// ---------------------------------------------------------------------------
constexpr int kInvYRows = 64;

template <typename T, int QJ, int MY>
__global__ void __launch_bounds__(kThreads)
inv_ypass_dense(const T* __restrict__ c, const T* __restrict__ byk, const int* __restrict__ m_ipy,
                const int* __restrict__ m_jx, const T* __restrict__ scale, T* __restrict__ u, int K, int ny, int Px,
                int L, int Py, int pys) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int CW = 4 * QJ;                           // C row width (x-frequency slots)
    constexpr int YT = kInvYRows * MY;                   // rows of y per tile
    T* C = reinterpret_cast<T*>(smem_raw);               // [Py][4][QJ]
    T* bys = C + (size_t)Py * CW;                        // [YT][Py + 1]
    T* ot = bys + (size_t)YT * (Py + 1);                 // [YT][Px]
    const int k = blockIdx.x, r = blockIdx.y;
    const T* src = c + ((long long)r * K + k) * L;
    for (int e = threadIdx.x; e < Py * CW; e += blockDim.x) C[e] = T(0);
    __syncthreads();
    for (int j = threadIdx.x; j < L; j += blockDim.x) {
        const int jx = m_jx[j];
        C[(size_t)m_ipy[j] * CW + (jx & 3) * QJ + (jx >> 2)] = src[j] * scale[j];
    }
    const int yy = threadIdx.x % kInvYRows, g = threadIdx.x / kInvYRows;   // g = 0..3
    T* dst = u + ((long long)r * K + k) * ny * Px;
    for (int y0 = 0; y0 < ny; y0 += YT) {
        const int yn = min(YT, ny - y0);
        __syncthreads();                                  // C complete; previous tile written out
        for (int e = threadIdx.x; e < yn * Py; e += blockDim.x) {
            const int a = e / Py, i = e - a * Py;
            bys[(size_t)a * (Py + 1) + i] = byk[(size_t)(y0 + a) * pys + i];
        }
        __syncthreads();
        T acc[MY][QJ];
#pragma unroll
        for (int m = 0; m < MY; ++m)
#pragma unroll
            for (int q = 0; q < QJ; ++q) acc[m][q] = T(0);
        const T* crow = C + g * QJ;
        for (int i = 0; i < Py; ++i, crow += CW) {
            T b[MY];
#pragma unroll
            for (int m = 0; m < MY; ++m) b[m] = bys[(size_t)(yy + kInvYRows * m) * (Py + 1) + i];
#pragma unroll
            for (int q = 0; q < QJ; ++q) {
                const T cv = crow[q];
#pragma unroll
                for (int m = 0; m < MY; ++m) acc[m][q] = fma(b[m], cv, acc[m][q]);
            }
        }
#pragma unroll
        for (int m = 0; m < MY; ++m) {
            const int row = yy + kInvYRows * m;
            if (row < yn) {
#pragma unroll
                for (int q = 0; q < QJ; ++q) {
                    const int jx = g + 4 * q;
                    if (jx < Px) ot[(size_t)row * Px + jx] = acc[m][q];
                }
            }
        }
        __syncthreads();
        for (int e = threadIdx.x; e < yn * Px; e += blockDim.x) dst[(size_t)y0 * Px + e] = ot[e];
    }
}

template <typename T, int QJ, int MY>
size_t inv_ypass_dense_smem(const zl_plan_s& p) {
    return ((size_t)p.Py * 4 * QJ + (size_t)kInvYRows * MY * (p.Py + 1) + (size_t)kInvYRows * MY * p.Px) * sizeof(T);
}

template <typename T, int QJ, int MY>
cudaError_t launch_inv_ypass_dense_my(const zl_plan_s& p, const Tables<T>& t, const T* scale, const T* c, T* u, int R,
                                      cudaStream_t s) {
    const size_t smem = inv_ypass_dense_smem<T, QJ, MY>(p);
    cudaError_t e = cudaFuncSetAttribute(inv_ypass_dense<T, QJ, MY>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    inv_ypass_dense<T, QJ, MY><<<dim3(p.d.K, R), kThreads, smem, s>>>(c, t.byk, t.m_ipy, t.m_jx, scale, u, p.d.K,
                                                                       p.d.ny, p.Px, p.L, p.Py, p.pys);
    return cudaGetLastError();
}

// rows per thread: 2 when the grid has 128 rows or more and the tile fits two CTAs per SM,
// else 1 (4 rows per thread, with fewer CTAs per SM, was slower at the larger grids)
template <typename T, int QJ>
cudaError_t launch_inv_ypass_dense(const zl_plan_s& p, const Tables<T>& t, const T* scale, const T* c, T* u, int R,
                                   cudaStream_t s) {
    constexpr size_t kTwoPerSm = 110 * 1024;
    if (p.d.ny >= 2 * kInvYRows && inv_ypass_dense_smem<T, QJ, 2>(p) <= kTwoPerSm)
        return launch_inv_ypass_dense_my<T, QJ, 2>(p, t, scale, c, u, R, s);
    return launch_inv_ypass_dense_my<T, QJ, 1>(p, t, scale, c, u, R, s);
}

// ---------------------------------------------------------------------------
// inverse, pass 2: inverse x-pass + per-column product,
// CTA = (grid row y, column tile, rhs r); one thread per column
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads)
inv_xpass_column(const T* __restrict__ u, const T* __restrict__ M, const T* __restrict__ bx, T* __restrict__ out,
                 int nw, int K, int nx, int ny, int Px) {
    extern __shared__ unsigned char smem_raw[];
    T* us = reinterpret_cast<T*>(smem_raw);   // [K][Px]
    T* ys = us + (size_t)K * Px;              // [K][blockDim]
    const int y = blockIdx.x;
    const int xt = blockIdx.y;
    const int r = blockIdx.z;
    const long long nh = (long long)nx * ny;
    for (int e = threadIdx.x; e < K * Px; e += blockDim.x) {
        const int k = e / Px, jx = e - k * Px;
        us[e] = u[(((long long)r * K + k) * ny + y) * Px + jx];
    }
    __syncthreads();
    const int xc = xt * blockDim.x + threadIdx.x;
    if (xc >= nx) return;
    const long long m = (long long)y * nx + xc;
    for (int k = 0; k < K; ++k) {
        T s = 0;
        for (int jx = 0; jx < Px; ++jx) s = fma(bx[(size_t)jx * nx + xc], us[k * Px + jx], s);
        ys[(size_t)k * blockDim.x + threadIdx.x] = s;
    }
    for (int l = 0; l < nw; ++l) {
        T s0 = 0, s1 = 0;
        int k = 0;
        for (; k + 1 < K; k += 2) {
            s0 = fma(M[((long long)k * nw + l) * nh + m], ys[(size_t)k * blockDim.x + threadIdx.x], s0);
            s1 = fma(M[((long long)(k + 1) * nw + l) * nh + m], ys[(size_t)(k + 1) * blockDim.x + threadIdx.x], s1);
        }
        if (k < K) s0 = fma(M[((long long)k * nw + l) * nh + m], ys[(size_t)k * blockDim.x + threadIdx.x], s0);
        out[((long long)r * nw + l) * nh + m] = s0 + s1;
    }
}


// ---------------------------------------------------------------------------
// inverse, pass 2, several right-hand sides per CTA: CTA = (grid row y, column tile,
// RC right-hand sides), one thread per column.  Member by member, the thread forms
// y_k = sum_jx b_jx(x) u[r][k][y][jx] for its RC right-hand sides (the basis column of
// the thread and the u rows of the CTA staged in shared memory, u with the right-hand
// sides innermost so that one vector load serves them all) and adds M[k][l][m] y_k to
// NWM x RC register accumulators, so every element of M is read once per RC
// right-hand sides instead of once per right-hand side.  NWM >= n_w.
// ---------------------------------------------------------------------------
template <typename T, int NWM, int RC>
__global__ void __launch_bounds__(128)
inv_xpass_column_rc(const T* __restrict__ u, const T* __restrict__ M, const T* __restrict__ bx, T* __restrict__ out,
                    int R, int nw, int K, int nx, int ny, int Px) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* us = reinterpret_cast<T*>(smem_raw);            // [K][Px][RC]
    T* bs = us + (size_t)K * Px * RC;                  // [Px][blockDim]
    const int y = blockIdx.x, xt = blockIdx.y, r0 = blockIdx.z * RC;
    const long long nh = (long long)nx * ny;
    for (int e = threadIdx.x; e < K * Px * RC; e += blockDim.x) {
        const int r = e % RC, kj = e / RC, k = kj / Px, jx = kj - k * Px;
        us[e] = (r0 + r < R) ? u[(((long long)(r0 + r) * K + k) * ny + y) * Px + jx] : T(0);
    }
    const int xc = xt * blockDim.x + threadIdx.x;
    for (int jx = 0; jx < Px; ++jx) bs[(size_t)jx * blockDim.x + threadIdx.x] = xc < nx ? bx[(size_t)jx * nx + xc] : T(0);
    __syncthreads();
    if (xc >= nx) return;
    const long long m = (long long)y * nx + xc;
    T acc[NWM][RC];
#pragma unroll
    for (int l = 0; l < NWM; ++l)
#pragma unroll
        for (int r = 0; r < RC; ++r) acc[l][r] = T(0);
    const T* bcol = bs + threadIdx.x;
    for (int k = 0; k < K; ++k) {
        T yk[RC];
#pragma unroll
        for (int r = 0; r < RC; ++r) yk[r] = T(0);
        const T* uk = us + (size_t)k * Px * RC;
        for (int jx = 0; jx < Px; ++jx) {
            const T b = bcol[(size_t)jx * blockDim.x];
#pragma unroll
            for (int r = 0; r < RC; ++r) yk[r] = fma(b, uk[jx * RC + r], yk[r]);
        }
#pragma unroll
        for (int l = 0; l < NWM; ++l) {
            if (l < nw) {
                const T mv = M[((long long)k * nw + l) * nh + m];
#pragma unroll
                for (int r = 0; r < RC; ++r) acc[l][r] = fma(mv, yk[r], acc[l][r]);
            }
        }
    }
#pragma unroll
    for (int l = 0; l < NWM; ++l)
#pragma unroll
        for (int r = 0; r < RC; ++r)
            if (l < nw && r0 + r < R) out[((long long)(r0 + r) * nw + l) * nh + m] = acc[l][r];
}

template <typename T, int NWM, int RC>
cudaError_t launch_inv_rc(const zl_plan_s& p, const T* u, const T* M, const T* bx, T* out, int R, cudaStream_t s) {
    const int nx = p.d.nx, threads = 128;
    const size_t smem = ((size_t)p.d.K * p.Px * RC + (size_t)p.Px * threads) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(inv_xpass_column_rc<T, NWM, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(p.d.ny, (nx + threads - 1) / threads, (R + RC - 1) / RC);
    inv_xpass_column_rc<T, NWM, RC><<<grid, threads, smem, s>>>(u, M, bx, out, R, p.d.nw, p.d.K, nx, p.d.ny, p.Px);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// inverse, pass 2, FP32 register-tiled form: CTA = (RC rhs, grid row y, 64-column chunk),
// looping over member chunks of KC = 128 / RC members, so that a chunk holds 128
// (rhs, member) rows:
//   phase 1 (x-pass): Y[(r, k)][x] = sum_jx u[r][k][y][jx] bx[jx][x], a GEMM with thread
//     tiles of 8 rows x 4 columns over 128-bit shared loads of the transposed u tile and
//     of the basis (lanes: 4 row groups x 8 column groups, warps: 4 x 2);
//   phase 2 (per-column product): out[r][l][x] += sum_k M[k][l][x] Y[(r, k)][x], thread =
//     (column, levels q + 4 i for its q < 4) with its RC x NLQ sums in registers across the
//     member chunks; each member-matrix element is read once per CTA.
// CTAs of the same row and column chunk (different rhs) are adjacent, so the
// member-matrix tile they share is read from L2.
// ---------------------------------------------------------------------------
constexpr int kIvXC = 64;                // grid columns per CTA
constexpr int kIvLdY = kIvXC + 4;        // row stride of Y and of the basis tile
constexpr int kIvLdU = 128 + 4;          // row stride of the transposed u tile

inline size_t inv_sgemm_smem(int Px) {
    return ((size_t)128 * kIvLdY + (size_t)Px * kIvLdU + (size_t)Px * kIvLdY) * sizeof(float);
}

template <int RC>
__global__ void __launch_bounds__(kThreads, 2)
inv_column_sgemm(const float* __restrict__ u, const float* __restrict__ M, const float* __restrict__ bx,
                 float* __restrict__ out, int R, int nw, int K, int nx, int ny, int Px) {
    constexpr int KC = 128 / RC;
    constexpr int NLQ = 32 / RC;                       // levels per thread in phase 2
    constexpr int KU = NLQ >= 16 ? 1 : 16 / NLQ;       // members per phase-2 step (KU divides KC)
    extern __shared__ float4 smem_f4[];
    float* Ys = reinterpret_cast<float*>(smem_f4);     // [128][kIvLdY], row = r * KC + k
    float* Ut = Ys + 128 * kIvLdY;                     // [Px][kIvLdU]
    float* Bs = Ut + (size_t)Px * kIvLdU;              // [Px][kIvLdY]
    const int tid = threadIdx.x;
    const int r0 = blockIdx.x * RC, y = blockIdx.y, x0 = blockIdx.z * kIvXC;
    const int xn = min(kIvXC, nx - x0);
    const long long nh = (long long)nx * ny;
    const int lane = tid & 31, warp = tid >> 5;
    for (int j = warp; j < Px; j += kThreads / 32)
        for (int xc = lane; xc < kIvXC; xc += 32) Bs[j * kIvLdY + xc] = xc < xn ? bx[(size_t)j * nx + x0 + xc] : 0.f;
    const int rg = (warp & 3) * 4 + (lane & 3);        // rows 4 rg + i and 64 + 4 rg + i (i < 4)
    const int cg = (warp >> 2) * 8 + (lane >> 2);      // columns 4 cg + j (j < 4)
    const int xc2 = tid & (kIvXC - 1);                 // phase 2: column
    const int lq = tid / kIvXC;                        // phase 2: levels lq + 4 i (i < NLQ)
    const bool col_ok = xc2 < xn;
    const long long m = (long long)y * nx + x0 + xc2;

    float acc[RC][NLQ];
#pragma unroll
    for (int r = 0; r < RC; ++r)
#pragma unroll
        for (int i = 0; i < NLQ; ++i) acc[r][i] = 0.f;

    for (int k0 = 0; k0 < K; k0 += KC) {
        __syncthreads();                               // the previous chunk's phase 2 is done with Ys
        for (int row = warp; row < 128; row += kThreads / 32) {
            const int r = row / KC, k = row - r * KC;
            const bool ok = r0 + r < R && k0 + k < K;
            const float* src = u + (((long long)(r0 + r) * K + k0 + k) * ny + y) * Px;
            for (int jx = lane; jx < Px; jx += 32) Ut[jx * kIvLdU + row] = ok ? src[jx] : 0.f;
        }
        __syncthreads();
        float c[8][4];
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
        for (int jx = 0; jx < Px; ++jx) {
            const float4 ua = *reinterpret_cast<const float4*>(Ut + jx * kIvLdU + 4 * rg);
            const float4 ub = *reinterpret_cast<const float4*>(Ut + jx * kIvLdU + 64 + 4 * rg);
            const float4 bv = *reinterpret_cast<const float4*>(Bs + jx * kIvLdY + 4 * cg);
            const float uu[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
            const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) c[i][j] = fmaf(uu[i], bb[j], c[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int row = (i < 4 ? 0 : 64) + 4 * rg + (i & 3);
            *reinterpret_cast<float4*>(Ys + row * kIvLdY + 4 * cg) = make_float4(c[i][0], c[i][1], c[i][2], c[i][3]);
        }
        __syncthreads();
        if (col_ok) {
            // KU members per step with all their member-matrix loads issued first; members
            // past K and levels past n_w are clamped to valid rows (their Y rows are zero,
            // their sums are never stored)
            const int kn = min(KC, K - k0);
            const float* Mm = M + m;
            const unsigned nhu = (unsigned)nh;
            for (int kk = 0; kk < kn; kk += KU) {
                float mv[KU][NLQ];
#pragma unroll
                for (int h = 0; h < KU; ++h)
#pragma unroll
                    for (int i = 0; i < NLQ; ++i)
                        mv[h][i] = __ldg(Mm + ((unsigned)min(k0 + kk + h, K - 1) * (unsigned)nw +
                                               (unsigned)min(lq + 4 * i, nw - 1)) * nhu);
#pragma unroll
                for (int h = 0; h < KU; ++h) {
                    float yv[RC];
#pragma unroll
                    for (int r = 0; r < RC; ++r) yv[r] = Ys[(r * KC + kk + h) * kIvLdY + xc2];
#pragma unroll
                    for (int i = 0; i < NLQ; ++i)
#pragma unroll
                        for (int r = 0; r < RC; ++r) acc[r][i] = fmaf(mv[h][i], yv[r], acc[r][i]);
                }
            }
        }
    }
    if (!col_ok) return;
#pragma unroll
    for (int r = 0; r < RC; ++r)
#pragma unroll
        for (int i = 0; i < NLQ; ++i)
            if (r0 + r < R && lq + 4 * i < nw) out[((long long)(r0 + r) * nw + lq + 4 * i) * nh + m] = acc[r][i];
}

template <int RC>
cudaError_t launch_inv_sgemm(const zl_plan_s& p, const float* u, const float* M, const float* bx, float* out, int R,
                             cudaStream_t s) {
    const size_t smem = inv_sgemm_smem(p.Px);
    cudaError_t e = cudaFuncSetAttribute(inv_column_sgemm<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((R + RC - 1) / RC, p.d.ny, (p.d.nx + kIvXC - 1) / kIvXC);
    inv_column_sgemm<RC><<<grid, kThreads, smem, s>>>(u, M, bx, out, R, p.d.nw, p.d.K, p.d.nx, p.d.ny, p.Px);
    return cudaGetLastError();
}

// rhs per CTA of the register-tiled inverse column pass, or 0 when it does not apply
// (P_x > 64 or n_w > 128): the largest of 8/4/2/1 whose phase-2 tile covers n_w levels
// (4 x 32 / RC) and that does not exceed R.
inline int inv_sgemm_rc(const zl_plan_s& p, int R) {
    if (p.Px > 64 || p.d.nw > 128) return 0;
    if ((unsigned long long)p.d.K * (unsigned long long)p.d.nw * (unsigned long long)p.nh >= (1ull << 32)) return 0;
    int rc = p.d.nw <= 16 ? 8 : p.d.nw <= 32 ? 4 : p.d.nw <= 64 ? 2 : 1;
    while (rc > 1 && rc > R) rc /= 2;
    return rc;
}

cudaError_t launch_inv_sgemm_any(const zl_plan_s& p, const float* u, const float* M, const float* bx, float* out,
                                 int R, cudaStream_t s) {
    switch (inv_sgemm_rc(p, R)) {
        case 8: return launch_inv_sgemm<8>(p, u, M, bx, out, R, s);
        case 4: return launch_inv_sgemm<4>(p, u, M, bx, out, R, s);
        case 2: return launch_inv_sgemm<2>(p, u, M, bx, out, R, s);
        default: return launch_inv_sgemm<1>(p, u, M, bx, out, R, s);
    }
}

// RC of the multi-rhs inverse column pass for this plan, or 0 when the one-rhs form runs:
// n_w <= 64, its shared staging under 160 KB, at least two right-hand sides, and rows of at
// least 64 columns (narrower rows would leave most of its 128-thread column tile idle).
// RC keeps the NWM x RC accumulators at 128 registers per thread in FP32, 64 in FP64.
template <typename T>
int inv_multi_fits(const zl_plan_s& p, int R) {
    const int nw = p.d.nw;
    auto fits = [&](int rc) { return ((size_t)p.d.K * p.Px * rc + (size_t)p.Px * 128) * sizeof(T) <= 160 * 1024; };
    if (R < 2 || p.d.nx < 64) return 0;
    if (sizeof(T) == 4) {
        if (nw <= 16 && fits(8)) return 8;
        if (nw <= 32 && fits(4)) return 4;
        if (nw <= 64 && fits(2)) return 2;
    } else {
        if (nw <= 16 && fits(4)) return 4;
        if (nw <= 32 && fits(2)) return 2;
    }
    return 0;
}

template <typename T>
cudaError_t launch_inv_multi(const zl_plan_s& p, const T* u, const T* M, const T* bx, T* out, int R, cudaStream_t s) {
    const int rc = inv_multi_fits<T>(p, R);
    if (sizeof(T) == 4) {
        if (rc == 8) return launch_inv_rc<T, 16, 8>(p, u, M, bx, out, R, s);
        if (rc == 4) return launch_inv_rc<T, 32, 4>(p, u, M, bx, out, R, s);
        if (rc == 2) return launch_inv_rc<T, 64, 2>(p, u, M, bx, out, R, s);
    } else {
        if (rc == 4) return launch_inv_rc<T, 16, 4>(p, u, M, bx, out, R, s);
        if (rc == 2) return launch_inv_rc<T, 32, 2>(p, u, M, bx, out, R, s);
    }
    return cudaErrorNotSupported;
}

// Right-hand sides per CTA of the forward column kernel: the plan's forced choice if it
// fits the shared-memory budget, else the largest of 8/4/2/1 that fits and has work.
inline int pick_rc(const zl_plan_s& p, int R, size_t row) {
    if (p.force_rc > 0 && (size_t)p.force_rc * row <= kRowSmemBudget) return p.force_rc;
    if (R >= 8 && 8 * row <= kRowSmemBudget) return 8;
    if (R >= 4 && 4 * row <= kRowSmemBudget) return 4;
    if (R >= 2 && 2 * row <= kRowSmemBudget) return 2;
    return 1;
}

template <typename T, int RC>
cudaError_t launch_fwd_rc(const zl_plan_s& p, const T* x, const T* M, const T* bx, T* t1, int R, cudaStream_t s,
                          Rows rows) {
    const int nx = p.d.nx, ny = rows.ny, K = p.d.K;
    const size_t smem = (size_t)KC * RC * (nx + 1) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(fwd_column_xpass<T, RC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid((K + KC - 1) / KC, (R + RC - 1) / RC, ny);
    fwd_column_xpass<T, RC><<<grid, kThreads, smem, s>>>(x, M, bx, t1, R, p.d.nw, K, nx, ny, p.Px, rows.y0, p.nh);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fwd(const zl_plan_s& p, const T* x, const T* M, const T* bx, T* t1, int R, cudaStream_t s,
                       Rows rows) {
    if constexpr (sizeof(T) == 4) {
        // the TMA-fed FP32 kernel where it applies; a tensor map it cannot encode (an
        // unaligned caller buffer) falls back to the per-column kernel
        if (f32_column_supported(p, R)) {
            const cudaError_t e = forward_column_f32(p, x, M, bx, t1, R, s, rows);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    switch (pick_rc(p, R, (size_t)KC * (p.d.nx + 1) * sizeof(T))) {
        case 8: return launch_fwd_rc<T, 8>(p, x, M, bx, t1, R, s, rows);
        case 4: return launch_fwd_rc<T, 4>(p, x, M, bx, t1, R, s, rows);
        case 2: return launch_fwd_rc<T, 2>(p, x, M, bx, t1, R, s, rows);
        default: return launch_fwd_rc<T, 1>(p, x, M, bx, t1, R, s, rows);
    }
}

// ---------------------------------------------------------------------------
// forward, pass 2 (general form): y-pass as a batched small GEMM per (rhs, member)
// pair, OUT[p_y][jx] = sum_y b_{p_y}(y) t1[y][pair][jx], then scale + compaction.
// Thread = (pair, jx); the kept y-basis rows are staged in shared memory and
// broadcast; t1 rows are read coalesced across the (pair, jx) threads.
// ---------------------------------------------------------------------------
constexpr int kYChunk = 64;

template <typename T, int PYT>
__global__ void __launch_bounds__(kThreads)
fwd_ypass_gemm(const T* __restrict__ t1, const T* __restrict__ byk, const int* __restrict__ m_ipy,
               const int* __restrict__ m_jx, const T* __restrict__ scale, T* __restrict__ out,
               int npairs, int ppc, int ny, int Px, int ldp, int L, int pys) {
    extern __shared__ unsigned char smem_raw[];
    T* sby = reinterpret_cast<T*>(smem_raw);       // [kYChunk][PYT]
    T* sout = sby + kYChunk * PYT;                   // [ppc][PYT][Px]
    const int tid = threadIdx.x;
    const int pl = tid / Px, jx = tid - pl * Px;
    const long long pair = (long long)blockIdx.x * ppc + pl;
    const bool active = pl < ppc && pair < npairs;
    const long long ystride = (long long)npairs * ldp;
    const T* src = t1 + (active ? pair * ldp + jx : 0);
    T acc[PYT];
#pragma unroll
    for (int i = 0; i < PYT; ++i) acc[i] = T(0);
    for (int y0 = 0; y0 < ny; y0 += kYChunk) {
        const int yn = min(kYChunk, ny - y0);
        __syncthreads();
        for (int e = tid; e < yn * PYT; e += blockDim.x) {
            const int yy = e / PYT, i = e - yy * PYT;
            sby[e] = i < pys ? byk[(long long)(y0 + yy) * pys + i] : T(0);
        }
        __syncthreads();
        if (active) {
            int yy = 0;
            for (; yy + 3 < yn; yy += 4) {   // four independent loads in flight per thread
                const T t0 = src[(long long)(y0 + yy) * ystride];
                const T t1v = src[(long long)(y0 + yy + 1) * ystride];
                const T t2 = src[(long long)(y0 + yy + 2) * ystride];
                const T t3 = src[(long long)(y0 + yy + 3) * ystride];
                const T* b = sby + yy * PYT;
#pragma unroll
                for (int i = 0; i < PYT; ++i) {
                    acc[i] = fma(b[i], t0, acc[i]);
                    acc[i] = fma(b[PYT + i], t1v, acc[i]);
                    acc[i] = fma(b[2 * PYT + i], t2, acc[i]);
                    acc[i] = fma(b[3 * PYT + i], t3, acc[i]);
                }
            }
            for (; yy < yn; ++yy) {
                const T tv = src[(long long)(y0 + yy) * ystride];
                const T* b = sby + yy * PYT;
#pragma unroll
                for (int i = 0; i < PYT; ++i) acc[i] = fma(b[i], tv, acc[i]);
            }
        }
    }
    if (active) {
        T* so = sout + (size_t)pl * PYT * Px;
#pragma unroll
        for (int i = 0; i < PYT; ++i) so[i * Px + jx] = acc[i];
    }
    __syncthreads();
    for (int pp = 0; pp < ppc; ++pp) {
        const long long pr = (long long)blockIdx.x * ppc + pp;
        if (pr >= npairs) break;
        const T* so = sout + (size_t)pp * PYT * Px;
        for (int j = tid; j < L; j += blockDim.x) {
            const T v = so[m_ipy[j] * Px + m_jx[j]];
            out[pr * L + j] = scale ? v * scale[j] : v;
        }
    }
}

// FP32 y-pass as one register-tiled GEMM over all pairs:
//   D[i][n] = sum_y byk[y][i] t1[y][n],   n = pair * Px + jx (the flattened t1 row),
// then x~[pair][j] = scale_j D[ipy_j][pair * Px + jx_j].  A CTA owns 64 CPT consecutive
// columns n (a pair may straddle two CTAs; each writes the modes whose column it holds)
// and all kept y-frequencies: thread = (CPT columns n + 64 c, group of PYG
// y-frequencies), CPT t1 values and one broadcast 128-bit basis load per 4 CPT products.
// The t1 and basis rows of the next 32 (16 with 4 columns per thread) values of y are
// loaded into registers while the current ones are used; the output tile reuses the
// shared memory of the stream.
constexpr int kYsN = 64;                 // columns per CTA and column slot

template <int PYG, int CPT>
struct YsPlan {
    static constexpr int YC = CPT >= 4 ? 16 : 32;  // rows of y per chunk
    static constexpr int IG = kThreads / kYsN;
    static constexpr int PYT = IG * PYG;           // kept y-frequencies covered (>= Py)
    static constexpr int NC = kYsN * CPT;          // columns per CTA
    static constexpr size_t stream = ((size_t)YC * NC + (size_t)YC * PYT) * sizeof(float);
    static constexpr size_t tile = (size_t)PYT * (NC + 1) * sizeof(float);
    static constexpr size_t bytes = stream > tile ? stream : tile;
};

template <int PYG, int CPT>
__global__ void __launch_bounds__(kThreads)
fwd_ypass_sgemm(const float* __restrict__ t1, const float* __restrict__ byk, const int* __restrict__ m_ipy,
                const int* __restrict__ m_jx, const float* __restrict__ scale, float* __restrict__ out, int npairs,
                int ny, int Px, int L, int pys) {
    using YP = YsPlan<PYG, CPT>;
    constexpr int PYT = YP::PYT, NC = YP::NC, kYsY = YP::YC;
    constexpr int TQ = kYsY * NC / kThreads;       // t1 values per thread per chunk
    constexpr int BQ = (kYsY * PYT + kThreads - 1) / kThreads;
    static_assert(PYG % 4 == 0, "128-bit basis loads");
    extern __shared__ float4 ys_smem4[];
    float* Ts = reinterpret_cast<float*>(ys_smem4);  // [kYsY][NC]
    float* Bs = Ts + kYsY * NC;                      // [kYsY][PYT]
    float* Ds = Ts;                                  // [PYT][NC + 1], after the stream
    const int tid = threadIdx.x;
    const int n = tid % kYsN, g = tid / kYsN;
    const long long ncols = (long long)npairs * Px;
    const long long n0 = (long long)blockIdx.x * NC;

    float tr[TQ], br[BQ];
    auto fetch = [&](int y0) {
#pragma unroll
        for (int q = 0; q < TQ; ++q) {
            const int e = tid + q * kThreads, row = e / NC, col = e % NC;
            tr[q] = (y0 + row < ny && n0 + col < ncols) ? t1[(long long)(y0 + row) * ncols + n0 + col] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < BQ; ++q) {
            const int e = tid + q * kThreads, row = e / PYT, i = e % PYT;
            br[q] = (e < kYsY * PYT && y0 + row < ny && i < pys) ? byk[(long long)(y0 + row) * pys + i] : 0.f;
        }
    };
    float acc[CPT][PYG];
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int i = 0; i < PYG; ++i) acc[c][i] = 0.f;
    fetch(0);
    for (int y0 = 0; y0 < ny; y0 += kYsY) {
        __syncthreads();                               // the previous chunk has been used
#pragma unroll
        for (int q = 0; q < TQ; ++q) Ts[tid + q * kThreads] = tr[q];
#pragma unroll
        for (int q = 0; q < BQ; ++q) {
            const int e = tid + q * kThreads;
            if (e < kYsY * PYT) Bs[e] = br[q];
        }
        __syncthreads();
        if (y0 + kYsY < ny) fetch(y0 + kYsY);
#pragma unroll 2
        for (int yy = 0; yy < kYsY; ++yy) {
            float t[CPT];
#pragma unroll
            for (int c = 0; c < CPT; ++c) t[c] = Ts[yy * NC + n + kYsN * c];
            const float4* b = reinterpret_cast<const float4*>(Bs + yy * PYT + g * PYG);
#pragma unroll
            for (int q = 0; q < PYG / 4; ++q) {
                const float4 bv = b[q];
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    acc[c][4 * q] = fmaf(bv.x, t[c], acc[c][4 * q]);
                    acc[c][4 * q + 1] = fmaf(bv.y, t[c], acc[c][4 * q + 1]);
                    acc[c][4 * q + 2] = fmaf(bv.z, t[c], acc[c][4 * q + 2]);
                    acc[c][4 * q + 3] = fmaf(bv.w, t[c], acc[c][4 * q + 3]);
                }
            }
        }
    }
    __syncthreads();                                   // the stream buffers become the output tile
#pragma unroll
    for (int c = 0; c < CPT; ++c)
#pragma unroll
        for (int i = 0; i < PYG; ++i) Ds[(g * PYG + i) * (NC + 1) + n + kYsN * c] = acc[c][i];
    __syncthreads();
    const long long p_lo = n0 / Px;
    const long long p_hi = min((long long)npairs - 1, (n0 + NC - 1) / Px);
    for (long long pr = p_lo; pr <= p_hi; ++pr) {
        const long long c0 = pr * Px - n0;             // column of the pair's x-frequency 0
        for (int j = tid; j < L; j += kThreads) {
            const long long col = c0 + m_jx[j];
            if (col < 0 || col >= NC) continue;
            const float v = Ds[m_ipy[j] * (NC + 1) + col];
            out[pr * L + j] = scale ? v * scale[j] : v;
        }
    }
}

template <int PYG, int CPT>
cudaError_t launch_ypass_sgemm_cpt(const zl_plan_s& p, const float* t1, const float* byk, const int* m_ipy,
                                   const int* m_jx, const float* scale, float* out, int R, cudaStream_t s, Rows rows) {
    using YP = YsPlan<PYG, CPT>;
    const long long npairs = (long long)R * p.d.K;
    const long long grid = (npairs * p.Px + YP::NC - 1) / YP::NC;
    cudaError_t e = cudaFuncSetAttribute(fwd_ypass_sgemm<PYG, CPT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)YP::bytes);
    if (e != cudaSuccess) return e;
    p.timer.begin(ZL_STAGE_FWD_YPASS, s);
    fwd_ypass_sgemm<PYG, CPT><<<(unsigned)grid, kThreads, YP::bytes, s>>>(
        t1, byk + (size_t)rows.y0 * p.pys, m_ipy, m_jx, scale, out, (int)npairs, rows.ny, p.Px, p.L, p.pys);
    p.timer.end(s);
    return cudaGetLastError();
}

// columns per thread: 4 while that still leaves about two CTAs per SM, else 1
template <int PYG>
cudaError_t launch_ypass_sgemm(const zl_plan_s& p, const float* t1, const float* byk, const int* m_ipy,
                               const int* m_jx, const float* scale, float* out, int R, cudaStream_t s, Rows rows) {
    const long long ncols = (long long)R * p.d.K * p.Px;
    if (ncols >= 2LL * 148 * 4 * kYsN)
        return launch_ypass_sgemm_cpt<PYG, 4>(p, t1, byk, m_ipy, m_jx, scale, out, R, s, rows);
    return launch_ypass_sgemm_cpt<PYG, 1>(p, t1, byk, m_ipy, m_jx, scale, out, R, s, rows);
}

// FP32 y-pass with the t1 rows of the CTA's pairs and the kept y-basis rows streamed
// through double-buffered shared memory by cp.async (16-byte copies), so that enough
// bytes are in flight to run at memory speed.  Needs ldp % 4 == 0 (16-byte rows).
// Each thread accumulates two adjacent x-frequencies (a column pair) of one (rhs,
// member) pair with packed two-lane FMAs (fma.rn.f32x2: two round-to-nearest FP32
// FMAs, the same arithmetic as two fmaf).  Threads are numbered column-major (the
// pairs of the CTA vary fastest), so a warp spans two or three neighbouring column
// pairs; each thread needs only the kept y-rows 0 .. yneed(jx) - 1 of its columns, and
// the warp runs the largest of its lanes' row counts, chosen once per streamed chunk.
// The output staging reuses the stream's shared memory.
constexpr int kYAsync = 16;

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint64_t f32x2_splat(float v) {
    uint64_t r;
    asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ void f32x2_fma(uint64_t& acc, uint64_t a, uint64_t b) {
    asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc) : "l"(a), "l"(b));
}
__device__ __forceinline__ float2 f32x2_unpack(uint64_t v) {
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// yn streamed y-rows of one column pair: kept y-rows 0 .. 4 N4 - 1 (a0: column jx, a1: jx + 1;
// entry i holds y-rows 2i and 2i + 1).
template <int PYT, int N4>
__device__ __forceinline__ void ypass_rows(uint64_t (&a0)[PYT / 2], uint64_t (&a1)[PYT / 2], const float* tt,
                                           const float* bb, int yn, int pw) {
#pragma unroll 1
    for (int yy = 0; yy < yn; ++yy) {
        const float2 tv = *reinterpret_cast<const float2*>(tt + yy * pw);
        const uint64_t tx = f32x2_splat(tv.x), ty = f32x2_splat(tv.y);
        const ulonglong2* b = reinterpret_cast<const ulonglong2*>(bb + yy * PYT);
#pragma unroll
        for (int i = 0; i < N4; ++i) {
            const ulonglong2 bv = b[i];
            f32x2_fma(a0[2 * i], bv.x, tx);
            f32x2_fma(a0[2 * i + 1], bv.y, tx);
            f32x2_fma(a1[2 * i], bv.x, ty);
            f32x2_fma(a1[2 * i + 1], bv.y, ty);
        }
    }
}

// ypass_rows<PYT, n4> for a warp-uniform n4 in 1 .. N4
template <int PYT, int N4>
__device__ __forceinline__ void ypass_rows_n(int n4, uint64_t (&a0)[PYT / 2], uint64_t (&a1)[PYT / 2],
                                             const float* tt, const float* bb, int yn, int pw) {
    if constexpr (N4 >= 1) {
        if (n4 == N4)
            ypass_rows<PYT, N4>(a0, a1, tt, bb, yn, pw);
        else
            ypass_rows_n<PYT, N4 - 1>(n4, a0, a1, tt, bb, yn, pw);
    }
}

template <int PYT>
__global__ void __launch_bounds__(kThreads)
fwd_ypass_async(const float* __restrict__ t1, const float* __restrict__ byk, const int* __restrict__ m_ipy,
                const int* __restrict__ m_jx, const int* __restrict__ yneed, const float* __restrict__ scale,
                float* __restrict__ out, int npairs, int ppc, int ny, int Px, int ldp, int L, int pys) {
    static_assert(PYT % 8 == 0, "16-byte rows of the kept y-basis");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int pw = ppc * ldp;                                   // floats of one y-row of this CTA
    float* st = reinterpret_cast<float*>(smem_raw);             // [2][kYAsync][pw]
    float* sb = st + 2 * kYAsync * pw;                          // [2][kYAsync][PYT]
    float* sout = st;                                           // [ppc][spitch], after the stream
    const int spitch = PYT * Px + 1;                            // odd: the lanes' stores hit distinct banks
    const int tid = threadIdx.x;
    const int half = ldp / 2;                                   // column pairs
    const int cp = tid / ppc, pl = tid - cp * ppc;              // column pair, pair in the CTA
    const int jx = 2 * cp;                                      // columns jx, jx + 1
    const long long pair0 = (long long)blockIdx.x * ppc;
    const int npl = (int)min((long long)ppc, npairs - pair0);  // pairs this CTA really has
    const bool active = cp < half && pl < npl;
    int need = 0;
    if (active) {
        if (jx < Px) need = yneed[jx];
        if (jx + 1 < Px) need = max(need, yneed[jx + 1]);
    }
    const int n4 = (need + 3) >> 2;                             // 16-byte groups of kept y-rows
    const int n4w = __reduce_max_sync(0xffffffffu, n4);         // the warp's row groups
    const long long ystride = (long long)npairs * ldp;
    const int nchunk = (ny + kYAsync - 1) / kYAsync;
    auto issue = [&](int c) {
        const int y0 = c * kYAsync, yn = min(kYAsync, ny - y0);
        float* dt = st + (c & 1) * kYAsync * pw;
        float* dbk = sb + (c & 1) * kYAsync * PYT;
        const int q = npl * ldp / 4;                            // 16-byte pieces per y-row
        for (int e = tid; e < yn * q; e += blockDim.x) {
            const int yy = e / q, i = e - yy * q;
            cp_async16(dt + yy * pw + 4 * i, t1 + (y0 + yy) * ystride + pair0 * ldp + 4 * i);
        }
        const int qb = PYT / 4;
        for (int e = tid; e < yn * qb; e += blockDim.x) {
            const int yy = e / qb, i = e - yy * qb;
            cp_async16(dbk + yy * PYT + 4 * i, byk + (long long)(y0 + yy) * pys + 4 * i);
        }
        cp_async_commit();
    };
    uint64_t a0[PYT / 2], a1[PYT / 2];
#pragma unroll
    for (int i = 0; i < PYT / 2; ++i) a0[i] = a1[i] = 0ull;
    issue(0);
    for (int c = 0; c < nchunk; ++c) {
        if (c + 1 < nchunk) {
            issue(c + 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int yn = min(kYAsync, ny - c * kYAsync);
        const float* tt = st + (c & 1) * kYAsync * pw + pl * ldp + jx;
        const float* bb = sb + (c & 1) * kYAsync * PYT;
        if (active) ypass_rows_n<PYT, PYT / 4>(n4w, a0, a1, tt, bb, yn, pw);
        __syncthreads();   // the buffer of chunk c is refilled by issue(c + 2)
    }
    if (active) {
        float* so = sout + (size_t)pl * spitch;
#pragma unroll
        for (int i = 0; i < PYT / 2; ++i) {
            if (2 * i < 4 * n4) {                              // rows past yneed are never gathered
                const float2 c0 = f32x2_unpack(a0[i]), c1 = f32x2_unpack(a1[i]);
                if (jx < Px) {
                    so[(2 * i) * Px + jx] = c0.x;
                    so[(2 * i + 1) * Px + jx] = c0.y;
                }
                if (jx + 1 < Px) {
                    so[(2 * i) * Px + jx + 1] = c1.x;
                    so[(2 * i + 1) * Px + jx + 1] = c1.y;
                }
            }
        }
    }
    __syncthreads();
    for (int pp = 0; pp < npl; ++pp) {
        const float* so = sout + (size_t)pp * spitch;
        float* o = out + (pair0 + pp) * L;
        for (int j = tid; j < L; j += blockDim.x) {
            const float v = so[m_ipy[j] * Px + m_jx[j]];
            o[j] = scale ? v * scale[j] : v;
        }
    }
}

template <int PYT>
cudaError_t launch_ypass_async(const zl_plan_s& p, const float* t1, int ldp, const float* byk, const int* m_ipy,
                               const int* m_jx, const int* yneed, const float* scale, float* out, int R,
                               cudaStream_t s, Rows rows) {
    const int npairs = R * p.d.K;
    const int ppc = kThreads / (ldp / 2);                       // pairs per CTA: ldp / 2 threads each
    const size_t stream = (size_t)2 * kYAsync * ppc * ldp + 2 * kYAsync * PYT,
                 staging = (size_t)ppc * ((size_t)PYT * p.Px + 1);
    const size_t smem = (stream > staging ? stream : staging) * sizeof(float);
    cudaError_t e = cudaFuncSetAttribute(fwd_ypass_async<PYT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (npairs + ppc - 1) / ppc;
    p.timer.begin(ZL_STAGE_FWD_YPASS, s);
    fwd_ypass_async<PYT><<<grid, kThreads, smem, s>>>(t1, byk + (size_t)rows.y0 * p.pys, m_ipy, m_jx, yneed, scale,
                                                      out, npairs, ppc, rows.ny, p.Px, ldp, p.L, p.pys);
    p.timer.end(s);
    return cudaGetLastError();
}

template <typename T, int PYT>
cudaError_t launch_ypass_gemm(const zl_plan_s& p, const T* t1, int ldp, const T* byk, const int* m_ipy,
                              const int* m_jx, const T* scale, T* out, int R, cudaStream_t s, Rows rows) {
    const int npairs = R * p.d.K;
    const int ppc = kThreads / p.Px;
    const size_t smem = ((size_t)kYChunk * PYT + (size_t)ppc * PYT * p.Px) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(fwd_ypass_gemm<T, PYT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (npairs + ppc - 1) / ppc;
    p.timer.begin(ZL_STAGE_FWD_YPASS, s);
    fwd_ypass_gemm<T, PYT><<<grid, kThreads, smem, s>>>(t1, byk + (size_t)rows.y0 * p.pys, m_ipy, m_jx, scale, out,
                                                         npairs, ppc, rows.ny, p.Px, ldp, p.L, p.pys);
    p.timer.end(s);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ypass(const zl_plan_s& p, const T* t1, int ldp, const T* by, const int* m_py, const int* m_jx,
                         const T* scale, T* out, int R, cudaStream_t s, const Tables<T>* tb, Rows rows) {
    const int ny = rows.ny, K = p.d.K;
    if (tb != nullptr && p.Px <= kThreads) {
        if (p.Py <= 8) return launch_ypass_gemm<T, 8>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 16) return launch_ypass_gemm<T, 16>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 24) return launch_ypass_gemm<T, 24>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 32) return launch_ypass_gemm<T, 32>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 40) return launch_ypass_gemm<T, 40>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 48) return launch_ypass_gemm<T, 48>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
        if (p.Py <= 64) return launch_ypass_gemm<T, 64>(p, t1, ldp, tb->byk, tb->m_ipy, m_jx, scale, out, R, s, rows);
    }
    int ychunk = ny;
    while ((size_t)(p.L + p.Px * (ychunk + 1)) * sizeof(T) > 96 * 1024 && ychunk > 1) ychunk = (ychunk + 1) / 2;
    const size_t smem = (size_t)(p.L + p.Px * (ychunk + 1)) * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(fwd_ypass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    p.timer.begin(ZL_STAGE_FWD_YPASS, s);
    fwd_ypass<T><<<dim3(K, R), kThreads, smem, s>>>(t1, by, m_py, m_jx, scale, out, R, K, ny, p.Px, ldp, p.L, ychunk,
                                                    p.d.ny, rows.y0);
    p.timer.end(s);
    return cudaGetLastError();
}

}  // namespace

cudaError_t forward_ypass_f32(const zl_plan_s& p, const float* t1, int ldp, const float* scale, float* out, int R,
                              cudaStream_t s, Rows rows) {
    // 16-byte rows and a kept y-basis that fits the register tile: the streaming form
    if (ldp % 4 == 0 && ldp / 2 <= kThreads && p.pys % 4 == 0 &&
        (size_t)(kThreads / (ldp / 2)) * ((size_t)ldp * 2 * kYAsync + (size_t)48 * p.Px) * 4 <= 200 * 1024) {
        const Tables<float>& t = p.tf;
        if (p.Py <= 16) return launch_ypass_async<16>(p, t1, ldp, t.byk, t.m_ipy, t.m_jx, t.yneed, scale, out, R, s,
                                                          rows);
        if (p.Py <= 24) return launch_ypass_async<24>(p, t1, ldp, t.byk, t.m_ipy, t.m_jx, t.yneed, scale, out, R, s,
                                                          rows);
        if (p.Py <= 32) return launch_ypass_async<32>(p, t1, ldp, t.byk, t.m_ipy, t.m_jx, t.yneed, scale, out, R, s,
                                                          rows);
        if (p.Py <= 40) return launch_ypass_async<40>(p, t1, ldp, t.byk, t.m_ipy, t.m_jx, t.yneed, scale, out, R, s,
                                                          rows);
        if (p.Py <= 48) return launch_ypass_async<48>(p, t1, ldp, t.byk, t.m_ipy, t.m_jx, t.yneed, scale, out, R, s,
                                                          rows);
    }
    return launch_ypass<float>(p, t1, ldp, p.tf.by, p.tf.m_py, p.tf.m_jx, scale, out, R, s, &p.tf, rows);
}

// the register-tiled FP32 y-pass over t1 rows of P_x values (the CUDA-core left inverse)
cudaError_t launch_ypass_f32_sgemm(const zl_plan_s& p, const float* t1, const Tables<float>& t, const float* scale,
                                   float* out, int R, cudaStream_t s, Rows rows) {
    if (p.Py <= 16) return launch_ypass_sgemm<4>(p, t1, t.byk, t.m_ipy, t.m_jx, scale, out, R, s, rows);
    if (p.Py <= 32) return launch_ypass_sgemm<8>(p, t1, t.byk, t.m_ipy, t.m_jx, scale, out, R, s, rows);
    if (p.Py <= 48) return launch_ypass_sgemm<12>(p, t1, t.byk, t.m_ipy, t.m_jx, scale, out, R, s, rows);
    return launch_ypass_sgemm<16>(p, t1, t.byk, t.m_ipy, t.m_jx, scale, out, R, s, rows);
}

template <typename T>
cudaError_t forward_plain(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* x, T* out,
                          int R, cudaStream_t s, Rows rows) {
    T* t1 = reinterpret_cast<T*>(p.t1);
    cudaError_t e;
    p.timer.begin(ZL_STAGE_FWD_COLUMN, s);
    e = launch_fwd<T>(p, x, M, t.bx, t1, R, s, rows);
    p.timer.end(s);
    if (e != cudaSuccess) return e;

    if constexpr (sizeof(T) == 4) {
        if (p.Py <= 64) return launch_ypass_f32_sgemm(p, t1, t, scale, out, R, s, rows);
    }
    return launch_ypass<T>(p, t1, p.Px, t.by, t.m_py, t.m_jx, scale, out, R, s, &t, rows);
}

template <typename T>
cudaError_t inverse_plain(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* c, T* out,
                          int R, cudaStream_t s) {
    const int nx = p.d.nx, ny = p.d.ny, K = p.d.K;
    T* u = reinterpret_cast<T*>(p.t1);
    size_t smem = (size_t)p.L * sizeof(T);
    cudaError_t e;
    p.timer.begin(ZL_STAGE_INV_YPASS, s);
    // the dense form when the kept y-frequencies are few (the GEMM does Py / (L / Px) times
    // the sparse form's multiply-adds, about 1.3 at the benchmark shapes)
    if (p.Py <= 64 && p.Px <= 64) {
        if (p.Px <= 16) e = launch_inv_ypass_dense<T, 4>(p, t, scale, c, u, R, s);
        else if (p.Px <= 32) e = launch_inv_ypass_dense<T, 8>(p, t, scale, c, u, R, s);
        else if (p.Px <= 48) e = launch_inv_ypass_dense<T, 12>(p, t, scale, c, u, R, s);
        else e = launch_inv_ypass_dense<T, 16>(p, t, scale, c, u, R, s);
    } else {
        e = cudaFuncSetAttribute(inv_ypass<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess) {
            inv_ypass<T><<<dim3(K, R), kThreads, smem, s>>>(c, t.by, t.m_py, t.grp_start, t.grp_modes, scale, u, K, ny,
                                                            p.Px, p.L);
            e = cudaGetLastError();
        }
    }
    p.timer.end(s);
    if (e != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
        if (f32_inverse_supported(p, R)) {
            p.timer.begin(ZL_STAGE_INV_COLUMN, s);
            e = inverse_column_f32(p, u, M, t.bx, out, R, s);
            p.timer.end(s);
            if (e != cudaErrorNotSupported) return e;
        }
        if (inv_sgemm_rc(p, R) > 0) {
            p.timer.begin(ZL_STAGE_INV_COLUMN, s);
            e = launch_inv_sgemm_any(p, u, M, t.bx, out, R, s);
            p.timer.end(s);
            return e;
        }
    }
    if (inv_multi_fits<T>(p, R) > 0) {
        p.timer.begin(ZL_STAGE_INV_COLUMN, s);
        e = launch_inv_multi<T>(p, u, M, t.bx, out, R, s);
        p.timer.end(s);
        return e;
    }
    int threads = nx < kThreads ? ((nx + 31) / 32) * 32 : kThreads;
    while ((size_t)K * (p.Px + threads) * sizeof(T) > 160 * 1024 && threads > 32) threads /= 2;
    smem = (size_t)K * (p.Px + threads) * sizeof(T);
    e = cudaFuncSetAttribute(inv_xpass_column<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(ny, (nx + threads - 1) / threads, R);
    p.timer.begin(ZL_STAGE_INV_COLUMN, s);
    inv_xpass_column<T><<<grid, threads, smem, s>>>(u, M, t.bx, out, p.d.nw, K, nx, ny, p.Px);
    p.timer.end(s);
    return cudaGetLastError();
}

// The forward pass of forward_plain with a caller-chosen intermediate buffer t1
// (at least R * K * ny * Px elements).  Used by zl_apply_left_inverse_static.
template <typename T>
cudaError_t forward_plain_on(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* x, T* out,
                             int R, cudaStream_t s, T* t1) {
    const Rows rows{0, p.d.ny};
    cudaError_t e = launch_fwd<T>(p, x, M, t.bx, t1, R, s, rows);
    if (e != cudaSuccess) return e;
    return launch_ypass<T>(p, t1, p.Px, t.by, t.m_py, t.m_jx, scale, out, R, s, &t, rows);
}

template <typename T>
cudaError_t preload_forward_plain() {
    cudaFuncAttributes a;
    const void* fns[] = {
        (const void*)fwd_column_xpass<T, 1>, (const void*)fwd_column_xpass<T, 2>, (const void*)fwd_column_xpass<T, 4>,
        (const void*)fwd_column_xpass<T, 8>, (const void*)fwd_ypass_gemm<T, 8>, (const void*)fwd_ypass_gemm<T, 16>,
        (const void*)fwd_ypass_gemm<T, 24>, (const void*)fwd_ypass_gemm<T, 32>, (const void*)fwd_ypass_gemm<T, 40>,
        (const void*)fwd_ypass_gemm<T, 48>, (const void*)fwd_ypass_gemm<T, 64>, (const void*)fwd_ypass<T>};
    for (const void* f : fns) {
        const cudaError_t e = cudaFuncGetAttributes(&a, f);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

template cudaError_t preload_forward_plain<double>();
template cudaError_t preload_forward_plain<float>();

template cudaError_t forward_plain_on<double>(const zl_plan_s&, const Tables<double>&, const double*, const double*,
                                              const double*, double*, int, cudaStream_t, double*);
template cudaError_t forward_plain_on<float>(const zl_plan_s&, const Tables<float>&, const float*, const float*,
                                             const float*, float*, int, cudaStream_t, float*);

template cudaError_t forward_plain<double>(const zl_plan_s&, const Tables<double>&, const double*, const double*,
                                           const double*, double*, int, cudaStream_t, Rows);
template cudaError_t forward_plain<float>(const zl_plan_s&, const Tables<float>&, const float*, const float*,
                                          const float*, float*, int, cudaStream_t, Rows);
template cudaError_t inverse_plain<double>(const zl_plan_s&, const Tables<double>&, const double*, const double*,
                                           const double*, double*, int, cudaStream_t);
template cudaError_t inverse_plain<float>(const zl_plan_s&, const Tables<float>&, const float*, const float*,
                                          const float*, float*, int, cudaStream_t);

}  // namespace zl
