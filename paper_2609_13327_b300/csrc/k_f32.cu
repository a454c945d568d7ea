// FP32 left inverse on the CUDA cores, fed by TMA: the per-column product of step V1
// (Sec. 3.10), w^(m) = A_m^+ x^(m), fused with the x-pass of V4 in one persistent kernel
// for FP32 plans (and the CUDA-core path of mixed plans).
//
// Work unit = (grid row y, RC right-hand sides, KC = 128 / RC members): the 128 rows
// (r, k) of the x-pass GEMM
//     t1[y][r][k][jx] = sum_x W[r][k][x] bx[jx][x],   W[r][k][x] = sum_l P[k][l][x] x[r][l][x],
// processed in chunks of 128 grid columns.  One copy-issuing thread streams the chunk's
// x tile [RC][LV][128] and member-matrix tile [KC][LV][128], LV levels per stage (4 with 8
// rhs per unit, else 2), into a
// ring of shared-memory stages with 3-D tensor copies (out-of-range levels, rhs and
// members arrive as zeros), running ahead across chunks and units.  Eight compute warps:
//   phase A (V1): thread = (column, half of the members), its KC/2 x RC sums in
//     registers over the levels, read from the ring (conflict-free: lanes = columns),
//     then written to W in shared memory;
//   phase B (x-pass): thread = 4 rows x NJ x-frequencies, 128-bit shared loads of 4
//     consecutive columns of W (8 distinct rows per instruction, row stride 132 words:
//     distinct banks) and of the basis (4 distinct rows per warp, broadcast).
// The chunk's sums start from zero and are added to the running sums afterwards, so no
// FP32 accumulation chain is longer than 128 terms.  The unit's output tile leaves
// through shared memory: for each rhs the KC members' rows are contiguous in t1.
//
// Waits on the stage barriers are bounded; a timeout records an error code in the
// plan's device word, raises an abort flag that makes every other wait give up, and the
// kernel runs the rest of its loop skeleton without work (so that every warp reaches
// every CTA barrier) and returns; the copy-issuing thread waits for its copies to land
// before it exits.

#include "zl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>

#include <algorithm>

namespace zl {

namespace {

using namespace tc;

constexpr int kComputeWarps = 8;
constexpr int kCompute = 32 * kComputeWarps;
constexpr int kThreadsF = kCompute + 32;      // + the copy-issuing warp
constexpr int XC = 128;                       // grid columns per chunk
constexpr int LD = XC + 4;                    // row stride (words) of W and of the basis tile
// levels per stage of the forward kernel: 4 with 8 rhs per unit (a 48 KB stage), else 2
__host__ __device__ constexpr int lv_of(int RC) { return RC >= 8 ? 4 : 2; }
constexpr int kMaxStages = 6;
constexpr unsigned long long kWaitCycles = 4000000000ull;   // ~2 s at 2 GHz

enum { B_FULL = 0, B_EMPTY = B_FULL + kMaxStages, B_COUNT = B_EMPTY + kMaxStages };

struct FPlan {
    uint32_t w, b, ring, stage, bars, total;
};

__host__ __device__ inline FPlan fplan(int RC, int N, int nstage) {
    const int KC = 128 / RC;
    FPlan f{};
    f.w = 0;                                                    // W [128][LD], then the output tile
    f.b = f.w + 128u * LD * 4u;                                 // basis tile [N][LD]
    f.ring = (f.b + (uint32_t)N * LD * 4u + 127u) & ~127u;      // stages: x [RC][LV][XC], P [KC][LV][XC]
    f.stage = (uint32_t)(RC + KC) * lv_of(RC) * XC * 4u;
    f.bars = f.ring + (uint32_t)nstage * f.stage;
    f.total = f.bars + B_COUNT * 8u + 8u;                       // + the abort flag
    return f;
}

// Polling modes of a bounded wait.  The single-thread roles (producers, MMA issuers) poll with
// the non-blocking test_wait, so they react to a completed phase within one poll; whole warps
// use try_wait, whose suspension leaves the issue slots of their scheduler to the warps that
// share it (polling everywhere measured no faster).
constexpr bool kWarpSpin = false;

template <bool kSpin>
__device__ __forceinline__ bool wait_bar_t(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_test_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (kSpin ? mbar_test_wait(bar, parity) : mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 0u) {
            if (*abort_flag) return false;
            if ((unsigned long long)(clock64() - t0) > kWaitCycles) return false;
        }
    }
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    return wait_bar_t<true>(bar, parity, abort_flag);
}

__device__ __forceinline__ void fail(volatile int* abort_flag, int* err, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

__device__ __forceinline__ void compute_bar() { asm volatile("bar.sync 1, %0;" ::"n"(kCompute) : "memory"); }

// 16-byte global -> shared asynchronous copy of `bytes` (0..16) valid bytes, the rest zero
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <int RC, int NJ>
__global__ void __launch_bounds__(kThreadsF, 1)
fwd_column_f32_kernel(const __grid_constant__ CUtensorMap tmap_x, const __grid_constant__ CUtensorMap tmap_p,
                      const float* __restrict__ bx, float* __restrict__ t1, int* __restrict__ err, int R, int nw,
                      int K, int nx, int ny, int Px, int y0, int nstage, int no_copies) {
    constexpr int KC = 128 / RC;
    constexpr int KH = KC / 2;
    constexpr int N = 8 * NJ;
    extern __shared__ __align__(1024) unsigned char smem[];
    const FPlan fp = fplan(RC, N, nstage);
    float* W = reinterpret_cast<float*>(smem + fp.w);
    float* B = reinterpret_cast<float*>(smem + fp.b);
    unsigned char* ring = smem + fp.ring;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + fp.bars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + B_COUNT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nkc = (K + KC - 1) / KC, nrc = (R + RC - 1) / RC;
    const int units = ny * nrc * nkc;
    const int nchunk = (nx + XC - 1) / XC;
    constexpr int LV = lv_of(RC);
    const int nlg = (nw + LV - 1) / LV;

    if (tid == 0) {
        for (int s = 0; s < nstage; ++s) {
            mbar_init(&bars[B_FULL + s], 1);
            mbar_init(&bars[B_EMPTY + s], kComputeWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kComputeWarps) {
        // ------------------------------------------------------------ copy-issuing thread
        if (lane != 0) return;
        prefetch_tmap(&tmap_x);
        prefetch_tmap(&tmap_p);
        uint32_t seq = 0;
        for (int u = blockIdx.x; u < units && !*abort_flag; u += gridDim.x) {
            const int kc = u % nkc, rc = (u / nkc) % nrc, y = u / (nkc * nrc);
            for (int c = 0; c < nchunk && !*abort_flag; ++c)
                for (int g = 0; g < nlg; ++g, ++seq) {
                    const uint32_t s = seq % (uint32_t)nstage, n = seq / (uint32_t)nstage;
                    if (n > 0 && !wait_bar(&bars[B_EMPTY + s], (n - 1) & 1u, abort_flag)) {
                        fail(abort_flag, err, 1);
                        break;
                    }
                    if (no_copies) continue;      // test hook: the consumers' waits run out
                    unsigned char* st = ring + s * fp.stage;
                    mbar_arrive_expect_tx(&bars[B_FULL + s], fp.stage);
                    tma_load_3d(st, &tmap_x, y * nx + c * XC, g * LV, rc * RC, &bars[B_FULL + s]);
                    tma_load_3d(st + (uint32_t)RC * LV * XC * 4u, &tmap_p, (y0 + y) * nx + c * XC, g * LV, kc * KC,
                                &bars[B_FULL + s]);
                }
        }
        // every copy lands before the CTA exits: wait for the last one into each stage
        if (!no_copies) {
            const uint32_t first = seq > (uint32_t)nstage ? seq - (uint32_t)nstage : 0u;
            for (uint32_t q = first; q < seq; ++q) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&bars[B_FULL + q % (uint32_t)nstage], (q / (uint32_t)nstage) & 1u) &&
                       (unsigned long long)(clock64() - t0) < kWaitCycles) {}
            }
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    const int ax = tid & (XC - 1), ah = tid >> 7;
    const int brow = (warp & 3) * 32 + (lane & 7);        // phase B rows brow + 8 i
    const int bcol = (warp >> 2) * 4 * NJ + (lane >> 3);  // phase B x-frequencies bcol + 4 j
    bool ok = true;
    uint32_t seq = 0;
    for (int u = blockIdx.x; u < units; u += gridDim.x) {
        const int kc = u % nkc, rc = (u / nkc) % nrc, y = u / (nkc * nrc);
        const int k0 = kc * KC, r0 = rc * RC;
        float acc[4][NJ];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j) acc[i][j] = 0.f;
        for (int c = 0; c < nchunk; ++c) {
            const int x0 = c * XC, xn = min(XC, nx - x0), xn4 = (xn + 3) & ~3;
            compute_bar();                               // W, the basis tile and the output tile are free
            // the basis tile by 16-byte asynchronous copies (zero-filled past P_x and past the
            // row's end), landing while phase A runs
            for (int e = tid; e < N * (XC / 4); e += kCompute) {
                const int j = e / (XC / 4), xc = 4 * (e % (XC / 4));
                const int valid = (j < Px && xc < xn) ? 4 * min(4, xn - xc) : 0;
                const float* src = bx + (valid ? (size_t)j * nx + x0 + xc : 0);
                cp_async16(B + j * LD + xc, src, valid);
            }
            cp_async_commit();
            float a[KH][RC];
#pragma unroll
            for (int k = 0; k < KH; ++k)
#pragma unroll
                for (int r = 0; r < RC; ++r) a[k][r] = 0.f;
            for (int g = 0; g < nlg; ++g, ++seq) {
                const uint32_t s = seq % (uint32_t)nstage;
                if (ok && !wait_bar_t<kWarpSpin>(&bars[B_FULL + s], (seq / (uint32_t)nstage) & 1u, abort_flag)) {
                    fail(abort_flag, err, 2);
                    ok = false;
                }
                ok = __all_sync(0xffffffffu, ok);
                if (ok) {
                    const float* xs = reinterpret_cast<const float*>(ring + s * fp.stage);   // [RC][LV][XC]
                    const float* ps = xs + RC * LV * XC;                                     // [KC][LV][XC]
                    const int lvn = min(LV, nw - g * LV);
#pragma unroll
                    for (int l = 0; l < LV; ++l) {
                        if (l < lvn) {
                            float xv[RC];
#pragma unroll
                            for (int r = 0; r < RC; ++r) xv[r] = xs[(r * LV + l) * XC + ax];
#pragma unroll
                            for (int k = 0; k < KH; ++k) {
                                const float pv = ps[((ah * KH + k) * LV + l) * XC + ax];
#pragma unroll
                                for (int r = 0; r < RC; ++r) a[k][r] = fmaf(pv, xv[r], a[k][r]);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[B_EMPTY + s]);
            }
            // columns past the row's end hold the next row's data (or zeros): W is zero there
            const bool live = ax < xn;
#pragma unroll
            for (int r = 0; r < RC; ++r)
#pragma unroll
                for (int k = 0; k < KH; ++k) W[(r * KC + ah * KH + k) * LD + ax] = live ? a[k][r] : 0.f;
            cp_async_wait_all();
            compute_bar();
            float part[4][NJ];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) part[i][j] = 0.f;
            const float* wp = W + brow * LD;
            const float* bp = B + bcol * LD;
#pragma unroll 4
            for (int xc = 0; xc < xn4; xc += 4) {
                float4 wv[4], bv[NJ];
#pragma unroll
                for (int i = 0; i < 4; ++i) wv[i] = *reinterpret_cast<const float4*>(wp + 8 * i * LD + xc);
#pragma unroll
                for (int j = 0; j < NJ; ++j) bv[j] = *reinterpret_cast<const float4*>(bp + 4 * j * LD + xc);
                // one component at a time over all 4 x NJ sums: consecutive FMAs are independent
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) part[i][j] = fmaf(wv[i].x, bv[j].x, part[i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) part[i][j] = fmaf(wv[i].y, bv[j].y, part[i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) part[i][j] = fmaf(wv[i].z, bv[j].z, part[i][j]);
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < NJ; ++j) part[i][j] = fmaf(wv[i].w, bv[j].w, part[i][j]);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NJ; ++j) acc[i][j] += part[i][j];
        }
        compute_bar();                                   // phase B is done with W: stage the output
        float* ot = W;                                   // [128][N + 1]
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < NJ; ++j) ot[(brow + 8 * i) * (N + 1) + bcol + 4 * j] = acc[i][j];
        compute_bar();
        if (ok) {
            const int kn = min(KC, K - k0);
            for (int r = 0; r < RC && r0 + r < R; ++r) {
                float* dst = t1 + (((long long)y * R + r0 + r) * K + k0) * Px;
                for (int k = warp; k < kn; k += kComputeWarps)
                    for (int jx = lane; jx < Px; jx += 32) dst[k * Px + jx] = ot[(r * KC + k) * (N + 1) + jx];
            }
        }
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

// 3-D map of a [n2][n1][n0] FP32 array with box {XC, b1, b2}.
bool encode3(CUtensorMap* m, const float* base, cuuint64_t n0, cuuint64_t n1, cuuint64_t n2, cuuint32_t b1,
             cuuint32_t b2) {
    const cuuint64_t gdim[3] = {n0, n1, n2};
    const cuuint64_t gstride[2] = {n0 * sizeof(float), n0 * n1 * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)XC, b1, b2};
    const cuuint32_t estride[3] = {1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), gdim, gstride, box, estride,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int g_num_sms[64] = {};

template <int RC, int NJ>
cudaError_t launch_f32(const zl_plan_s& p, const float* x, const float* M, const float* bx, float* t1, int R,
                       cudaStream_t s, Rows rows) {
    constexpr int KC = 128 / RC;
    CUtensorMap tx, tp;
    if (!encode3(&tx, x, (cuuint64_t)rows.ny * p.d.nx, p.d.nw, R, lv_of(RC), RC) ||
        !encode3(&tp, M, (cuuint64_t)p.nh, p.d.nw, p.d.K, lv_of(RC), KC))
        return cudaErrorNotSupported;
    const FPlan f0 = fplan(RC, 8 * NJ, 0);
    const int nstage = std::min<int>(kMaxStages, (int)((227u * 1024u - f0.total) / f0.stage));
    if (nstage < 2) return cudaErrorNotSupported;
    const uint32_t smem = fplan(RC, 8 * NJ, nstage).total;
    cudaError_t e = cudaFuncSetAttribute(fwd_column_f32_kernel<RC, NJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int dev = p.device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_num_sms[dev] == 0) {
        e = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const long long units = (long long)rows.ny * ((R + RC - 1) / RC) * ((p.d.K + KC - 1) / KC);
    const int grid = (int)std::min<long long>(units, g_num_sms[dev]);
    fwd_column_f32_kernel<RC, NJ><<<grid, kThreadsF, smem, s>>>(tx, tp, bx, t1, p.d_werr, R, p.d.nw, p.d.K, p.d.nx,
                                                                rows.ny, p.Px, rows.y0, nstage,
                                                                p.test_wait_timeout);
    return cudaGetLastError();
}

template <int RC>
cudaError_t launch_f32_nj(const zl_plan_s& p, const float* x, const float* M, const float* bx, float* t1, int R,
                          cudaStream_t s, Rows rows) {
    if (p.Px <= 16) return launch_f32<RC, 2>(p, x, M, bx, t1, R, s, rows);
    if (p.Px <= 32) return launch_f32<RC, 4>(p, x, M, bx, t1, R, s, rows);
    if (p.Px <= 48) return launch_f32<RC, 6>(p, x, M, bx, t1, R, s, rows);
    return launch_f32<RC, 8>(p, x, M, bx, t1, R, s, rows);
}

// ---------------------------------------------------------------------------
// Inverse column pass (square root and adjoint), TMA-fed:
//   out[r][l][x] = sum_k M[k][l][x] Y[r][k][x],   Y[r][k][x] = sum_jx u[r][k][y][jx] bx[jx][x]
// (the inverse x-pass fused with the per-column product).  Work unit = (grid row y, RC
// right-hand sides, 128 grid columns), looping over member chunks of KC = 128 / RC
// members (128 rows (r, k)):
//   phase 1: Y = U B for the chunk's rows, thread tile 8 consecutive rows x 4 columns in
//     each half of the 128 columns (128-bit shared loads of the transposed u tile and of
//     the basis); the u rows of the chunk arrive transposed by 4-byte asynchronous copies
//     issued during the previous chunk's phase 2;
//   phase 2: thread = (column, parity of the level), its RC x NLH sums (levels h + 2 i)
//     in registers across the member chunks; the member-matrix tile of KS members x all
//     levels x 128 columns arrives per stage by one tensor copy.
// The member matrix is the streamed operand; it is read once per (row, rhs chunk).
// ---------------------------------------------------------------------------
constexpr int kIvStageMax = 32768;

struct IPlan {
    uint32_t y, b, u, ring, stage, bars, total;
    int pu, ks;
};

__host__ __device__ inline IPlan iplan(int RC, int Px, int nw, int nstage) {
    const int KC = 128 / RC;
    IPlan f{};
    f.pu = LD;                                                   // row stride of the transposed u tile
    int ks = 1;
    while (ks * 2 <= KC && (ks * 2) * nw * XC * 4 <= kIvStageMax) ks *= 2;
    f.ks = ks;
    f.y = 0;                                                     // Y [128][LD]
    f.b = f.y + 128u * LD * 4u;                                  // basis tile [Px][LD]
    f.u = f.b + (uint32_t)Px * LD * 4u;                          // u tile, transposed: [Px][LD] (rows (r, k))
    f.ring = (f.u + (uint32_t)Px * LD * 4u + 127u) & ~127u;      // stages: M [ks][nw][XC]
    f.stage = (uint32_t)ks * nw * XC * 4u;
    f.bars = f.ring + (uint32_t)nstage * f.stage;
    f.total = f.bars + B_COUNT * 8u + 8u;
    return f;
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src, int bytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(bytes) : "memory");
}

template <int RC>
__global__ void __launch_bounds__(kThreadsF, 1)
inv_column_f32_kernel(const __grid_constant__ CUtensorMap tmap_m, const float* __restrict__ u,
                      const float* __restrict__ bx, float* __restrict__ out, int* __restrict__ err, int R, int nw,
                      int K, int nx, int ny, int Px, int nstage) {
    constexpr int KC = 128 / RC;
    constexpr int NLH = 64 / RC;                           // levels per thread in phase 2 (n_w <= 2 NLH)
    extern __shared__ __align__(1024) unsigned char smem[];
    const IPlan ip = iplan(RC, Px, nw, nstage);
    const int KS = ip.ks, PU = ip.pu;
    float* Ys = reinterpret_cast<float*>(smem + ip.y);
    float* Bs = reinterpret_cast<float*>(smem + ip.b);
    float* Us = reinterpret_cast<float*>(smem + ip.u);
    unsigned char* ring = smem + ip.ring;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + ip.bars);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bars + B_COUNT);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nrc = (R + RC - 1) / RC, nxc = (nx + XC - 1) / XC;
    const int units = ny * nrc * nxc;
    const int nmc = (K + KC - 1) / KC;
    const int ngr = KC / KS;                               // member groups (stages) per member chunk
    const long long nh = (long long)nx * ny;

    if (tid == 0) {
        for (int s = 0; s < nstage; ++s) {
            mbar_init(&bars[B_FULL + s], 1);
            mbar_init(&bars[B_EMPTY + s], kComputeWarps);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();

    if (warp == kComputeWarps) {
        // ------------------------------------------------------------ copy-issuing thread
        if (lane != 0) return;
        prefetch_tmap(&tmap_m);
        uint32_t seq = 0;
        for (int un = blockIdx.x; un < units && !*abort_flag; un += gridDim.x) {
            const int xc = un % nxc, y = un / (nxc * nrc);
            for (int mc = 0; mc < nmc && !*abort_flag; ++mc)
                for (int g = 0; g < ngr; ++g, ++seq) {
                    const uint32_t s = seq % (uint32_t)nstage, n = seq / (uint32_t)nstage;
                    if (n > 0 && !wait_bar(&bars[B_EMPTY + s], (n - 1) & 1u, abort_flag)) {
                        fail(abort_flag, err, 3);
                        break;
                    }
                    mbar_arrive_expect_tx(&bars[B_FULL + s], ip.stage);
                    tma_load_3d(ring + s * ip.stage, &tmap_m, y * nx + xc * XC, 0, mc * KC + g * KS, &bars[B_FULL + s]);
                }
        }
        const uint32_t first = seq > (uint32_t)nstage ? seq - (uint32_t)nstage : 0u;
        for (uint32_t q = first; q < seq; ++q) {
            const long long t0 = clock64();
            while (!mbar_try_wait(&bars[B_FULL + q % (uint32_t)nstage], (q / (uint32_t)nstage) & 1u) &&
                   (unsigned long long)(clock64() - t0) < kWaitCycles) {}
        }
        return;
    }

    // ---------------------------------------------------------------- compute warps
    const int rw = warp & 3, cw = warp >> 2;
    const int rg = lane & 3, cg = lane >> 2;
    const int row0 = rw * 32 + rg * 8;                     // phase 1 rows row0 + i (i < 8)
    const int col0 = cw * 64 + cg * 4;                     // phase 1 columns col0 + 32 hf + {0..3} (hf < 2)
    const int x2 = tid & (XC - 1), h = tid >> 7;           // phase 2: column, level parity
    bool ok = true;
    uint32_t seq = 0;
    // u rows of member chunk mc of unit (y, r0), transposed (lane = row): 4-byte asynchronous
    // copies, zeros outside
    auto fetch_u = [&](int y, int r0, int mc) {
        const int row = (warp & 3) * 32 + lane;
        const int r = row / KC, k = mc * KC + row % KC;
        const bool live = r0 + r < R && k < K;
        const float* src = u + (((long long)(r0 + r) * K + k) * ny + y) * Px;
        for (int jx = warp >> 2; jx < Px; jx += 2) cp_async4(Us + jx * PU + row, live ? src + jx : u, live ? 4 : 0);
        cp_async_commit();
    };
    for (int un = blockIdx.x; un < units; un += gridDim.x) {
        const int xc = un % nxc, rc = (un / nxc) % nrc, y = un / (nxc * nrc);
        const int r0 = rc * RC, x0 = xc * XC, xn = min(XC, nx - x0);
        compute_bar();                                     // the previous unit is done with every tile
        for (int e = tid; e < Px * (XC / 4); e += kCompute) {
            const int j = e / (XC / 4), c4 = 4 * (e % (XC / 4));
            const int valid = c4 < xn ? 4 * min(4, xn - c4) : 0;
            cp_async16(Bs + j * LD + c4, bx + (valid ? (size_t)j * nx + x0 + c4 : 0), valid);
        }
        fetch_u(y, r0, 0);
        float acc[RC][NLH];
#pragma unroll
        for (int r = 0; r < RC; ++r)
#pragma unroll
            for (int i = 0; i < NLH; ++i) acc[r][i] = 0.f;
        for (int mc = 0; mc < nmc; ++mc) {
            cp_async_wait_all();
            compute_bar();                                 // u tile and basis tile landed; Ys is free
#pragma unroll 1
            for (int hf = 0; hf < 2; ++hf) {
                const int cc = col0 + 32 * hf;
                float c[8][4];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) c[i][j] = 0.f;
                for (int jx = 0; jx < Px; ++jx) {
                    const float4 u0 = *reinterpret_cast<const float4*>(Us + jx * PU + row0);
                    const float4 u1 = *reinterpret_cast<const float4*>(Us + jx * PU + row0 + 4);
                    const float4 bv = *reinterpret_cast<const float4*>(Bs + jx * LD + cc);
                    const float uu[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
                    const float bb[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
                    for (int j = 0; j < 4; ++j)
#pragma unroll
                        for (int i = 0; i < 8; ++i) c[i][j] = fmaf(uu[i], bb[j], c[i][j]);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i)
                    *reinterpret_cast<float4*>(Ys + (row0 + i) * LD + cc) = make_float4(c[i][0], c[i][1], c[i][2], c[i][3]);
            }
            compute_bar();                                 // Y complete; the u tile is free
            if (mc + 1 < nmc) fetch_u(y, r0, mc + 1);
            for (int g = 0; g < ngr; ++g, ++seq) {
                const uint32_t s = seq % (uint32_t)nstage;
                if (ok && !wait_bar_t<kWarpSpin>(&bars[B_FULL + s], (seq / (uint32_t)nstage) & 1u, abort_flag)) {
                    fail(abort_flag, err, 4);
                    ok = false;
                }
                ok = __all_sync(0xffffffffu, ok);
                if (ok) {
                    const float* ms = reinterpret_cast<const float*>(ring + s * ip.stage);   // [KS][nw][XC]
                    for (int kk = 0; kk < KS; ++kk) {
                        float yv[RC];
#pragma unroll
                        for (int r = 0; r < RC; ++r) yv[r] = Ys[(r * KC + g * KS + kk) * LD + x2];
                        const float* mk = ms + (size_t)kk * nw * XC + x2;
#pragma unroll
                        for (int i = 0; i < NLH; ++i) {
                            const int l = h + 2 * i;
                            if (l < nw) {
                                const float mv = mk[l * XC];
#pragma unroll
                                for (int r = 0; r < RC; ++r) acc[r][i] = fmaf(mv, yv[r], acc[r][i]);
                            }
                        }
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&bars[B_EMPTY + s]);
            }
        }
        if (ok && x2 < xn) {
            const long long m = (long long)y * nx + x0 + x2;
#pragma unroll
            for (int r = 0; r < RC; ++r)
#pragma unroll
                for (int i = 0; i < NLH; ++i)
                    if (r0 + r < R && h + 2 * i < nw) out[((long long)(r0 + r) * nw + h + 2 * i) * nh + m] = acc[r][i];
        }
    }
}

int inv_rc_of(int nw) { return nw <= 16 ? 8 : nw <= 32 ? 4 : 2; }

template <int RC>
cudaError_t launch_inv_f32(const zl_plan_s& p, const float* u, const float* M, const float* bx, float* out, int R,
                           cudaStream_t s) {
    CUtensorMap tm;
    const cuuint64_t gdim[3] = {(cuuint64_t)p.nh, (cuuint64_t)p.d.nw, (cuuint64_t)p.d.K};
    const cuuint64_t gstride[2] = {(cuuint64_t)p.nh * sizeof(float), (cuuint64_t)p.nh * p.d.nw * sizeof(float)};
    const IPlan i0 = iplan(RC, p.Px, p.d.nw, 0);
    const cuuint32_t box[3] = {(cuuint32_t)XC, (cuuint32_t)p.d.nw, (cuuint32_t)i0.ks};
    const cuuint32_t estride[3] = {1, 1, 1};
    if (encode_fn()(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(M), gdim, gstride, box, estride,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    const int nstage = std::min<int>(kMaxStages, (int)((227u * 1024u - i0.total) / i0.stage));
    if (nstage < 2) return cudaErrorNotSupported;
    const uint32_t smem = iplan(RC, p.Px, p.d.nw, nstage).total;
    cudaError_t e = cudaFuncSetAttribute(inv_column_f32_kernel<RC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int dev = p.device;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (g_num_sms[dev] == 0) {
        e = cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
    }
    const long long units = (long long)p.d.ny * ((R + RC - 1) / RC) * ((p.d.nx + XC - 1) / XC);
    const int grid = (int)std::min<long long>(units, g_num_sms[dev]);
    inv_column_f32_kernel<RC><<<grid, kThreadsF, smem, s>>>(tm, u, bx, out, p.d_werr, R, p.d.nw, p.d.K, p.d.nx,
                                                            p.d.ny, p.Px, nstage);
    return cudaGetLastError();
}

}  // namespace

bool f32_column_supported(const zl_plan_s& p, int R) {
    return p.Px <= 64 && R >= 4 && p.force_rc == 0 && p.d.nx % 4 == 0 && p.d_werr != nullptr &&
           encode_fn() != nullptr;
}

cudaError_t forward_column_f32(const zl_plan_s& p, const float* x, const float* M, const float* bx, float* t1, int R,
                               cudaStream_t s, Rows rows) {
    if (R >= 8) return launch_f32_nj<8>(p, x, M, bx, t1, R, s, rows);
    return launch_f32_nj<4>(p, x, M, bx, t1, R, s, rows);
}

bool f32_inverse_supported(const zl_plan_s& p, int R) {
    return p.Px <= 64 && p.d.nw <= 64 && R >= 2 && p.d.nx % 4 == 0 && p.d_werr != nullptr && encode_fn() != nullptr;
}

cudaError_t inverse_column_f32(const zl_plan_s& p, const float* u, const float* M, const float* bx, float* out, int R,
                               cudaStream_t s) {
    int rc = inv_rc_of(p.d.nw);
    while (rc > 2 && rc > R) rc /= 2;
    if (rc == 8) return launch_inv_f32<8>(p, u, M, bx, out, R, s);
    if (rc == 4) return launch_inv_f32<4>(p, u, M, bx, out, R, s);
    return launch_inv_f32<2>(p, u, M, bx, out, R, s);
}

}  // namespace zl
