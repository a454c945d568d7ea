// FP32 left inverse on the CUDA cores, fed by TMA: the per-column product of step V1
// (Sec. 3.10), w^(m) = A_m^+ x^(m), fused with the x-pass of V4 in one persistent kernel
// for FP32 plans (and the CUDA-core path of mixed plans).
//
// Work unit = (grid row y, RC right-hand sides, KC = 128 / RC members): the 128 rows
// (r, k) of the x-pass GEMM
//     t1[y][r][k][jx] = sum_x W[r][k][x] bx[jx][x],   W[r][k][x] = sum_l P[k][l][x] x[r][l][x],
// processed in chunks of 128 grid columns.  One copy-issuing thread streams the chunk's
// x tile [RC][LV][128] and member-matrix tile [KC][LV][128], LV levels per stage, into a
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
constexpr int LV = 2;                         // levels per stage
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
    f.stage = (uint32_t)(RC + KC) * LV * XC * 4u;
    f.bars = f.ring + (uint32_t)nstage * f.stage;
    f.total = f.bars + B_COUNT * 8u + 8u;                       // + the abort flag
    return f;
}

__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (uint32_t i = 1;; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 1023u) == 0u) {
            if (*abort_flag) return false;
            if ((unsigned long long)(clock64() - t0) > kWaitCycles) return false;
        }
    }
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
                if (ok && !wait_bar(&bars[B_FULL + s], (seq / (uint32_t)nstage) & 1u, abort_flag)) {
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
#pragma unroll 2
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

// 3-D map of a [n2][n1][n0] FP32 array with box {XC, LV, b2}.
bool encode3(CUtensorMap* m, const float* base, cuuint64_t n0, cuuint64_t n1, cuuint64_t n2, cuuint32_t b2) {
    const cuuint64_t gdim[3] = {n0, n1, n2};
    const cuuint64_t gstride[2] = {n0 * sizeof(float), n0 * n1 * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)XC, (cuuint32_t)LV, b2};
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
    if (!encode3(&tx, x, (cuuint64_t)rows.ny * p.d.nx, p.d.nw, R, RC) ||
        !encode3(&tp, M, (cuuint64_t)p.nh, p.d.nw, p.d.K, KC))
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

}  // namespace zl
