// Tensor-core y-pass of the mixed-precision left inverse: the second half of step V4
// (Sec. 3.10), x~_k[j] = lambda_j^{-1/2} sum_y b_{p_y(j)}(y) c_k(y, p_x(j)), with
// c = t1 the x-pass output of the column kernel, stored [ny][R K][ldp] (ldp = Px
// rounded up to 4).
//
// As a GEMM: rows m = (pair, x-frequency slot) of t1, K = y, N = the kept y-frequencies.
//   D[m][i]       = sum_y T(m, y) b_hi(i, y)      (i < PYB)
//   D[m][PYB + i] = sum_y T(m, y) b_lo(i, y)
// with T = T_hi + T_lo split to FP16 and the K dimension carrying both halves
// ([T_hi | T_lo] against [b | b] per 8 rows of y), so every one of the four
// products is accumulated in FP32 in TMEM; the epilogue adds the two N halves.
// The basis is scaled by 16 (exactly) so that b_lo stays a normal FP16 number, and
// T by a power of two chosen from max |t1| (recorded by the column kernel), so that
// T_hi cannot overflow and T_lo keeps its precision; both scalings are undone
// exactly in the epilogue.
//
// A unit is ppu = floor(128 / ldp) pairs (M = ppu * ldp <= 128 rows) over all y.  Warp
// roles (448 threads): warp 0 lanes 0-1 = producers (one 2-D tensor copy of 32 y-rows of
// the unit's t1 block per stage, plus the basis of those rows when it is not resident),
// warp 1 = TMEM allocator + MMA issuer, warps 2-9 = converters (thread = row m and half
// of a stage: FP32 -> scaled FP16 hi/lo A operand of two 8-row slots of y), warps 10-13 =
// epilogue (TMEM -> per-pair mode gather -> x~, through a shared staging tile).
// Accumulators are double-buffered in TMEM so the drain of unit u overlaps the MMAs of
// unit u + 1.
//
// The conversion is this kernel's bottleneck (a chain of dependent instructions per
// value, measured: the ring depth of t1 stages does not change the kernel's time), so it
// runs on eight warps, two per scheduler, with one proxy fence per stage.  A stage
// returns to the producers as soon as the converters have read it (the MMAs read only
// the converted A slots and the basis).  Both K-chunks of an MMA's B operand are the same
// 8 y-rows of the basis, so the basis is stored once and its descriptor steps 0 bytes
// from one K-chunk to the next.  All waits are bounded.

#include "zl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <vector>

namespace zl {

struct YtcOperands {
    __half* bimg = nullptr;    // per y-block of 8 rows: N rows x [chunk 0 | chunk 1] x 8 FP16, K-major core matrices
    unsigned* t1max = nullptr; // max |t1| (float bits), written by the column kernel
    int* d_err = nullptr;
    int pyb = 0;               // kept y-frequencies rounded up to 8
    int nstage_y = 0;          // stages of 32 rows of y covering ny
    int resident = 0;          // 1: the whole basis image stays in shared memory
    uint32_t smem = 0;
};

namespace {

using namespace tc;

constexpr int YC = 32;                  // rows of y per stage (one tensor copy)
constexpr int YB = 8;                   // rows of y per MMA (one A slot)
constexpr int S = 4;                    // stage ring depth
constexpr int AG = 4;                   // A groups (one stage's four 8-row slots each)
constexpr int SA = AG * (YC / YB);      // A slots
constexpr int NE = 4;                   // ring of the commits that free A groups (one per two stages)
constexpr int kThreads = 448;
constexpr int kConvWarp0 = 2, kEpiWarp0 = 10;   // 8 converter warps: rows 0-127 x stage halves
constexpr uint32_t kTmemCols = 256;     // two accumulators of up to 128 columns
constexpr uint32_t kASlot = 4096;       // 128 rows x 32 B
constexpr float kBasisScale = 16.0f;
constexpr unsigned long long kWaitCycles = 4000000000ull;

// B_FULL: a stage's copies landed; B_TEMPTY: the stage may be refilled (its converters have
// read it, and the MMAs too when the stage carries the basis); B_EMPTY: commit c, issued after
// stage 2c + 1, i.e. the MMAs of every stage up to 2c + 1 completed (frees their A groups);
// B_AFULL: one per A group and stage half (slots 2h, 2h + 1), filled by the half's 4 warps
enum { B_FULL = 0, B_TEMPTY = B_FULL + S, B_EMPTY = B_TEMPTY + S, B_AFULL = B_EMPTY + NE,
       B_DFULL = B_AFULL + 2 * AG, B_DEMPTY = B_DFULL + 2, B_GFULL = B_DEMPTY + 2, B_GFREE, B_BASIS, B_FIN, B_COUNT };

struct Plan {
    uint32_t stage_t, stage_b, stage, ring, basis, aring, gather, bars, total;
};

// rows_u = ppu * ldp rows of t1 per stage row of y; nb = N = 2 * pyb.  resident > 0: the
// basis of all `resident` stages of y stays in shared memory (loaded once per CTA) and a
// stage holds t1 only; resident == 0: every stage carries its rows of the basis (per
// 8-row block of y: nb rows x 16 B, one K-chunk).
__host__ __device__ inline Plan smem_plan(int rows_u, int nb, int resident) {
    Plan s{};
    s.stage_t = ((uint32_t)rows_u * YC * 4u + 1023u) & ~1023u;
    s.stage_b = (uint32_t)(YC / YB) * (uint32_t)nb * 16u;
    s.stage = resident > 0 ? s.stage_t : (s.stage_t + s.stage_b + 1023u) & ~1023u;
    uint32_t o = 0;
    s.ring = o;
    o += (uint32_t)S * s.stage;
    s.basis = o;
    o += (uint32_t)resident * s.stage_b;
    o = (o + 1023u) & ~1023u;
    s.aring = o;
    o += SA * kASlot;
    s.gather = o;
    o += 128u * (uint32_t)(nb / 2 + 1) * 4u;
    o = (o + 127u) & ~127u;
    s.bars = o;
    o += ((B_COUNT * 8u + 8u) + 127u) & ~127u;
    s.total = o;
    return s;
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

__device__ __forceinline__ bool warp_wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const bool ok = wait_bar_t<kWarpSpin>(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void fail(volatile int* abort_flag, int* err, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int c0, int c1, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(dst)), "l"(tmap), "r"(c0), "r"(c1), "r"(smem_u32(bar))
        : "memory");
}

// 16 consecutive TMEM columns of this lane -> v[0..15]
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    tmem_ld16(taddr, r);
    tmem_ld_wait();
    tmem_regs_ready(r);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int NB>
__global__ void __launch_bounds__(kThreads, 1)
fwd_ypass_tc_kernel(const __grid_constant__ CUtensorMap tmap_t, const __half* __restrict__ bimg,
                    const unsigned* __restrict__ t1max, const int* __restrict__ m_ipy, const int* __restrict__ m_jx,
                    const float* __restrict__ scale, float* __restrict__ out, int* __restrict__ err, int npairs,
                    int ldp, int ppu, int L, int nstage_y, int resident, int staged_tab) {
    constexpr int PYB = NB / 2;
    extern __shared__ __align__(1024) uint8_t smem[];
    const int rows_u = ppu * ldp;
    const Plan sp = smem_plan(rows_u, NB, resident ? nstage_y : 0);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + sp.bars);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + B_COUNT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    float* gather = reinterpret_cast<float*>(smem + sp.gather);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int units = (npairs + ppu - 1) / ppu;
    const int my_units = (int)blockIdx.x < units ? (units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t tbytes = (uint32_t)rows_u * YC * 4u;

    if (tid == 0) {
        for (int i = 0; i < S; ++i) {
            mbar_init(&bars[B_FULL + i], 1);
            mbar_init(&bars[B_TEMPTY + i], resident ? 8 : 9);   // converter warps (+ the MMA commit)
        }
        for (int i = 0; i < NE; ++i) mbar_init(&bars[B_EMPTY + i], 1);
        for (int i = 0; i < 2 * AG; ++i) mbar_init(&bars[B_AFULL + i], 4);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&bars[B_DFULL + i], 1);
            mbar_init(&bars[B_DEMPTY + i], 128);
        }
        mbar_init(&bars[B_GFULL], 128);
        mbar_init(&bars[B_GFREE], 128);
        mbar_init(&bars[B_BASIS], 1);
        mbar_init(&bars[B_FIN], 1);
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmap_t);
    }
    if (warp == 1) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer
        // Lanes 0 and 1 issue the copies of even and odd stages: a copy costs its issuing
        // thread a roughly fixed time, so two threads keep twice the bytes in flight.
        if (lane < 2) {
            if (resident && lane == 0) {
                const uint32_t bytes = (uint32_t)nstage_y * sp.stage_b;
                mbar_arrive_expect_tx(&bars[B_BASIS], bytes);
                for (int st = 0; st < nstage_y; ++st)
                    bulk_g2s(smem + sp.basis + (uint32_t)st * sp.stage_b, bimg + (size_t)st * (sp.stage_b / 2), sp.stage_b,
                             &bars[B_BASIS]);
            }
            uint32_t sc = 0, mine = 0;
            constexpr uint32_t S2 = (uint32_t)S;
            bool go = true;
            for (int ui = 0; ui < my_units && go && !*abort_flag; ++ui) {
                const int u = (int)blockIdx.x + ui * (int)gridDim.x;
                for (int st = 0; st < nstage_y; ++st, ++sc) {
                    if ((int)(sc & 1u) != lane) continue;
                    const uint32_t s = sc % S2;
                    if (sc >= S2 && !wait_bar(&bars[B_TEMPTY + s], ((sc / S2) - 1) & 1u, abort_flag)) {
                        fail(abort_flag, err, 1);
                        go = false;
                        break;
                    }
                    uint8_t* dst = smem + sp.ring + s * sp.stage;
                    mbar_arrive_expect_tx(&bars[B_FULL + s], tbytes + (resident ? 0u : sp.stage_b));
                    tma_load_2d(dst, &tmap_t, u * rows_u, st * YC, &bars[B_FULL + s]);
                    if (!resident)
                        bulk_g2s(dst + sp.stage_t, bimg + (size_t)st * (sp.stage_b / 2), sp.stage_b, &bars[B_FULL + s]);
                    ++mine;
                }
            }
            // every copy this lane issued lands before the CTA exits.  Its copies are the stages
            // lane + 2 i (i < mine); S is even, so they all go to the slots of the lane's parity,
            // and the last copy into each such slot is one of its last S / 2.
            static_assert(S % 2 == 0, "two issuing lanes");
            constexpr uint32_t half = S2 / 2u;
            for (uint32_t i = mine > half ? mine - half : 0; i < mine; ++i) {
                const uint32_t c = (uint32_t)lane + 2u * i;
                const long long t0 = clock64();
                while (!mbar_try_wait(&bars[B_FULL + c % S2], (c / S2) & 1u) &&
                       (unsigned long long)(clock64() - t0) < kWaitCycles) {}
            }
            if (resident && lane == 0) {
                const long long t0 = clock64();
                while (!mbar_try_wait(&bars[B_BASIS], 0) && (unsigned long long)(clock64() - t0) < kWaitCycles) {}
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_f16_f32(128, NB);
            const uint64_t dA0 = smem_desc(smem_u32(smem + sp.aring), 128u, 256u);
            // B: both K-chunks ([b | b] against [T_hi | T_lo]) are the same core matrices, so the
            // K-direction stride is 0; 8-row groups of N are 128 B apart
            const uint64_t dB0 = resident ? smem_desc(smem_u32(smem + sp.basis), 0u, 128u)
                                          : smem_desc(smem_u32(smem + sp.ring + sp.stage_t), 0u, 128u);
            bool ok = true;
            if (resident && !wait_bar(&bars[B_BASIS], 0, abort_flag)) ok = false;
            uint32_t sc = 0;
            for (int ui = 0; ui < my_units && ok; ++ui) {
                const uint32_t d = (uint32_t)ui & 1u;
                if (ui >= 2 && !wait_bar(&bars[B_DEMPTY + d], ((ui >> 1) - 1) & 1u, abort_flag)) { ok = false; break; }
                tc_fence_after();
                for (int st = 0; st < nstage_y && ok; ++st, ++sc) {
                    const uint32_t s = sc % S, g = sc % AG;
                    if (!resident && !wait_bar(&bars[B_FULL + s], (sc / S) & 1u, abort_flag)) { ok = false; break; }
                    const uint32_t boff = resident ? (uint32_t)st * sp.stage_b : s * sp.stage;
                    for (int hh = 0; hh < 2 && ok; ++hh) {
                        if (!wait_bar(&bars[B_AFULL + 2 * g + (uint32_t)hh], (sc / AG) & 1u, abort_flag)) { ok = false; break; }
                        tc_fence_after();
#pragma unroll
                        for (int bb = 0; bb < 2; ++bb) {
                            const int b = 2 * hh + bb;
                            const uint32_t a = g * (YC / YB) + (uint32_t)b;
                            const uint64_t da = dA0 + ((a * kASlot) >> 4);
                            const uint64_t db = dB0 + ((boff + (uint32_t)b * NB * 16u) >> 4);
                            mma_f16(tbase + d * 128u, da, db, idesc, (st > 0 || b > 0) ? 1u : 0u);
                        }
                    }
                    // a commit after every second stage frees the A groups of both; a stage
                    // carrying the basis is freed by a commit of its own
                    if (ok) {
                        if (sc & 1u) mma_commit(&bars[B_EMPTY + (sc >> 1) % NE]);
                        if (!resident) mma_commit(&bars[B_TEMPTY + s]);
                    }
                }
                if (ok) mma_commit(&bars[B_DFULL + d]);
            }
            if (!ok) fail(abort_flag, err, 2);
            mma_commit(&bars[B_FIN]);
            const long long t0 = clock64();
            while (!mbar_try_wait(&bars[B_FIN], 0) && (unsigned long long)(clock64() - t0) < kWaitCycles) {}
        }
    } else if (warp < kEpiWarp0) {
        // ------------------------------------------------------------ converters: row m, stage half h
        const int ct = tid - 32 * kConvWarp0;                     // 0 .. 255
        const int m = ct & 127;                                    // row of the A operand
        const int h = ct >> 7;                                     // slots 2h, 2h + 1 of each stage
        int e2 = 0;
        (void)frexpf(__uint_as_float(*t1max), &e2);
        e2 = max(-100, min(100, e2));
        const float ts = ldexpf(1.0f, 14 - e2);                    // max |T| * ts < 2^14
        bool ok = true;
        uint32_t sc = 0;
        for (int ui = 0; ui < my_units && ok; ++ui) {
            for (int st = 0; st < nstage_y && ok; ++st, ++sc) {
                const uint32_t s = sc % S;
                if (!warp_wait_bar(&bars[B_FULL + s], (sc / S) & 1u, abort_flag)) { ok = false; break; }
                // A group sc % AG was last read by the MMAs of stage sc - AG, which commit
                // (sc - AG) / 2 covers
                if (sc >= (uint32_t)AG) {
                    const uint32_t c = (sc - AG) >> 1;
                    if (!warp_wait_bar(&bars[B_EMPTY + c % NE], (c / NE) & 1u, abort_flag)) {
                        ok = false;
                        break;
                    }
                }
                const float* tt = reinterpret_cast<const float*>(smem + sp.ring + s * sp.stage);
                const uint32_t g = sc % AG;
                const uint32_t a0 = g * (YC / YB) + 2u * (uint32_t)h;
                if (m < rows_u) {
#pragma unroll
                    for (int bb = 0; bb < 2; ++bb) {
                        const int b = 2 * h + bb;
                        float v[YB];
#pragma unroll
                        for (int e = 0; e < YB; ++e) v[e] = tt[(b * YB + e) * rows_u + m] * ts;
                        uint32_t hi[4], lo[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const __half2 hh = __floats2half2_rn(v[2 * e], v[2 * e + 1]);
                            const float2 hf = __half22float2(hh);
                            const __half2 l = __floats2half2_rn(v[2 * e] - hf.x, v[2 * e + 1] - hf.y);
                            hi[e] = *reinterpret_cast<const uint32_t*>(&hh);
                            lo[e] = *reinterpret_cast<const uint32_t*>(&l);
                        }
                        uint8_t* dst = smem + sp.aring + (a0 + (uint32_t)bb) * kASlot + (m >> 3) * 256u + (m & 7) * 16u;
                        *reinterpret_cast<uint4*>(dst) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
                        *reinterpret_cast<uint4*>(dst + 128u) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
                    }
                }
                // this thread's A rows are written and its reads of the stage done: one proxy
                // fence for both slots, then one arrival per warp
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(&bars[B_AFULL + 2 * g + (uint32_t)h]);
                    mbar_arrive(&bars[B_TEMPTY + s]);
                }
            }
        }
        if (!ok) fail(abort_flag, err, 3);
    } else {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;                                    // TMEM lane quarter
        const int m = 32 * q + lane;                               // accumulator row
        const int et = tid - 32 * kEpiWarp0;                       // 0 .. 127
        int e2 = 0;
        (void)frexpf(__uint_as_float(*t1max), &e2);
        e2 = max(-100, min(100, e2));
        const float unscale = ldexpf(1.0f, e2 - 14) / kBasisScale;
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        constexpr int GP = PYB + 1;                                // gather row pitch (odd)
        // the mode table (offset of mode j in a pair's gather rows, and its scale) in shared
        // memory after the barriers when it fits, read once per CTA instead of per pair; the
        // first B_GFULL wait below orders these writes before every epilogue thread's reads
        int* tab_off = reinterpret_cast<int*>(smem + sp.total);
        float* tab_scale = reinterpret_cast<float*>(tab_off + L);
        if (staged_tab)
            for (int j = et; j < L; j += 128) {
                tab_off[j] = m_jx[j] * GP + m_ipy[j];
                tab_scale[j] = scale ? scale[j] : 1.0f;
            }
        bool ok = true;
        for (int ui = 0; ui < my_units && ok; ++ui) {
            const int u = (int)blockIdx.x + ui * (int)gridDim.x;
            const uint32_t d = (uint32_t)ui & 1u;
            if (!warp_wait_bar(&bars[B_DFULL + d], (ui >> 1) & 1u, abort_flag)) { ok = false; break; }
            tc_fence_after();
            float v[NB];
#pragma unroll
            for (int c = 0; c < NB; c += 16) ld16(tbase + lane_off + d * 128u + (uint32_t)c, v + c);
            tc_fence_before();
            mbar_arrive(&bars[B_DEMPTY + d]);
            // the staging tile is free once every epilogue thread has gathered the previous unit
            if (ui >= 1 && !warp_wait_bar(&bars[B_GFREE], (ui - 1) & 1, abort_flag)) { ok = false; break; }
#pragma unroll
            for (int i = 0; i < PYB; ++i) gather[m * GP + i] = (v[i] + v[PYB + i]) * unscale;
            mbar_arrive(&bars[B_GFULL]);
            if (!warp_wait_bar(&bars[B_GFULL], ui & 1, abort_flag)) { ok = false; break; }
            const int p0 = u * ppu;
            for (int pl = 0; pl < ppu; ++pl) {
                const int pair = p0 + pl;
                if (pair >= npairs) break;
                float* o = out + (size_t)pair * L;
                if (staged_tab) {
                    const float* gp = gather + pl * ldp * GP;
                    for (int j = et; j < L; j += 128) o[j] = gp[tab_off[j]] * tab_scale[j];
                } else {
                    for (int j = et; j < L; j += 128) {
                        const float g = gather[(pl * ldp + m_jx[j]) * GP + m_ipy[j]];
                        o[j] = scale ? g * scale[j] : g;
                    }
                }
            }
            mbar_arrive(&bars[B_GFREE]);
        }
        if (!ok) fail(abort_flag, err, 4);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        __syncwarp();
        tmem_dealloc(tbase, kTmemCols);
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

double by_value(int N, int p, int m) {
    if (p == 0) return 1.0 / std::sqrt((double)N);
    if (N % 2 == 0 && p == N - 1) return ((m & 1) ? -1.0 : 1.0) / std::sqrt((double)N);
    const int j = (p + 1) / 2;
    const long long r = ((long long)j * m) % N;
    const double a = 2.0 * M_PI * (double)r / (double)N;
    return std::sqrt(2.0 / N) * ((p & 1) ? std::cos(a) : std::sin(a));
}

// Plans of different shapes share a template instance, so its limit is the largest that a
// plan may use (227 KB).
template <int NB>
cudaError_t set_smem(uint32_t) {
    return cudaFuncSetAttribute(fwd_ypass_tc_kernel<NB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
}

}  // namespace

bool ytc_supported(const zl_plan_s& p, int ldp) {
    return p.Py >= 1 && p.Py <= 64 && ldp % 4 == 0 && ldp <= 128 && encode_fn() != nullptr;
}

zl_status ytc_prepare(zl_plan_s& p, int ldp, cudaStream_t s) {
    if (!ytc_supported(p, ldp)) return ZL_ERR_UNSUPPORTED;
    YtcOperands* t = new YtcOperands();
    t->pyb = (p.Py + 7) / 8 * 8;
    const int nb = 2 * t->pyb;
    t->nstage_y = (p.d.ny + YC - 1) / YC;
    const int ppu = 128 / ldp;
    t->resident = smem_plan(ppu * ldp, nb, t->nstage_y).total <= 227u * 1024u ? 1 : 0;
    t->smem = smem_plan(ppu * ldp, nb, t->resident ? t->nstage_y : 0).total;
    // kept y-frequencies in ascending order (the order of the byk table's columns)
    std::vector<int> pylist;
    {
        std::vector<char> used(p.d.ny, 0);
        for (int sidx : p.modes) used[sidx / p.d.nx] = 1;
        for (int q = 0; q < p.d.ny; ++q)
            if (used[q]) pylist.push_back(q);
    }
    const size_t yblocks = (size_t)t->nstage_y * (YC / YB);
    // per 8-row block of y: nb rows (b_hi rows, then b_lo rows) x 8 FP16 values of y, in 8-row
    // core matrices of 128 B (one K-chunk; the MMA reads it for both of its K-chunks)
    const size_t per_block = (size_t)nb * 8;                        // FP16 elements per 8-row block
    std::vector<__half> img(yblocks * per_block, __float2half_rn(0.f));
    for (size_t yb = 0; yb < yblocks; ++yb)
        for (int n = 0; n < nb; ++n) {
            const int i = n % t->pyb, part = n / t->pyb;               // part 0: b_hi rows, 1: b_lo rows
            for (int e = 0; e < YB; ++e) {
                const int y = (int)yb * YB + e;
                double b = 0.0;
                if (y < p.d.ny && i < (int)pylist.size()) b = kBasisScale * by_value(p.d.ny, pylist[i], y);
                const __half hi = __double2half(b);
                const __half v = part == 0 ? hi : __double2half(b - (double)__half2float(hi));
                const size_t off = yb * per_block * 2 + (size_t)(n >> 3) * 128 + (size_t)(n & 7) * 16 + (size_t)e * 2;
                img[off / 2] = v;
            }
        }
    cudaError_t e = zl::dev_malloc((void**)&t->bimg, img.size() * sizeof(__half));
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&t->t1max, sizeof(unsigned));
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&t->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyAsync(t->bimg, img.data(), img.size() * sizeof(__half), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->t1max, 0, sizeof(unsigned), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        switch (nb) {
            case 16: e = set_smem<16>(t->smem); break;
            case 32: e = set_smem<32>(t->smem); break;
            case 48: e = set_smem<48>(t->smem); break;
            case 64: e = set_smem<64>(t->smem); break;
            case 80: e = set_smem<80>(t->smem); break;
            case 96: e = set_smem<96>(t->smem); break;
            case 112: e = set_smem<112>(t->smem); break;
            case 128: e = set_smem<128>(t->smem); break;
            default: e = cudaErrorInvalidValue;
        }
    }
    if (e != cudaSuccess || t->smem > 227 * 1024) {
        cudaFree(t->bimg);
        cudaFree(t->t1max);
        cudaFree(t->d_err);
        delete t;
        if (e == cudaErrorMemoryAllocation) return ZL_ERR_ALLOC;
        return e == cudaSuccess ? ZL_ERR_UNSUPPORTED : ZL_ERR_CUDA;
    }
    p.ytc = t;
    return ZL_OK;
}

void ytc_release(zl_plan_s& p) {
    if (!p.ytc) return;
    cudaFree(p.ytc->bimg);
    cudaFree(p.ytc->t1max);
    cudaFree(p.ytc->d_err);
    delete p.ytc;
    p.ytc = nullptr;
}

unsigned* ytc_max_word(const zl_plan_s& p) { return p.ytc ? p.ytc->t1max : nullptr; }

cudaError_t ytc_read_error(const zl_plan_s& p, int* code) {
    *code = 0;
    if (!p.ytc) return cudaSuccess;
    return cudaMemcpy(code, p.ytc->d_err, sizeof(int), cudaMemcpyDeviceToHost);
}

cudaError_t ytc_clear_error(const zl_plan_s& p) {
    if (!p.ytc) return cudaSuccess;
    return cudaMemset(p.ytc->d_err, 0, sizeof(int));
}

cudaError_t forward_ypass_tc(const zl_plan_s& p, const float* t1, int ldp, const float* scale, float* out, int R,
                             cudaStream_t s) {
    const YtcOperands& t = *p.ytc;
    const int npairs = R * p.d.K;
    const int ppu = 128 / ldp, rows_u = ppu * ldp;
    const int nb = 2 * t.pyb;
    CUtensorMap tmap;
    const cuuint64_t gdim[2] = {(cuuint64_t)npairs * ldp, (cuuint64_t)p.d.ny};
    const cuuint64_t gstride[1] = {(cuuint64_t)npairs * ldp * sizeof(float)};
    const cuuint32_t box[2] = {(cuuint32_t)rows_u, (cuuint32_t)YC};
    const cuuint32_t estride[2] = {1, 1};
    const CUresult cr = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(t1), gdim, gstride, box,
                                    estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int units = (npairs + ppu - 1) / ppu;
    const int grid = std::min(units, 148);
    // the mode table goes to shared memory when it fits next to the kernel's plan
    const size_t tab_bytes = (size_t)p.L * 8u;
    const int staged_tab = (size_t)t.smem + tab_bytes <= 227u * 1024u ? 1 : 0;
    const size_t smem = t.smem + (staged_tab ? tab_bytes : 0);
    p.timer.begin(ZL_STAGE_FWD_YPASS, s);
#define ZL_YTC_LAUNCH(NBV)                                                                                           \
    fwd_ypass_tc_kernel<NBV><<<grid, kThreads, smem, s>>>(tmap, t.bimg, t.t1max, p.tf.m_ipy, p.tf.m_jx, scale, out, \
                                                          t.d_err, npairs, ldp, ppu, p.L, t.nstage_y, t.resident,   \
                                                          staged_tab)
    switch (nb) {
        case 16: ZL_YTC_LAUNCH(16); break;
        case 32: ZL_YTC_LAUNCH(32); break;
        case 48: ZL_YTC_LAUNCH(48); break;
        case 64: ZL_YTC_LAUNCH(64); break;
        case 80: ZL_YTC_LAUNCH(80); break;
        case 96: ZL_YTC_LAUNCH(96); break;
        case 112: ZL_YTC_LAUNCH(112); break;
        case 128: ZL_YTC_LAUNCH(128); break;
        default: return cudaErrorInvalidValue;
    }
#undef ZL_YTC_LAUNCH
    p.timer.end(s);
    return cudaGetLastError();
}

}  // namespace zl
