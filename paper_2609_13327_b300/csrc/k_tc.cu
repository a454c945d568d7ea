// Tensor-core left inverse (ZL_MIXED): steps V1-V3 plus the x-pass of V4 in one
// persistent, warp-specialised tcgen05 kernel.
//
// Work unit = (grid row y, chunk of RC = 16 right-hand sides).  For every
// column m of the row the per-column product of step V1 (Sec. 3.10),
//     w^(m) = A_m^+ x^(m),   a K x n_w by n_w x RC product,
// runs on the tensor cores with FP16 operand splits P = P_hi + P_lo and
// x = x_hi + x_lo.  One MMA per K-step yields all four partial products: the A
// operand stacks [P_hi; P_lo] along M (128 rows = 2 x 64 members) and the B
// operand stacks [x_hi; x_lo] along N (32 = 2 x RC), so TMEM lane k holds
// P_hi x_hi | P_hi x_lo and lane 64 + k holds P_lo x_hi | P_lo x_lo.  The
// epilogue adds the two N halves, giving P_hi x (lanes < 64) and the small
// correction P_lo x (lanes >= 64), and writes the A operand W of the x-pass:
// P_hi x split again into FP16 hi/lo (W_hi, W_lo), P_lo x rounded once to FP16
// (W_c, its own rounding error is 2^-11 of a term that is itself 2^-11 of w).
// The x-pass multiplies W by the pruned real-Fourier basis of the row (N = 48
// >= P_x kept x-frequencies, b = b_hi + b_lo) and accumulates the whole row in
// TMEM; its K dimension runs along the grid row, 8 columns per K-chunk, and two
// MMAs per 128-row tile and 8-column group give
//     W_hi b_hi + W_c b_hi   (K-chunks [W_hi | W_c]  x [b_hi | b_hi])
//     W_lo b_hi + W_hi b_lo  (K-chunks [W_lo | W_hi] x [b_hi | b_lo]),
// dropping only the 2^-22 terms W_lo b_lo and W_c b_lo.  The regrouping of
// w^(m) into member segments (steps V2-V3, the paper's inter-processor
// exchange) thus never leaves the SM.  The y-pass, Delta^{-1/2} scaling and
// compaction (the rest of V4, and V5) follow in fwd_ypass_tc_kernel (k_ytc.cu).
//
// Shared-memory bandwidth (about 128 B per clock, shared by the tensor pipe's
// operand reads, the bulk copies and the warps' loads and stores) bounds this
// kernel, so the operand layout minimises bytes moved per column: one 4 KB A
// read per V1 K-step, one conversion pass over x, 48 KB of W per 8 columns.
//
// TMEM: 384 columns of x-pass accumulators (8 tiles x 48) and 128 columns of
// V1 accumulators, i.e. 4 grid columns x 32; V1 therefore runs in half-groups
// of 4 columns, and V1 of half-group n + 1 waits until the epilogue has drained
// D1 of half-group n.  The x-pass of group g needs the W of both half-groups of
// g, so it runs about one group behind V1 on its own issuing thread and keeps the
// tensor pipe busy while the epilogue drains D1 and writes W.
//
// Operand supply: the engine behind the bulk copies spends a roughly fixed
// time per copy, so operands arrive in few, large copies: the [P_hi; P_lo]
// images of a half-group's four columns are contiguous in the plan's image
// array and land in one 4 x 8 KB copy (a 3-slot ring), the x tile of a group
// in one 3-D tensor-map load, the basis of a group in one 2.3 KB copy, and one
// L2 prefetch per group warms the images needed two groups later.
//
// Warp roles (384 threads): warp 0 lane 0 = producer of the pseudo-inverse
// images and of the per-group x-pass basis, warp 1 lane 0 = producer of the x
// tiles, warp 2 = TMEM allocator + single-thread issuer of the V1 MMAs, warp 11 lane
// 0 = single-thread issuer of the x-pass MMAs (warp w issues on scheduler w % 4;
// schedulers 2 and 3 are shared with the lighter W_c epilogue warps), warps 3-10 =
// converters (x tile -> FP16 [x_hi; x_lo] B operand, two group slots) and epilogue
// (TMEM -> W; TMEM -> intermediate t1 [ny][R][K][pxp]); two epilogue warps share each
// TMEM lane quarter and split the unit's right-hand sides.  The two issuers wait only
// for their own operands (measured: a single issuer spent about a third of each group
// in waits, fences and commits while the tensor pipe ran dry), so one issues while the
// other waits; their MMAs write disjoint TMEM columns (D1 and D2), and each commits
// its own completions.  All waits are bounded; on timeout the kernel records an error
// code, drains its own copies, frees TMEM and returns.

#include "zl_internal.cuh"
#include "tc_ptx.cuh"

#include <cuda.h>
#include <cuda_fp16.h>

#include <cmath>
#include <vector>

namespace zl {

struct TcOperands {
    __half* pimg = nullptr;    // [nh][128 rows][nwp] K-major image of [P_hi; P_lo] per column
    uint8_t* bximg = nullptr;  // per 8-column group: K-chunks [b_hi | b_hi | b_lo] x 6 row groups x 128 B
    int* d_err = nullptr;      // device error word (0 = ok)
    int nwp = 0;               // V1 K extent: n_w rounded up to 16 or 32
    int pxp = 0;               // row stride of t1 (Px rounded up to 4)
    int num_sms = 0;
    uint32_t smem = 0;
};

namespace {

using namespace tc;

constexpr int RC = 16;                 // right-hand sides per unit
constexpr int N1 = 2 * RC;             // V1 N: [x_hi; x_lo]
constexpr int GC = 8;                  // columns per group (one x-pass K-chunk)
constexpr int HG = 4;                  // columns per V1 half-group
constexpr int N2 = 48;                 // x-pass N: kept x-frequencies padded
constexpr int MT = 8;                  // x-pass M tiles: 64 members x 16 rhs / 128
constexpr int SPH = 3;                 // P image ring depth in half-groups (4 images per slot)
constexpr int SX = 2;                  // x tile ring depth
constexpr int SB = 3;                  // x-pass basis ring depth
constexpr int NEPI = 8;                // epilogue / converter warps
constexpr int kEpiWarp0 = 3;           // warps 0: P/basis producer, 1: x producer, 2: V1 MMA
constexpr int kMmaWarp = 2;
constexpr int kXWarp = 1;
constexpr int kXpassWarp = kEpiWarp0 + NEPI;   // 11: x-pass MMA issuer
constexpr int kThreadsTc = 32 * (kXpassWarp + 1);
constexpr int kEpiThreads = 32 * NEPI;
constexpr uint32_t kD1Col = MT * N2;   // 384: V1 accumulators after the x-pass accumulators
constexpr uint32_t kTmemCols = 512;
static_assert(kD1Col + HG * N1 <= kTmemCols, "TMEM columns");
constexpr uint32_t kWChunk = 16384;    // one K-chunk of W: 1024 rows x 16 B
constexpr uint32_t kWBytes = 3 * kWChunk;   // chunks: 0 = W_lo, 1 = W_hi, 2 = W_c
constexpr uint32_t kBxChunk = 768;     // one K-chunk of the x-pass basis: 48 rows x 16 B
constexpr uint32_t kBxStage = 3 * kBxChunk;   // chunks: b_hi, b_hi, b_lo
constexpr unsigned long long kWaitCycles = 4000000000ull;   // ~2 s at 2 GHz

// Completion rings.  The V1 issuer commits once per V1 half-group n (V1DONE, slot n % kDoneV),
// the x-pass issuer once per group g (XDONE, slot g % kDoneX: W is free, the basis stage is
// free, and a unit that ended at group g has its whole row in D2).  A waiter never lags the
// newest commit by a full ring (the V1 issuer runs at most one group ahead of the x-pass, the
// producer and the epilogue at most SB groups behind it), so the phase parity is unambiguous.
constexpr int kDoneV = 8;
constexpr int kDoneX = 8;
constexpr uint32_t kL2Ahead = 2;       // groups between an L2 prefetch and the shared-memory load
enum {
    B_PFULL = 0,
    B_XFULL = B_PFULL + SPH,
    B_XEMPTY = B_XFULL + SX,
    B_BXFULL = B_XEMPTY + SX,          // x-pass basis stages
    B_V1DONE = B_BXFULL + SB,
    B_XDONE = B_V1DONE + kDoneV,
    B_B1FULL = B_XDONE + kDoneX,       // two slots: the B operand of group g lives in slot g % 2
    B_D1EMPTY = B_B1FULL + 2,
    B_WFULL,
    B_D2EMPTY,
    B_STG,                             // the epilogue warps have left the W buffer (D2 staging)
    B_FIN,
    B_COUNT
};

// barriers, then the TMEM base-address slot and the abort flag
constexpr uint32_t kBarBytes = ((B_COUNT * 8u + 8u) + 127u) & ~127u;
static_assert(B_COUNT * 8 + 8 <= (int)kBarBytes, "barrier region too small");

struct SmemPlan {
    uint32_t pring, xring, bxring, b1, w, bars, total;
};

// B operand of one column: 32 rows ([x_hi; x_lo]) x nwp FP16, plus 16 bytes so that the
// eight columns of a group fall in different banks
__host__ __device__ constexpr uint32_t b1_stride(int nwp) { return 64u * nwp + 16u; }

__host__ __device__ constexpr SmemPlan smem_plan(int nwp) {
    SmemPlan s{};
    uint32_t o = 0;
    s.pring = o;
    o += SPH * HG * 256u * nwp;          // per slot: 4 images of 128 rows x nwp x 2 B
    s.xring = o;
    o += SX * 512u * nwp;                // RC x nwp x GC x 4 B
    s.bxring = o;
    o += SB * kBxStage;
    o = (o + 127u) & ~127u;
    s.b1 = o;
    o += 2 * GC * b1_stride(nwp);
    o = (o + 127u) & ~127u;
    s.w = o;
    o += kWBytes;
    s.bars = o;
    o += kBarBytes;
    s.total = o;
    return s;
}
static_assert(smem_plan(32).total <= 232448, "shared memory plan exceeds 227 KB");

// Bounded waits.  The first poll is the non-blocking test_wait (cheaper than a try_wait on a
// completed phase); the clock and the abort flag are looked at only every 1024 polls.  The
// single-thread roles (producers, MMA issuers) keep polling with test_wait, so they react to a
// completed phase within one poll; whole warps use try_wait, whose suspension leaves the issue
// slots of their scheduler to the warps that share it (polling everywhere measured no faster).
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

// Wait used by whole warps before warp-collective tcgen05.ld: the outcome is made warp-uniform.
__device__ __forceinline__ bool warp_wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    const bool ok = wait_bar_t<kWarpSpin>(bar, parity, abort_flag);
    return __all_sync(0xffffffffu, ok);
}

__device__ __forceinline__ void fail(volatile int* abort_flag, int* err, int code) {
    *abort_flag = 1;
    atomicCAS(err, 0, code);
}

__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Bounded drain of a producer ring slot: wait for the last phase issued into it.
__device__ __forceinline__ void drain_slot(uint64_t* bar, uint32_t issued, uint32_t slot, uint32_t depth) {
    if (issued <= slot) return;
    const uint32_t n = (issued - slot + depth - 1) / depth;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, (n - 1) & 1u) && (unsigned long long)(clock64() - t0) < kWaitCycles) {}
}

template <int NWP>
__global__ void __launch_bounds__(kThreadsTc, 1)
fwd_column_tc_kernel(const __grid_constant__ CUtensorMap tmap_x, const __half* __restrict__ pimg,
                     const uint8_t* __restrict__ bximg, float* __restrict__ t1, int* __restrict__ err,
                     int R, int K, int nx, int ny, int pxp, int starve, int y0, unsigned* __restrict__ t1max) {
    constexpr int nwp = NWP;
    extern __shared__ __align__(1024) uint8_t smem[];
    constexpr SmemPlan sp = smem_plan(NWP);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem + sp.bars);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + B_COUNT);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    uint8_t* spring = smem + sp.pring;
    uint8_t* sxring = smem + sp.xring;
    uint8_t* sbxring = smem + sp.bxring;
    uint8_t* sb1 = smem + sp.b1;
    uint8_t* sw = smem + sp.w;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int n_rc = (R + RC - 1) / RC;
    const int units = ny * n_rc;
    const int G = nx / GC;
    // units of this CTA: blockIdx.x + i * gridDim.x; groups (and half-groups) are numbered across them
    const int my_units = blockIdx.x < units ? (units - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    const uint32_t total_groups = (uint32_t)my_units * (uint32_t)G;
    constexpr uint32_t PBYTES = 256u * NWP;
    constexpr uint32_t PSLOT = HG * PBYTES;
    constexpr uint32_t XBYTES = 512u * NWP;
    constexpr uint32_t B1S = b1_stride(NWP);
    constexpr uint32_t B1SLOT = GC * B1S;
    constexpr uint32_t b1_sbo = (uint32_t)(NWP / 8) * 128u;

    if (tid == 0) {
        for (int i = 0; i < SPH; ++i) mbar_init(&bars[B_PFULL + i], 1);
        for (int i = 0; i < SX; ++i) {
            mbar_init(&bars[B_XFULL + i], 1);
            mbar_init(&bars[B_XEMPTY + i], kEpiThreads);
        }
        for (int i = 0; i < SB; ++i) mbar_init(&bars[B_BXFULL + i], 1);
        for (int i = 0; i < kDoneV; ++i) mbar_init(&bars[B_V1DONE + i], 1);
        for (int i = 0; i < kDoneX; ++i) mbar_init(&bars[B_XDONE + i], 1);
        mbar_init(&bars[B_B1FULL], kEpiThreads);
        mbar_init(&bars[B_B1FULL + 1], kEpiThreads);
        mbar_init(&bars[B_D1EMPTY], kEpiThreads);
        mbar_init(&bars[B_WFULL], kEpiThreads);
        mbar_init(&bars[B_D2EMPTY], kEpiThreads);
        mbar_init(&bars[B_STG], kEpiThreads);
        mbar_init(&bars[B_FIN], 2);            // one commit per issuer
        *abort_flag = 0;
        fence_mbar_init();
        prefetch_tmap(&tmap_x);
    }
    if (warp == kMmaWarp) tmem_alloc(tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = *tslot;

    if (warp == 0) {
        // ------------------------------------------------------------ producer: images + x-pass basis
        // (starve: a test of the failure path; no copy is issued, so the V1 issuer's bounded
        // wait for the first image runs out)
        if (lane == 0 && !starve) {
            uint32_t pc = 0, bc = 0;           // half-groups, basis stages issued
            for (uint32_t n = 0; n < 2 * total_groups; ++n) {
                const uint32_t gi = n >> 1;
                const int u = (int)blockIdx.x + (int)(gi / G) * (int)gridDim.x;
                const int y = u / n_rc;
                // image slot n % SPH was last used by V1 of half-group n - SPH; for even n = 2gi the
                // basis stage gi % SB was last used by the x-pass of group gi - SB
                const uint32_t ps = n % SPH;
                if (n >= SPH) {
                    const uint32_t np = n - SPH;
                    if (!wait_bar(&bars[B_V1DONE + np % kDoneV], (np / kDoneV) & 1u, abort_flag)) { fail(abort_flag, err, 1); break; }
                }
                if ((n & 1u) == 0) {
                    const uint32_t bs = bc % SB;
                    if (gi >= (uint32_t)SB) {
                        const uint32_t gp = gi - SB;
                        if (!wait_bar(&bars[B_XDONE + gp % kDoneX], (gp / kDoneX) & 1u, abort_flag)) { fail(abort_flag, err, 1); break; }
                    }
                    mbar_arrive_expect_tx(&bars[B_BXFULL + bs], kBxStage);
                    bulk_g2s(sbxring + bs * kBxStage, bximg + (size_t)(gi % G) * kBxStage, kBxStage, &bars[B_BXFULL + bs]);
                    ++bc;
                }
                mbar_arrive_expect_tx(&bars[B_PFULL + ps], PSLOT);
                const size_t col = (size_t)(y + y0) * nx + (size_t)(gi % G) * GC + (n & 1u) * HG;
                bulk_g2s(spring + ps * PSLOT, pimg + col * 128u * nwp, PSLOT, &bars[B_PFULL + ps]);
                ++pc;
                // warm L2 with the eight images of the group this CTA reaches two groups later
                const uint32_t ga = gi + kL2Ahead;
                if ((n & 1u) == 0 && ga < total_groups) {
                    const int ua = (int)blockIdx.x + (int)(ga / G) * (int)gridDim.x;
                    const size_t cola = (size_t)(ua / n_rc + y0) * nx + (size_t)(ga % G) * GC;
                    prefetch_l2(pimg + cola * 128u * nwp, GC * PBYTES);
                }
            }
            // every issued copy must land before the CTA exits
            for (uint32_t s = 0; s < SPH; ++s) drain_slot(&bars[B_PFULL + s], pc, s, SPH);
            for (uint32_t s = 0; s < SB; ++s) drain_slot(&bars[B_BXFULL + s], bc, s, SB);
        }
    } else if (warp == kXWarp) {
        // ------------------------------------------------------------ producer: x tiles
        if (lane == 0) {
            uint32_t xc = 0;
            for (uint32_t gi = 0; gi < total_groups; ++gi) {
                const int u = (int)blockIdx.x + (int)(gi / G) * (int)gridDim.x;
                const int g = (int)(gi % G);
                const int y = u / n_rc, r0 = (u % n_rc) * RC;
                const uint32_t xs = xc % SX, xph = (xc / SX) & 1u;
                if (!wait_bar(&bars[B_XEMPTY + xs], xph ^ 1u, abort_flag)) { fail(abort_flag, err, 1); break; }
                mbar_arrive_expect_tx(&bars[B_XFULL + xs], XBYTES);
                tma_load_3d(sxring + xs * XBYTES, &tmap_x, y * nx + g * GC, 0, r0, &bars[B_XFULL + xs]);
                ++xc;
                const uint32_t ga = gi + kL2Ahead;
                if (ga < total_groups) {
                    const int ua = (int)blockIdx.x + (int)(ga / G) * (int)gridDim.x;
                    prefetch_l2_3d(&tmap_x, (ua / n_rc) * nx + (int)(ga % G) * GC, 0, (ua % n_rc) * RC);
                }
            }
            for (uint32_t s = 0; s < SX; ++s) drain_slot(&bars[B_XFULL + s], xc, s, SX);
        }
    } else if (warp == kMmaWarp) {
        // ------------------------------------------------------------ V1 MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc_v1 = idesc_f16_f32(128, N1);
            constexpr uint32_t a_sbo = (uint32_t)(NWP / 8) * 128u;
            // Base descriptors: an operand b bytes further on is the base plus (b >> 4) in the
            // start-address field, so each MMA below costs one 64-bit add per operand.
            const uint64_t dA0 = smem_desc(smem_u32(spring), 128u, a_sbo);
            const uint64_t dB0 = smem_desc(smem_u32(sb1), 128u, b1_sbo);
            bool ok = true;
            // V1 of half-group n (columns 4(n % 2) .. +3 of group n / 2) into the D1 columns
            for (uint32_t n = 0; n < 2 * total_groups && ok; ++n) {
                const uint32_t g = n >> 1, h = n & 1u;
                // the B operand of group g serves both half-groups: its wait is done once
                if (h == 0 && !wait_bar(&bars[B_B1FULL + (g & 1u)], (g >> 1) & 1u, abort_flag)) { ok = false; break; }
                if (!wait_bar(&bars[B_D1EMPTY], (n & 1u) ^ 1u, abort_flag)) { ok = false; break; }
                const uint64_t db = dB0 + (((g & 1u) * B1SLOT + h * HG * B1S) >> 4);
                const uint32_t ps = n % SPH;
                if (!wait_bar(&bars[B_PFULL + ps], (n / SPH) & 1u, abort_flag)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int j = 0; j < HG; ++j) {
                    const uint64_t da = dA0 + ((ps * PSLOT + (uint32_t)j * PBYTES) >> 4);
#pragma unroll
                    for (int ks = 0; ks < NWP / 16; ++ks)
                        mma_f16(tbase + kD1Col + (uint32_t)(j * N1), da + (uint64_t)(ks * 16),
                                db + (uint64_t)((j * B1S + ks * 256u) >> 4), idesc_v1, ks > 0 ? 1u : 0u);
                }
                mma_commit(&bars[B_V1DONE + n % kDoneV]);   // D1, B1, the image slot
            }
            if (!ok) fail(abort_flag, err, 2);
            mma_commit(&bars[B_FIN]);
            const long long t0 = clock64();
            while (!mbar_try_wait(&bars[B_FIN], 0) && (unsigned long long)(clock64() - t0) < kWaitCycles) {}
        }
    } else if (warp == kXpassWarp) {
        // ------------------------------------------------------------ x-pass MMA issuer
        if (lane == 0) {
            constexpr uint32_t idesc_x = idesc_f16_f32(128, N2);
            const uint64_t dW0 = smem_desc(smem_u32(sw), kWChunk, 128u);
            const uint64_t dX0 = smem_desc(smem_u32(sbxring), kBxChunk, 128u);
            bool ok = true;
            // x-pass of group gi (W, the basis stage and, first group of a unit, the drained D2)
            for (uint32_t gi = 0; gi < total_groups && ok; ++gi) {
                const uint32_t bs = gi % SB;
                const bool first = (gi % G) == 0;
                if (!wait_bar(&bars[B_WFULL], gi & 1u, abort_flag)) { ok = false; break; }
                if (first && !wait_bar(&bars[B_D2EMPTY], ((gi / G) & 1u) ^ 1u, abort_flag)) { ok = false; break; }
                if (!wait_bar(&bars[B_BXFULL + bs], (gi / SB) & 1u, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint64_t db0 = dX0 + ((bs * kBxStage) >> 4);   // K-chunks [b_hi | b_hi]
                const uint64_t db1 = db0 + (kBxChunk >> 4);          // K-chunks [b_hi | b_lo]
                const uint64_t dw0 = dW0 + (kWChunk >> 4);           // K-chunks [W_hi | W_c]
                const uint64_t dw1 = dW0;                            // K-chunks [W_lo | W_hi]
                const uint32_t acc0 = first ? 0u : 1u;
#pragma unroll
                for (int t = 0; t < MT; ++t) mma_f16(tbase + (uint32_t)(t * N2), dw0 + ((t * 2048u) >> 4), db0, idesc_x, acc0);
#pragma unroll
                for (int t = 0; t < MT; ++t) mma_f16(tbase + (uint32_t)(t * N2), dw1 + ((t * 2048u) >> 4), db1, idesc_x, 1u);
                mma_commit(&bars[B_XDONE + gi % kDoneX]);   // W, the basis stage, D2 of a finished unit
            }
            if (!ok) fail(abort_flag, err, 2);
            mma_commit(&bars[B_FIN]);
            const long long t0 = clock64();
            while (!mbar_try_wait(&bars[B_FIN], 0) && (unsigned long long)(clock64() - t0) < kWaitCycles) {}
        }
    } else {
        // ------------------------------------------------------------ converters + epilogue
        const int ew = warp - kEpiWarp0;               // 0 .. NEPI-1
        const int q = warp & 3;                        // TMEM lane quarter this warp may access
        const int rset = ew >> 2;                      // rhs half of the unit this warp finalises
        const uint32_t lane_off = (uint32_t)(32 * q) << 16;
        const int kk = (q & 1) * 32 + lane;            // member of this thread's TMEM lane
        const bool hi_part = q < 2;                    // lanes < 64: P_hi x, lanes >= 64: P_lo x
        bool ok = true;

        // x tile of group c ([RC][nwp][GC] FP32) -> B operand slot c % 2: per column, rows
        // 0..15 = x_hi, 16..31 = x_lo.  A warp handles one (rhs, octet of levels) per step:
        // lane (il, j) reads levels il and il + 4 of column j (conflict-free: 32 distinct
        // banks), one shuffle pairs neighbouring levels, and each lane stores one 4-byte
        // pair of x_hi and one of x_lo (banks 4j + pair: conflict-free).
        auto convert = [&](uint32_t c) -> bool {
            const uint32_t xs = c % SX, xph = (c / SX) & 1u;
            if (!warp_wait_bar(&bars[B_XFULL + xs], xph, abort_flag)) return false;
            const float* xt = reinterpret_cast<const float*>(sxring + xs * XBYTES);
            uint8_t* b1 = sb1 + (c & 1u) * B1SLOT;
            const int il = lane >> 3, j = lane & 7;
            const bool odd = (il & 1) != 0;
            const int l0 = odd ? il + 3 : il;          // first level of this lane's pair in the octet
#pragma unroll 2
            for (int it = ew; it < RC * (NWP / 8); it += NEPI) {
                const int r = it / (NWP / 8), o = it % (NWP / 8);
                const float* src = xt + (r * NWP + 8 * o) * GC + j;
                const float a = src[il * GC];
                const float b = src[(il + 4) * GC];
                const float recv = __shfl_xor_sync(0xffffffffu, odd ? a : b, 8);
                uint32_t hi, lo;
                split2(odd ? recv : a, odd ? b : recv, hi, lo);
                uint8_t* dst = b1 + j * B1S + (r >> 3) * b1_sbo + o * 128u + (r & 7) * 16u + l0 * 2u;
                *reinterpret_cast<uint32_t*>(dst) = hi;
                *reinterpret_cast<uint32_t*>(dst + 32u * NWP) = lo;   // rows 16..31
            }
            fence_proxy_async_smem();
            mbar_arrive(&bars[B_B1FULL + (c & 1u)]);
            mbar_arrive(&bars[B_XEMPTY + xs]);
            return true;
        };

        // D2 of a finished unit (its last x-pass has completed): rows (r, k) -> t1[y][r0 + r][k][0..pxp).
        // A warp's 32 rows of a tile are one member block of one rhs, i.e. 32 consecutive rows of
        // t1: each lane puts its row into the warp's staging area (the W buffer is free here: the
        // x-pass that read it has completed) and the warp then writes the block with coalesced
        // 16-byte stores.
        auto drain_d2 = [&](uint32_t gl) -> bool {
            const int u = (int)blockIdx.x + (int)(gl / G) * (int)gridDim.x;
            const int y = u / n_rc, r0 = (u % n_rc) * RC;
            float4* stg = reinterpret_cast<float4*>(sw + (uint32_t)ew * 32u * (uint32_t)pxp * 4u);
            const int q4 = pxp / 4;                                  // float4 per row
            tc_fence_after();
#pragma unroll 1
            for (int t = rset; t < MT; t += 2) {
                const int row0 = 128 * t + 32 * q;                   // the warp's first row
                const int r = row0 >> 6, k0 = row0 & 63;             // one rhs, members k0 .. k0 + 31
                static_assert(N2 == 48, "three 16-column TMEM loads per row");
                uint32_t d0[16], d1[16], d2[16];
                tmem_ld16(tbase + lane_off + (uint32_t)(t * N2), d0);
                tmem_ld16(tbase + lane_off + (uint32_t)(t * N2 + 16), d1);
                tmem_ld16(tbase + lane_off + (uint32_t)(t * N2 + 32), d2);
                tmem_ld_wait();
                tmem_regs_ready(d0);
                tmem_regs_ready(d1);
                tmem_regs_ready(d2);
                const int nk = min(32, K - k0);                      // member rows of this block that exist
                const bool live = r0 + r < R && nk > 0;
                if (t1max != nullptr) {   // max |t1| of the launch, for the y-pass's FP16 scaling
                    float mx = 0.f;
                    if (live && lane < nk)
#pragma unroll
                        for (int i = 0; i < 16; ++i)
                            mx = fmaxf(mx, fmaxf(fabsf(__uint_as_float(d0[i])),
                                                 fmaxf(fabsf(__uint_as_float(d1[i])), fabsf(__uint_as_float(d2[i])))));
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                    if (lane == 0) atomicMax(t1max, __float_as_uint(mx));
                }
                if (live) {
                    float4* mine = stg + lane * q4;
                    auto put = [&](int c, const uint32_t (&d)[16], int i) {
                        if (c < q4)
                            mine[c] = make_float4(__uint_as_float(d[i]), __uint_as_float(d[i + 1]), __uint_as_float(d[i + 2]),
                                                  __uint_as_float(d[i + 3]));
                    };
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        put(c, d0, 4 * c);
                        put(4 + c, d1, 4 * c);
                        put(8 + c, d2, 4 * c);
                    }
                    __syncwarp();
                    float4* dst = reinterpret_cast<float4*>(t1 + (((size_t)y * R + r0 + r) * K + k0) * pxp);
                    for (int i = lane; i < nk * q4; i += 32) dst[i] = stg[i];
                    __syncwarp();
                }
            }
            tc_fence_before();
            mbar_arrive(&bars[B_D2EMPTY]);
            return true;
        };

        if (total_groups > 0 && !convert(0)) ok = false;
        if (ok && total_groups > 1 && !convert(1)) ok = false;
        // D1 of half-group n: 4 columns x (8 rhs x_hi products + 8 rhs x_lo products) -> w
        auto drain_d1 = [&](uint32_t n, float (&w)[HG][8]) -> bool {
            if (!warp_wait_bar(&bars[B_V1DONE + n % kDoneV], (n / kDoneV) & 1u, abort_flag)) return false;
            tc_fence_after();
            uint32_t vh[HG][8], vl[HG][8];             // products with x_hi and with x_lo
#pragma unroll
            for (int j = 0; j < HG; ++j) {
                tmem_ld8(tbase + lane_off + kD1Col + (uint32_t)(j * N1 + rset * 8), vh[j]);
                tmem_ld8(tbase + lane_off + kD1Col + (uint32_t)(j * N1 + RC + rset * 8), vl[j]);
            }
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < HG; ++j) {
                tmem_regs_ready(vh[j]);
                tmem_regs_ready(vl[j]);
            }
            tc_fence_before();
            mbar_arrive(&bars[B_D1EMPTY]);
#pragma unroll
            for (int j = 0; j < HG; ++j)
#pragma unroll
                for (int rl = 0; rl < 8; ++rl) w[j][rl] = __uint_as_float(vh[j][rl]) + __uint_as_float(vl[j][rl]);
            return true;
        };

        // One iteration per group, both V1 half-groups in sequence (the sums of the first
        // half-group never cross a loop iteration).
        bool pending = false;                          // a finished unit whose D2 is still to be drained
        uint32_t pending_g = 0, ndrain = 0;
        for (uint32_t g = 0; g < total_groups && ok; ++g) {
            float s0[HG][8], s1[HG][8];                // w of this lane: column x rhs (8 of the unit's 16)
            // ---- first half-group: columns 0-3
            if (!drain_d1(2 * g, s0)) { ok = false; break; }
            // V1 of group g - 1 has completed, so its B operand slot takes group g + 1; the MMA
            // thread needs that slot a whole group later, while D1 is needed right away
            if (g >= 1 && g + 1 < total_groups && !convert(g + 1)) { ok = false; break; }
            // ---- second half-group: columns 4-7
            if (!drain_d1(2 * g + 1, s1)) { ok = false; break; }
            // ---- the x-pass of group g - 1 has completed: W is free, and a unit that ended at
            // group g - 1 has its whole row in D2
            if (g >= 1) {
                const uint32_t gp = g - 1;
                if (!warp_wait_bar(&bars[B_XDONE + gp % kDoneX], (gp / kDoneX) & 1u, abort_flag)) { ok = false; break; }
            }
            if (pending) {
                if (!drain_d2(pending_g)) { ok = false; break; }
                pending = false;
                // the D2 staging used the W buffer: every epilogue warp must be done with it
                mbar_arrive(&bars[B_STG]);
                if (!warp_wait_bar(&bars[B_STG], ndrain & 1u, abort_flag)) { ok = false; break; }
                ++ndrain;
            }
            // ---- W of group g: rows (r, k), 8 columns per 16-byte row in each K-chunk
#pragma unroll
            for (int rl = 0; rl < 8; ++rl) {
                const uint32_t row = (uint32_t)(rset * 8 + rl) * 64u + (uint32_t)kk;
                const uint32_t off = (row >> 3) * 128u + (row & 7u) * 16u;
                if (hi_part) {
                    uint4 hi, lo;
                    split2(s0[0][rl], s0[1][rl], hi.x, lo.x);
                    split2(s0[2][rl], s0[3][rl], hi.y, lo.y);
                    split2(s1[0][rl], s1[1][rl], hi.z, lo.z);
                    split2(s1[2][rl], s1[3][rl], hi.w, lo.w);
                    *reinterpret_cast<uint4*>(sw + kWChunk + off) = hi;   // W_hi
                    *reinterpret_cast<uint4*>(sw + off) = lo;             // W_lo
                } else {
                    const uint4 c = make_uint4(pack_half2(s0[0][rl], s0[1][rl]), pack_half2(s0[2][rl], s0[3][rl]),
                                               pack_half2(s1[0][rl], s1[1][rl]), pack_half2(s1[2][rl], s1[3][rl]));
                    *reinterpret_cast<uint4*>(sw + 2 * kWChunk + off) = c;   // W_c
                }
            }
            fence_proxy_async_smem();
            mbar_arrive(&bars[B_WFULL]);
            if ((g % G) == (uint32_t)G - 1) {
                pending = true;
                pending_g = g;
            }
        }
        if (ok && pending) {
            const uint32_t gp = total_groups - 1;
            if (!warp_wait_bar(&bars[B_XDONE + gp % kDoneX], (gp / kDoneX) & 1u, abort_flag) || !drain_d2(pending_g)) ok = false;
        }
        if (!ok) fail(abort_flag, err, 3);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == kMmaWarp) {
        __syncwarp();
        tmem_dealloc(tbase, kTmemCols);
    }
}

// Pseudo-inverse image: pimg[m][row][l] in the K-major core-matrix layout,
// row < 64: P_hi[k = row], row >= 64: P_lo[k = row - 64]; zero outside K x n_w.
__global__ void build_pimg_kernel(const float* __restrict__ P, __half* __restrict__ pimg, int K, int nw, int nwp,
                                  long long nh) {
    const long long total = nh * 64 * nwp;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total; i += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(i % nwp);
        const int k = (int)((i / nwp) % 64);
        const long long m = i / ((long long)nwp * 64);
        const float v = (k < K && l < nw) ? P[((long long)k * nw + l) * nh + m] : 0.f;
        const __half hi = __float2half_rn(v);
        const __half lo = __float2half_rn(v - __half2float(hi));
        uint8_t* base = reinterpret_cast<uint8_t*>(pimg) + (size_t)m * 256u * nwp;
        const uint32_t sbo = (uint32_t)(nwp / 8) * 128u;
        *reinterpret_cast<__half*>(base + kmajor_offset((uint32_t)k, (uint32_t)l, 128u, sbo)) = hi;
        *reinterpret_cast<__half*>(base + kmajor_offset((uint32_t)(k + 64), (uint32_t)l, 128u, sbo)) = lo;
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

double basis_value_d(int N, int p, int m) {
    if (p == 0) return 1.0 / std::sqrt((double)N);
    if (N % 2 == 0 && p == N - 1) return ((m & 1) ? -1.0 : 1.0) / std::sqrt((double)N);
    const int j = (p + 1) / 2;
    const long long r = ((long long)j * m) % N;
    const double a = 2.0 * M_PI * (double)r / (double)N;
    return std::sqrt(2.0 / N) * ((p & 1) ? std::cos(a) : std::sin(a));
}

}  // namespace

bool tc_supported(const zl_plan_s& p) {
    return p.d.nx % GC == 0 && p.d.K <= 64 && p.d.nw <= 32 && p.Px <= N2 && p.nh % 4 == 0;
}

zl_status tc_prepare(zl_plan_s& p, cudaStream_t s) {
    if (!tc_supported(p) || encode_fn() == nullptr) return ZL_ERR_UNSUPPORTED;
    int dev = 0, sms = 0, cc_major = 0, cc_minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return ZL_ERR_CUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (cc_major != 10) return ZL_ERR_UNSUPPORTED;
    TcOperands* t = new TcOperands();
    t->nwp = p.d.nw <= 16 ? 16 : 32;
    t->pxp = (p.Px + 3) / 4 * 4;
    t->num_sms = sms;
    t->smem = smem_plan(t->nwp).total;
    const int nx = p.d.nx;
    cudaError_t e = cudaSuccess;
    const size_t pimg_bytes = (size_t)p.nh * 256u * t->nwp;
    const size_t bx_bytes = (size_t)(nx / GC) * kBxStage;
    e = zl::dev_malloc((void**)&t->pimg, pimg_bytes);
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&t->bximg, bx_bytes);
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&t->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(t->pimg, 0, pimg_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(t->d_err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        build_pimg_kernel<<<1184, 256, 0, s>>>(reinterpret_cast<const float*>(p.P), t->pimg, p.d.K, p.d.nw, t->nwp, p.nh);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        // x-pass basis image, one stage per 8-column group g: K-chunk c holds
        // B[jx][m] = b_{p_x}(8g + m), split hi (chunks 0 and 1) / lo (chunk 2); rows jx >= Px are 0
        std::vector<__half> img(bx_bytes / 2, __float2half_rn(0.f));
        for (int g = 0; g < nx / GC; ++g)
            for (int c = 0; c < 3; ++c)
                for (int jx = 0; jx < p.Px; ++jx)
                    for (int m = 0; m < GC; ++m) {
                        const double b = basis_value_d(nx, p.xfreq[jx], g * GC + m);
                        const __half hi = __double2half(b);
                        const __half v = c < 2 ? hi : __double2half(b - (double)__half2float(hi));
                        const size_t off = (size_t)g * kBxStage +
                                           kmajor_offset((uint32_t)jx, (uint32_t)(c * GC + m), kBxChunk, 128u);
                        img[off / 2] = v;
                    }
        e = cudaMemcpyAsync(t->bximg, img.data(), bx_bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    // t1 rows are padded to pxp for 16-byte stores
    if (e == cudaSuccess && t->pxp != p.Px) {
        void* t1 = nullptr;
        e = zl::dev_malloc((void**)&t1, (size_t)p.d.max_rhs * p.d.K * p.d.ny * t->pxp * sizeof(float));
        if (e == cudaSuccess) {
            cudaFree(p.t1);
            p.t1 = t1;
        }
    }
    if (e == cudaSuccess)
        e = t->nwp == 16
                ? cudaFuncSetAttribute(fwd_column_tc_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem)
                : cudaFuncSetAttribute(fwd_column_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)t->smem);
    if (e == cudaSuccess) {   // the tensor-core y-pass, where its shape fits (else the CUDA-core one)
        const zl_status ys = ytc_prepare(p, t->pxp, s);
        if (ys != ZL_OK && ys != ZL_ERR_UNSUPPORTED) e = ys == ZL_ERR_ALLOC ? cudaErrorMemoryAllocation : cudaErrorUnknown;
    }
    if (e != cudaSuccess) {
        ytc_release(p);
        cudaFree(t->pimg);
        cudaFree(t->bximg);
        cudaFree(t->d_err);
        delete t;
        return e == cudaErrorMemoryAllocation ? ZL_ERR_ALLOC : ZL_ERR_CUDA;
    }
    p.tc = t;
    return ZL_OK;
}

void tc_release(zl_plan_s& p) {
    ytc_release(p);
    if (!p.tc) return;
    cudaFree(p.tc->pimg);
    cudaFree(p.tc->bximg);
    cudaFree(p.tc->d_err);
    delete p.tc;
    p.tc = nullptr;
}

int tc_t1_stride(const zl_plan_s& p) { return p.tc ? p.tc->pxp : p.Px; }

cudaError_t tc_clear_error(const zl_plan_s& p) {
    if (p.d_werr) {
        const cudaError_t e = cudaMemset(p.d_werr, 0, sizeof(int));
        if (e != cudaSuccess) return e;
    }
    if (!p.tc) return cudaSuccess;
    const cudaError_t e = cudaMemset(p.tc->d_err, 0, sizeof(int));
    return e != cudaSuccess ? e : ytc_clear_error(p);
}

// The code of the TMA-fed FP32 column kernel (plus 32), else the tensor-core column
// kernel's, else the tensor-core y-pass's (plus 16).
cudaError_t tc_read_error(const zl_plan_s& p, int* code) {
    *code = 0;
    if (p.d_werr) {
        int w = 0;
        const cudaError_t e = cudaMemcpy(&w, p.d_werr, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return e;
        if (w != 0) {
            *code = 32 + w;
            return cudaSuccess;
        }
    }
    if (!p.tc) return cudaSuccess;
    cudaError_t e = cudaMemcpy(code, p.tc->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || *code != 0) return e;
    int yc = 0;
    e = ytc_read_error(p, &yc);
    if (yc != 0) *code = 16 + yc;
    return e;
}

cudaError_t forward_tc(const zl_plan_s& p, const float* x, float* out, int R, cudaStream_t s, Rows rows,
                       const float* scale) {
    const TcOperands& t = *p.tc;
    CUtensorMap tmap;
    // x holds the grid rows rows.y0 .. rows.y0 + rows.ny - 1 (the whole grid by default)
    const cuuint64_t nhx = (cuuint64_t)rows.ny * p.d.nx;
    const cuuint64_t gdim[3] = {nhx, (cuuint64_t)p.d.nw, (cuuint64_t)R};
    const cuuint64_t gstride[2] = {nhx * sizeof(float), nhx * p.d.nw * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)GC, (cuuint32_t)t.nwp, (cuuint32_t)RC};
    const cuuint32_t estride[3] = {1, 1, 1};
    const CUresult cr = encode_fn()(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(x), gdim, gstride, box,
                                    estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return cudaErrorInvalidValue;
    const int units = rows.ny * ((R + RC - 1) / RC);
    const int grid = units < t.num_sms ? units : t.num_sms;
    // the tensor-core y-pass needs the whole grid (its basis image starts at row 0) and max |t1|
    const bool ytc = p.ytc != nullptr && rows.y0 == 0 && rows.ny == p.d.ny;
    unsigned* t1max = ytc ? ytc_max_word(p) : nullptr;
    if (t1max != nullptr) {
        const cudaError_t em = cudaMemsetAsync(t1max, 0, sizeof(unsigned), s);
        if (em != cudaSuccess) return em;
    }
    p.timer.begin(ZL_STAGE_FWD_COLUMN, s);
    if (t.nwp == 16)
        fwd_column_tc_kernel<16><<<grid, kThreadsTc, t.smem, s>>>(tmap, t.pimg, t.bximg, reinterpret_cast<float*>(p.t1),
                                                                  t.d_err, R, p.d.K, p.d.nx, rows.ny, t.pxp,
                                                                  p.test_wait_timeout, rows.y0, t1max);
    else
        fwd_column_tc_kernel<32><<<grid, kThreadsTc, t.smem, s>>>(tmap, t.pimg, t.bximg, reinterpret_cast<float*>(p.t1),
                                                                  t.d_err, R, p.d.K, p.d.nx, rows.ny, t.pxp,
                                                                  p.test_wait_timeout, rows.y0, t1max);
    p.timer.end(s);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (ytc) return forward_ypass_tc(p, reinterpret_cast<const float*>(p.t1), t.pxp, scale, out, R, s);
    return forward_ypass_f32(p, reinterpret_cast<const float*>(p.t1), t.pxp, scale, out, R, s, rows);
}

}  // namespace zl
