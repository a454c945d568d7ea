// Internal declarations shared by the libzl translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <vector>

#include "../../include/zl.h"

namespace zl {

// Device-resident tables of the horizontal transform, in the plan's element type T.
//   bx      [Px][nx]   b_{p_x}(x) for the kept x-frequencies, in kept order
//   by      [ny][ny]   b_{p_y}(y), row p_y
//   m_py    [L]        packed y-index of output mode j
//   m_jx    [L]        index into the kept x-frequency list of output mode j
//   inv_sqrt_lam, sqrt_lam [L]
//   grp_start [Px+1], grp_modes [L]: output modes grouped by jx (for the inverse y-pass)
template <typename T>
struct Tables {
    T* bx = nullptr;
    T* by = nullptr;
    T* inv_sqrt_lam = nullptr;
    T* sqrt_lam = nullptr;
    int* m_py = nullptr;
    int* m_jx = nullptr;
    int* grp_start = nullptr;
    int* grp_modes = nullptr;
    int* m_ipy = nullptr;   // [L] index of mode j's p_y in the list of kept y-frequencies
    T* byk = nullptr;       // [ny][pys] b_{p_y}(y) of the kept y-frequencies, zero-padded to pys
    int* yneed = nullptr;   // [Px] 1 + the largest m_ipy among the kept modes of x-frequency jx
};

struct TcOperands;   // tensor-core path state (k_tc.cu)
struct YtcOperands;  // tensor-core y-pass state (k_ytc.cu)

// Optional CUDA-event bracketing of every kernel stage (zl_set_stage_timing).
struct StageTimer {
    struct Rec {
        int stage;
        cudaEvent_t a, b;
    };
    bool on = false;
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;   // events of cleared records, reused
    cudaEvent_t take();
    void begin(int stage, cudaStream_t s);
    void end(cudaStream_t s);
    void clear();
    ~StageTimer();
};

}  // namespace zl

struct zl_plan_s {
    zl_desc d;
    int device = 0;         // the CUDA device current at setup
    long long nh = 0;
    int g = 0;              // min(nw, K)
    int L = 0;              // kept modes
    int Px = 0;             // kept x-frequencies
    int Py = 0;             // kept y-frequencies
    int pys = 0;            // Py rounded up to 16 (row stride of the kept y-basis table)
    int bad_column = -1;
    std::vector<int> modes; // kept packed indices (host copy)
    std::vector<double> lamS; // their eigenvalues
    std::vector<int> xfreq; // kept x-frequencies (packed x-index), in the order of the x-pass
    size_t esize = 0;       // element size of caller buffers (8 or 4)

    // member matrices, [K][nw][nh]: the plan's copy of Z and the pseudo-inverse P (P[k][l][m] = (A_m^+)[k][l])
    void* Zc = nullptr;
    void* P = nullptr;
    // intermediate of the separable transform: forward [ny][max_rhs][K][ldp], inverse [max_rhs][K][ny][Px]
    void* t1 = nullptr;
    zl::Tables<double> td;
    zl::Tables<float> tf;
    zl::TcOperands* tc = nullptr;
    zl::YtcOperands* ytc = nullptr;
    // zl_apply_left_inverse_host (allocated on first use): two device staging slots of
    // h_piece right-hand sides each for x and for x~, the copy-in and copy-out streams, and
    // per slot the events "copied in", "kernels done", "copied out"
    void* h_x = nullptr;
    void* h_xt = nullptr;
    int h_piece = 0;
    cudaStream_t h_in = nullptr, h_out = nullptr;
    cudaEvent_t h_start = nullptr, h_in_done[2] = {}, h_comp_done[2] = {}, h_out_done[2] = {};
    int* d_status = nullptr;
    // device word of the TMA-fed FP32 column kernel: 0, or the code of a bounded wait that
    // gave up
    int* d_werr = nullptr;
    mutable zl::StageTimer timer;
    // kernel choice (set by the batch autotuner; defaults = the built-in heuristics):
    // force_plain runs a mixed plan's left inverse on the CUDA-core FP32 kernels instead of
    // the tensor cores, force_rc (1, 2, 4 or 8; 0 = heuristic) fixes the right-hand sides per
    // CTA of the CUDA-core forward column kernel
    bool force_plain = false;
    int force_rc = 0;
    // test hook of the failure-detection path (zl_set_test_wait_timeout): the tensor-core
    // kernel's image producer issues no copies, so a bounded wait runs out
    int test_wait_timeout = 0;
};

namespace zl {

// Every device allocation of the library goes through dev_malloc, so that the test hook
// zl_set_test_alloc_failure can make the n-th one fail as if the device were full.
cudaError_t dev_malloc(void** ptr, size_t bytes);

// k_setup.cu
cudaError_t launch_setup_columns(const zl_desc& d, long long nh, const void* Z, void* P, int* d_status,
                                 cudaStream_t s);
size_t setup_smem_bytes(int nw, int K);

// A range of grid rows: y0 .. y0 + ny - 1 (the whole grid: {0, desc.ny}).
struct Rows {
    int y0;
    int ny;
};

// k_plain.cu: forward (V1-V5 shape) and inverse (V_b, then per-column product) passes
//   forward:  out[r][k][j] = scale[j] * sum_m V_b[m][s_j] * sum_l M[k][l][m] x[r][l][m]
//   inverse:  out[r][l][m] = sum_k M[k][l][m] * sum_j V_b[m][s_j] scale[j] c[r][k][j]
//   forward_plain over a row range: x holds only rows y0 .. y0 + ny - 1 ([R][n_w][ny nx]); the
//   y-sum runs over those rows only, and a null scale leaves the modes unscaled (partial sums)
template <typename T>
cudaError_t forward_plain(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* x, T* out,
                          int R, cudaStream_t s, Rows rows);
template <typename T>
cudaError_t forward_plain_on(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* x, T* out,
                             int R, cudaStream_t s, T* t1);
template <typename T>
cudaError_t inverse_plain(const zl_plan_s& p, const Tables<T>& t, const T* M, const T* scale, const T* c, T* out,
                          int R, cudaStream_t s);

// Loads every kernel forward_plain_on<T> can launch (cudaFuncGetAttributes), so that a
// later launch loads no module code under lazy module loading.
template <typename T>
cudaError_t preload_forward_plain();

// zl_static.cu: the allocation-free entry point's scratch address on p.device, and its kernels
zl_status static_scratch_prepare(const zl_plan_s& p);

// y-pass of the forward transform on an FP32 intermediate with row stride ldp
cudaError_t forward_ypass_f32(const zl_plan_s& p, const float* t1, int ldp, const float* scale, float* out, int R,
                              cudaStream_t s, Rows rows);

// k_diag.cu: matrix-form diagnostics (per-column SVD, Xi, delta)
size_t column_svd_smem_per_warp(int nw, int K);
cudaError_t launch_column_svd(const zl_plan_s& p, double* E, double* Lam, double* F, cudaStream_t s);
cudaError_t launch_xi(const double* M, int n, double* acc, cudaStream_t s);
template <typename T>
cudaError_t launch_scale_modes(const T* partial, const T* scale, T* xt, long long rows, int L, cudaStream_t s);
template <typename T>
cudaError_t launch_delta(const T* xt, const T* back, T* d, double* norms, long long len, int R, cudaStream_t s);

// k_tc.cu: tensor-core left inverse (ZL_MIXED)
bool tc_supported(const zl_plan_s& p);
zl_status tc_prepare(zl_plan_s& p, cudaStream_t s);
void tc_release(zl_plan_s& p);
cudaError_t forward_tc(const zl_plan_s& p, const float* x, float* out, int R, cudaStream_t s, Rows rows,
                       const float* scale);
// TMA-fed FP32 column kernel (k_f32.cu): FP32 data, P_x <= 64, R >= 4, n_x a multiple of 4
bool f32_column_supported(const zl_plan_s& p, int R);
cudaError_t forward_column_f32(const zl_plan_s& p, const float* x, const float* M, const float* bx, float* t1, int R,
                               cudaStream_t s, Rows rows);
// TMA-fed FP32 inverse column pass (k_f32.cu): FP32 data, P_x <= 64, n_w <= 64, R >= 2, n_x a multiple of 4
bool f32_inverse_supported(const zl_plan_s& p, int R);
cudaError_t inverse_column_f32(const zl_plan_s& p, const float* u, const float* M, const float* bx, float* out, int R,
                               cudaStream_t s);

cudaError_t tc_read_error(const zl_plan_s& p, int* code);
cudaError_t tc_clear_error(const zl_plan_s& p);

// k_ytc.cu: tensor-core y-pass of the mixed left inverse (t1 from the tensor-core column kernel)
bool ytc_supported(const zl_plan_s& p, int ldp);
zl_status ytc_prepare(zl_plan_s& p, int ldp, cudaStream_t s);
void ytc_release(zl_plan_s& p);
unsigned* ytc_max_word(const zl_plan_s& p);
cudaError_t ytc_read_error(const zl_plan_s& p, int* code);
cudaError_t ytc_clear_error(const zl_plan_s& p);
cudaError_t forward_ypass_tc(const zl_plan_s& p, const float* t1, int ldp, const float* scale, float* out, int R,
                             cudaStream_t s);

}  // namespace zl
