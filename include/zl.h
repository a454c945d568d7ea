/*
 * zl.h -- C ABI of libzl: the swift left inverse of the square root of a
 * horizontally localized ensemble covariance, on one NVIDIA B300 (sm_103a).
 *
 * Method: Sardelli & Bishop, "A swift algorithm to calculate the left inverse
 * of a square root of a horizontally localized climatological ensemble
 * covariance matrix" (arxiv 2609.13327).
 *
 * Notation (the paper's):
 *   n_h = nx*ny grid columns (index m = y*nx + x), n_w variables per column
 *   (levels x kinds, index l), K members (index k), n = n_w*n_h.
 *   Z     the scaled ensemble z_k = (e_k - mean)/sqrt(K-1) (Sec. 3.3), stored
 *         [K][n_w][n_h]: member-major, then segment l, then column m (the
 *         segment ordering of Sec. 3.4).
 *   C_b   the n_h x n_h horizontal localization block (Sec. 3.6); every block
 *         of the localization equals C_b.  libzl accepts the localizations
 *         diagonalised by the packed real-Fourier basis of a periodic grid
 *         (circulant in 1-D, block-circulant with circulant blocks in 2-D,
 *         even in each axis): the caller gives their eigenvalues.
 *   Zh    = C^{1/2} (triangle) Z = A V Delta^{1/2}, the modulated-ensemble
 *         square root (Sec. 3.7, 3.9), n x K*L.
 *   Zh^-  = Delta^{-1/2} V^T A^{-1}, its left inverse (Sec. 3.9, Eq.
 *         InverseSquareRootAlmost).  When n_w != K, A^{-1} is replaced by the
 *         pseudo-inverse A^+ = blockdiag over columns of A_m^+ (minimum norm
 *         for n_w < K, least squares for n_w > K); this is a genuine left
 *         inverse iff n_w >= K.
 *
 * Packed real-Fourier basis (per axis of length N; s = p_y*nx + p_x in 2-D):
 *   b_0 = 1/sqrt(N); b_{2j-1}(m) = sqrt(2/N) cos(2 pi j m/N);
 *   b_{2j}(m) = sqrt(2/N) sin(2 pi j m/N); b_{N-1}(m) = (-1)^m/sqrt(N) if N even.
 *
 * Conventions for every entry point:
 *   - Device pointers are raw CUDA device addresses, owned by the caller; libzl
 *     never frees them.  Host pointers are plain host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Applies are stream-ordered and asynchronous; nothing in an
 *     apply allocates memory or synchronises the host, except the *_host
 *     variant, which synchronises `stream` before returning.
 *   - Element type follows the plan's precision: double for ZL_FP64, float for
 *     ZL_FP32 and ZL_MIXED (tensor-core operands are internal only).
 *   - No exception or exit crosses the ABI.  Argument errors are detected
 *     before any work is queued, so output buffers are untouched when an
 *     entry point returns ZL_ERR_ARG or ZL_ERR_SHAPE.
 */
#ifndef ZL_H
#define ZL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct zl_plan_s* zl_plan;   /* opaque; owned by libzl, freed by zl_destroy */

typedef enum {
    ZL_OK = 0,
    ZL_ERR_ARG = 1,          /* null pointer, bad enum, non-finite or negative parameter   */
    ZL_ERR_SHAPE = 2,        /* a size outside the supported range                          */
    ZL_ERR_RANK = 3,         /* some A_m is rank-deficient (Gram pivot test), see get_info   */
    ZL_ERR_ALLOC = 4,        /* cudaMalloc failed during setup                              */
    ZL_ERR_CUDA = 5,         /* a CUDA runtime call or kernel launch failed                 */
    ZL_ERR_TIMEOUT = 6,      /* a bounded device-side wait gave up                          */
    ZL_ERR_UNSUPPORTED = 7   /* valid request that this library version does not implement */
} zl_status;

typedef enum {
    ZL_FP64 = 0,   /* FP64 throughout: the plain GPU form of the algorithm                  */
    ZL_FP32 = 1,   /* FP32 CUDA-core arithmetic, FP64 setup                                 */
    ZL_MIXED = 2   /* left inverse on tcgen05 tensor cores (FP16 hi/lo operand splits,
                      FP32 accumulation), FP64 setup; other operators as ZL_FP32            */
} zl_precision;

typedef struct {
    int nx;             /* grid points along x (>= 1)                                        */
    int ny;             /* grid points along y (>= 1; 1 for a ring)                          */
    int nw;             /* variables per vertical column n_w = n_G * n_v (>= 1)              */
    int K;              /* ensemble members (>= 1)                                           */
    zl_precision prec;
    double tau;         /* keep mode s iff lambda_s > tau * max(lambda); tau >= 0            */
    int max_rhs;        /* right-hand sides per internal pass (workspace size); >= 1        */
} zl_desc;

/*
 * zl_setup -- precompute everything the applies need (the paper's experiment
 * steps (a)-(e), Sec. 4.7, and the economical eigendecomposition of C_b,
 * Sec. 3.9).
 *
 *   desc      sizes and precision (copied).
 *   Z         device, [K][nw][ny*nx], double (ZL_FP64) or float; read only
 *             during the call (libzl keeps its own copy).
 *   spectrum  host, [ny*nx] doubles: eigenvalue of C_b for every packed mode s,
 *             all finite, max > 0.  Modes with lambda_s <= tau*max are dropped
 *             ("non-zero eigenvalues", Sec. 3.9); L = number kept.
 *   stream    queue for the setup work; the call synchronises it.
 *             A tau for which no mode is kept (L = 0, e.g. tau >= 1) is
 *             rejected with ZL_ERR_SHAPE before any device work.
 *   out       receives the plan.  On ZL_OK and on ZL_ERR_RANK *out is a valid
 *             plan (on ZL_ERR_RANK every apply returns ZL_ERR_RANK; query the
 *             first rank-deficient column with zl_get_info, then zl_destroy).
 *             On any other error *out is NULL.
 *
 * Per column m the plan holds the pseudo-inverse A_m^+ (K x n_w), formed in
 * FP64 from the Gram matrix G_m = A_m A_m^T (n_w <= K) or A_m^T A_m (n_w > K),
 * its Cholesky factor, and one Newton step P <- P (2I - A_m P) (resp.
 * (2I - P A_m) P) whose residual is formed in FP64.  Column m is
 * rank-deficient when a Cholesky pivot is <= 1e-13 * trace(G_m) (rank(A) =
 * sum_m rank(A_m), supporting information S2).
 */
zl_status zl_setup(const zl_desc* desc, const void* Z, const double* spectrum,
                   void* stream, zl_plan* out);

/*
 * zl_get_info -- sizes of a plan.  Any output pointer may be NULL.
 *   L           kept modes; nw, K, nh as in the descriptor;
 *   bad_column  first rank-deficient column, or -1.
 */
zl_status zl_get_info(zl_plan plan, int* L, int* nw, int* K, long long* nh, int* bad_column);

/* zl_get_desc -- the plan's descriptor (as given to zl_setup or stored by zl_plan_save). */
zl_status zl_get_desc(zl_plan plan, zl_desc* desc);

/*
 * zl_get_runtime_info -- which kernel path the plan's left inverse takes and
 * whether a device-side wait has given up.  Either pointer may be NULL.
 *   tensor_core_path  1 if zl_apply_left_inverse runs the tcgen05 kernel
 *                     (ZL_MIXED plans whose shape it supports: nx a multiple of
 *                     8, nw <= 32, K <= 64, at most 48 kept x-frequencies,
 *                     and not switched to the CUDA-core kernels by the batch
 *                     autotuner), 0 if it runs the CUDA-core kernels.
 *   device_error      0, or the code a TMA-fed kernel recorded when one of its
 *                     bounded waits timed out (the call then returns
 *                     ZL_ERR_TIMEOUT): 1-15 the tensor-core column kernel,
 *                     17-31 the tensor-core y-pass, 33-34 the FP32 column
 *                     kernel.  Reading it synchronises the device.
 *                     The code stays recorded until zl_set_test_wait_timeout
 *                     (plan, 0) clears it; the results of the applies queued
 *                     since the timeout are undefined.
 */
zl_status zl_get_runtime_info(zl_plan plan, int* tensor_core_path, int* device_error);

/*
 * zl_set_test_wait_timeout -- a test hook of the failure-detection path; the
 * paper has no counterpart.  enable = 1: from the next apply on, the
 * copy-issuing thread of the plan's TMA-fed left-inverse kernel (the
 * tensor-core kernel's image producer, or the FP32 column kernel's stage
 * producer) issues no copies, so the first bounded wait for a copy runs out
 * (about 2 s), the kernel records a nonzero device error (the tensor-core
 * kernel frees its TMEM) and returns; the results of such an apply are
 * undefined and zl_get_runtime_info reports ZL_ERR_TIMEOUT.  enable = 0:
 * restores normal operation and clears the recorded device error.  No GPU
 * fault is involved and the context stays usable.  The call synchronises the
 * device.  Errors: ZL_ERR_ARG (invalid plan, enable not 0 or 1),
 * ZL_ERR_UNSUPPORTED (the plan's left inverse runs neither TMA-fed kernel:
 * FP64 plans, or FP32 data with n_x not a multiple of 4, more than 64 kept
 * x-frequencies or max_rhs < 4), ZL_ERR_CUDA.
 */
zl_status zl_set_test_wait_timeout(zl_plan plan, int enable);

/*
 * zl_set_test_alloc_failure -- a test hook of the error paths; the paper has no
 * counterpart.  n > 0: the n-th device allocation the library makes from now on
 * (setup, batch setup, host staging) fails as if the device were full, and the
 * call that made it returns ZL_ERR_ALLOC after releasing everything it had
 * allocated; n = 0 switches the hook off.  Process-wide.  Errors: ZL_ERR_ARG
 * (n < 0).
 *
 * Logging: when the environment variable ZL_LOG is set (and not "0") at the
 * first apply, every apply writes one JSON line to stderr with the operator,
 * R, the sizes, the precision and the column and y-pass kernels it runs.
 */
zl_status zl_set_test_alloc_failure(int n);

/*
 * zl_get_modes -- the kept packed mode indices s (ascending), host int[L].
 * Output coefficient j of every member refers to mode modes[j].
 */
zl_status zl_get_modes(zl_plan plan, int* modes);

/*
 * zl_apply_left_inverse -- x~ = Zh^- x for R state vectors: steps V1-V5 of
 * Sec. 3.10.  V1: w^(m) = A_m^+ x^(m) for every column; V2-V3: regroup w into
 * its K member segments; V4: x~_k = Delta_b^{-1/2} V_b^T w_k; V5: concatenate.
 *
 *   x    device, [R][nw][ny*nx] (segment order), read only.
 *   xt   device, [R][K][L], written; may not alias x.
 *   R    >= 0 (0 is a no-op); any R, processed in passes of max_rhs.
 */
zl_status zl_apply_left_inverse(zl_plan plan, const void* x, void* xt, int R, void* stream);

/*
 * zl_apply_left_inverse_rows -- one slab's share of the left inverse, for a
 * horizontal domain split into slabs of grid rows (the paper's parallel
 * decomposition, Sec. 3.10: steps V1-V3 need only the slab's own columns, and
 * V4's transform along y is a sum over rows).  For the rows y0 .. y1 - 1:
 *   partial[r][k][j] = sum_{y in [y0, y1)} b_{p_y(j)}(y) * c_k(y, p_x(j)),
 *   c_k(y, .) = the x-pass (V_b^T along x) of w_k = A^+ x on grid row y,
 * i.e. x~ without the Delta^{-1/2} scaling.  The sum of the partials of slabs
 * that cover the grid (one all-reduce of K L values per right-hand side when
 * the slabs live on different GPUs), scaled by zl_scale_modes, is
 * zl_apply_left_inverse's result.
 *
 *   y0, y1   0 <= y0 < y1 <= ny, else ZL_ERR_SHAPE
 *   x        device, [R][nw][(y1 - y0) * nx]: the slab's rows of every segment
 *            (the rows a rank holding the slab stores), read only
 *   partial  device, [R][K][L], written
 * Same kernels, precision and passes of max_rhs as zl_apply_left_inverse.
 */
zl_status zl_apply_left_inverse_rows(zl_plan plan, int y0, int y1, const void* x, void* partial, int R,
                                     void* stream);

/*
 * zl_scale_modes -- xt[r][k][j] = lambda_j^{-1/2} partial[r][k][j] (step V4's
 * Delta_b^{-1/2}), completing the sum of slab partials of
 * zl_apply_left_inverse_rows.  partial and xt: device [R][K][L]; they may be
 * the same buffer.
 */
zl_status zl_scale_modes(zl_plan plan, const void* partial, void* xt, int R, void* stream);

/*
 * zl_apply_left_inverse_host -- the same operator on HOST buffers: copies x to
 * the device, applies, copies x~ back, and synchronises `stream`.  x and xt
 * should be page-locked for the copies to be asynchronous.  The right-hand
 * sides go in pieces (about max_rhs / 4, at least 16): the copy-in of a piece
 * runs on an internal stream while the kernels of the previous piece run on
 * `stream` and the copy-back of the one before runs on a second internal
 * stream.  The copies start after the work already queued on `stream`.  When
 * the call returns, on success or error, nothing it queued is still running.
 * The device staging (two pieces of x and of x~), the two streams and the
 * events are owned by the plan and created on first use (this is the only
 * entry point that may allocate after setup).  Not safe to call concurrently
 * on one plan.
 */
zl_status zl_apply_left_inverse_host(zl_plan plan, const void* x, void* xt, int R, void* stream);

/*
 * zl_apply_sqrt -- x = Zh x~ = A V Delta^{1/2} x~ (Sec. 3.9):
 * y_k = V_b Delta_b^{1/2} x~_k, then x^(m) = A_m y^(m) per column.
 *   xt device [R][K][L] read only;  x device [R][nw][ny*nx] written.
 */
zl_status zl_apply_sqrt(zl_plan plan, const void* xt, void* x, int R, void* stream);

/*
 * zl_apply_adjoint -- g = (Zh^-)^T y = (A^+)^T V Delta^{-1/2} y, the transpose
 * of Eq. InverseSquareRootAlmost: v_k = V_b Delta_b^{-1/2} y_k, then
 * g^(m) = (A_m^+)^T v^(m) per column.  This is the gradient map of
 * J(x) = 1/2 ||Zh^- x||^2: grad J = zl_apply_adjoint(zl_apply_left_inverse(x)).
 *   y device [R][K][L] read only;  g device [R][nw][ny*nx] written.
 */
zl_status zl_apply_adjoint(zl_plan plan, const void* y, void* g, int R, void* stream);

/*
 * zl_apply_sqrt_adjoint -- t = Zh^T x = Delta^{1/2} V^T A^T x.
 *   x device [R][nw][ny*nx] read only;  t device [R][K][L] written.
 */
zl_status zl_apply_sqrt_adjoint(zl_plan plan, const void* x, void* t, int R, void* stream);

/*
 * zl_standardize_ensemble -- a forecast ensemble in standardized variables
 * (Sec. 2.1-2.2): row j of the output is Zh^- (e_j - mean) / sqrt(K_f - 1), the
 * standardized variables transform applied to forecast perturbation j, so that
 * P~^e = sum_j xt_j xt_j^T is the standardized ensemble covariance that the
 * Hybrid suggested in Sec. 2.2 localizes.
 *
 *   members  device, [K_f][nw][ny*nx]: the forecast members e_j (not centred),
 *            read only
 *   xt       device, [K_f][K][L], written; may not alias members
 *   Kf       number of forecast members, >= 2 (above max_rhs the left inverse
 *            runs in passes)
 *
 * Zh^- is linear: the members are mapped by the plan's left-inverse kernels and
 * the centring over members and the 1/sqrt(K_f - 1) scaling are applied to the
 * coefficients (mean accumulated in FP64).  Allocates nothing.
 * Errors: ZL_ERR_ARG (null pointers, aliasing, K_f < 2), and those of
 * zl_apply_left_inverse.
 */
zl_status zl_standardize_ensemble(zl_plan plan, const void* members, void* xt, int Kf, void* stream);

/*
 * Stage timing (profiling aid).  Each apply runs two kernel stages:
 *   ZL_STAGE_FWD_COLUMN  per-column product fused with the x-pass of V_b^T
 *                        (left inverse and Zh^T; the dominant kernel)
 *   ZL_STAGE_FWD_YPASS   y-pass of V_b^T, Delta scaling, compaction to [K][L]
 *   ZL_STAGE_INV_YPASS   scaling and y-pass of V_b (square root and adjoint)
 *   ZL_STAGE_INV_COLUMN  x-pass of V_b fused with the per-column product
 * While timing is enabled every stage launch is bracketed by two CUDA events
 * recorded on the launching stream (the events are created on demand).
 * zl_set_stage_timing(plan, 1) clears earlier records; (plan, 0) stops
 * recording and keeps them.  zl_get_stage_times waits for the recorded events
 * and returns the number of launches and their summed duration.
 */
typedef enum {
    ZL_STAGE_FWD_COLUMN = 0,
    ZL_STAGE_FWD_YPASS = 1,
    ZL_STAGE_INV_YPASS = 2,
    ZL_STAGE_INV_COLUMN = 3,
    ZL_NUM_STAGES = 4
} zl_stage;

zl_status zl_set_stage_timing(zl_plan plan, int enable);
zl_status zl_get_stage_times(zl_plan plan, int stage, int* launches, double* total_ms);

/*
 * zl_apply_left_inverse_static -- the same operator as zl_apply_left_inverse
 * (x [R][nw][ny*nx] -> x~ [R][K][L], device buffers, stream-ordered), for
 * callers that cannot allocate device memory when they apply it: a real-time
 * loop whose device memory budget is fixed at start-up, code running inside a
 * host callback where allocation calls are not allowed, or a process whose
 * device memory is owned by another framework's pool.  This call allocates
 * nothing.  The paper has no counterpart; it is a property of this library.
 *
 * It runs the CUDA-core kernels (for ZL_MIXED plans too, on the FP32
 * pseudo-inverse: FP32 accuracy) and keeps the intermediate of the separable
 * transform in a 16 MiB scratch array compiled into libzl.  Right-hand sides
 * are processed in passes of at most 16 MiB / (K * ny * Px * element size) of
 * them (and at most max_rhs); a plan for which even one right-hand side needs
 * more than 16 MiB (K * ny * Px * element size > 16 MiB, Px = kept
 * x-frequencies) is rejected with ZL_ERR_SHAPE before any work is queued.
 *
 * The array exists on a device once the driver has loaded libzl's module
 * holding it there.  zl_setup looks up the array's device address on the
 * plan's device (which loads that module, under lazy module loading too) and
 * loads every kernel this entry point launches, so from the first zl_setup on
 * a device the 16 MiB stay reserved there until the process exits, and this
 * call neither allocates nor loads anything: it only launches kernels.  If
 * the array cannot be created (device memory full), zl_setup returns
 * ZL_ERR_ALLOC.  Every call, on every stream, shares the one array, so calls
 * that overlap on the GPU race: serialise them (one stream, or events).
 * Nothing in the array needs clearing between calls: each pass overwrites the
 * part it reads.
 */
zl_status zl_apply_left_inverse_static(zl_plan plan, const void* x, void* xt, int R, void* stream);

/* ------------------------------------------------------------ diagnostics
 * The matrix-form and vector-form accuracy measures of the paper's experiment
 * (Sec. 4.7-4.9), computed on the GPU.  Meant for moderate sizes.
 */

/*
 * zl_column_svd -- the per-column singular value decomposition of Eq. svdOfAm
 * (Sec. 3.9), A_m = E_m Lambda_m F_m^T, for every grid column m of the plan's
 * ensemble copy (its storage precision), in FP64, by one-sided Jacobi
 * rotations (a warp per column).  g = min(nw, K) <= 64.
 *
 *   E    device, double [nh][nw][g]: E_m, orthonormal columns
 *   lam  device, double [nh][g]: the singular values, descending
 *   F    device, double [nh][K][g]: F_m, orthonormal columns
 *
 * Sign convention: in each singular triplet the entry of largest magnitude of
 * F_m's column is positive.  Stream-ordered; allocates nothing.  Errors:
 * ZL_ERR_ARG (null pointers, invalid plan), ZL_ERR_RANK (a rank-deficient
 * plan), ZL_ERR_SHAPE (g > 64), ZL_ERR_CUDA.
 */
zl_status zl_column_svd(zl_plan plan, double* E, double* lam, double* F, void* stream);

/*
 * zl_xi_indicators -- the matrix-form accuracy indicators of Sec. 4.8:
 * Xi = I - M M^T for M = Zh^- Zh (so that Zh^- Ph Zh^-^T = M M^T with
 * Ph = Zh Zh^T, Eq. MatrixDifferenceSwiftAlgorithm), reduced on the device to
 *   out[0] = sum_ij Xi_ij^2   (the paper's RMSE_Xi is its square root: a
 *                              Frobenius norm, no mean)
 *   out[1] = max_ij |Xi_ij|    (MAX_Xi)
 *   M    device, double [n][n] row-major (column j = Zh^- Zh e_j, built with
 *        the plan's own applies); n = K L.
 *   out  device, double[2]; overwritten (cleared on `stream` first).
 * FP64 CUDA-core tiles, O(n^3) work.  Errors: ZL_ERR_ARG, ZL_ERR_SHAPE
 * (n > 2^20), ZL_ERR_CUDA.
 */
zl_status zl_xi_indicators(const double* M, int n, double* out, void* stream);

/*
 * zl_delta -- the vector-form indicator of Sec. 4.9 (Eq. vectorDifferencedelta,
 * RMSEdelta): d = x~ - back and ||d_r||_2 per right-hand side, where the caller
 * formed back = Zh^- (Zh x~) with zl_apply_sqrt and zl_apply_left_inverse.
 *   xt, back  device, [R][K][L] in the plan's element type, read only
 *   d         device, [R][K][L], written (may alias xt or back)
 *   norms     device, double[R], written
 * Errors: ZL_ERR_ARG, ZL_ERR_CUDA.
 */
zl_status zl_delta(zl_plan plan, const void* xt, const void* back, void* d, double* norms, int R, void* stream);

/*
 * zl_plan_save / zl_plan_load -- checkpoint a plan and restore it without
 * redoing the setup's per-column factorisation (the paper has no counterpart).
 * The file holds the descriptor, the kept modes and their eigenvalues, the
 * rank status, the plan's copy of Z and the pseudo-inverse P (its storage
 * precision: 2 K n_w n_h elements, about 1 GB at 256x256x32, K = 64, FP32), in
 * the library's native layout (not portable across library versions or byte orders).
 * zl_plan_load validates the header (magic, sizes, ascending modes, positive
 * eigenvalues) and rejects any mismatch or short file with ZL_ERR_ARG before
 * touching the device; it then builds the tables and the tensor-core operands
 * from the stored P and returns a plan whose applies give the same bits as the
 * saved plan's (ZL_ERR_RANK with a valid plan when the saved plan was
 * rank-deficient).  Both synchronise: save reads the device buffers, load uses
 * `stream` and synchronises it.  Errors: ZL_ERR_ARG (null arguments, an
 * unreadable or unwritable file, a malformed header), ZL_ERR_ALLOC,
 * ZL_ERR_CUDA.
 */
zl_status zl_plan_save(zl_plan plan, const char* path);
zl_status zl_plan_load(const char* path, void* stream, zl_plan* out);

/* zl_destroy -- free a plan and everything it owns (NULL is a no-op).  The
 * caller must make sure no queued apply still uses it. */
zl_status zl_destroy(zl_plan plan);

/* zl_status_string -- static, human-readable name of a status code. */
const char* zl_status_string(zl_status s);

/*
 * zl_gaussian_spectrum -- host helper: eigenvalues, in packed order s =
 * p_y*nx + p_x, of the separable periodized Gaussian localization
 * c(d) = sum_p exp(-(d+pN)^2/(2 ell^2)) / sum_p exp(-(pN)^2/(2 ell^2)) per axis
 * (unit diagonal, as Sec. 2 and Sec. 4.4 require of a localization):
 * lambda(s) = lambda_x(f(p_x)) * lambda_y(f(p_y)),
 * lambda_axis(f) = sum_{d<N} c(d) cos(2 pi f d / N).
 *   out  host, double[nx*ny].
 */
zl_status zl_gaussian_spectrum(int nx, int ny, double ell, double* out);

/* ------------------------------------------------------------------ batches
 * Many independent instances (each its own grid, n_w, K, localization and
 * number of right-hand sides) applied together.  The paper's algorithm runs
 * on each instance unchanged (Sec. 3.10); the batch is a property of this
 * library.
 */
typedef struct zl_batch_s* zl_batch;   /* opaque; owned by libzl, freed by zl_destroy_batch */

/*
 * zl_setup_batch -- one plan per instance (exactly as zl_setup would build it
 * from descs[i], Z[i], spectra[i]; same layouts, precisions and errors), then
 * an autotuner picks each instance's kernel variant by timing, on the
 * instance's own shape with max_rhs right-hand sides, the variants that meet
 * the plan's accuracy: the tcgen05 path (ZL_MIXED plans it supports), the
 * register-tiled FP32 CUDA-core column kernel, and the per-column CUDA-core
 * kernel with 8, 4, 2 or 1 right-hand sides per CTA.  Choices are
 * cached per shape for the process and, if the environment variable
 * ZL_AUTOTUNE_CACHE names a file, appended to and read from that file.
 * Setup synchronises `stream` and allocates (per-plan memory plus temporary
 * tuning buffers of the largest instance).
 *
 *   n                number of instances, >= 1
 *   descs, Z, spectra  host arrays of n entries (Z[i]: device pointer)
 *   out              receives the batch; NULL on any error (every plan built
 *                    so far is destroyed)
 *   failed_instance  may be NULL; receives the index of the instance whose
 *                    setup failed, else -1
 */
zl_status zl_setup_batch(int n, const zl_desc* descs, const void* const* Z, const double* const* spectra,
                         void* stream, zl_batch* out, int* failed_instance);

/*
 * zl_batch_get_info -- the plan of instance i (owned by the batch: query it
 * with zl_get_info / zl_get_modes / zl_get_runtime_info, apply it alone with
 * the single-plan entry points, never zl_destroy it) and the autotuned variant
 * (0 = the default heuristic: tcgen05 for the ZL_MIXED plans it supports, else
 * the register-tiled FP32 column kernel where its tile fits; 1..4 = the
 * per-column CUDA-core kernel with 8, 4, 2, 1 right-hand sides per CTA; 5 = a
 * ZL_MIXED plan on the CUDA-core FP32 path with the default heuristic).  Either
 * output may be NULL.
 */
zl_status zl_batch_get_info(zl_batch batch, int i, zl_plan* plan, int* variant);

/*
 * zl_apply_left_inverse_batch -- x~_i = Zh_i^- x_i for every instance i.
 *
 *   x, xt   host arrays of n device pointers: x[i] [R[i]][nw_i][nh_i] (read),
 *           xt[i] [R[i]][K_i][L_i] (written); x[i] may not alias xt[i];
 *           entries with R[i] == 0 are skipped and may be NULL
 *   R       host array of n right-hand-side counts (>= 0; above max_rhs of an
 *           instance its apply runs in passes)
 *
 * The first call with a given (x, xt, R) captures the applies of all
 * instances into one CUDA graph (one concurrent branch per instance) and
 * later calls with the same buffers and counts replay it with one
 * cudaGraphLaunch on `stream`; the batch keeps the 4 most recently used
 * graphs.  Capturing allocates nothing on the device and does not
 * synchronise.  Calls on one batch must not overlap in host threads.
 * Errors: ZL_ERR_ARG (null arrays, R[i] < 0, a null or aliased pair with
 * R[i] > 0), ZL_ERR_RANK (some instance is rank-deficient), ZL_ERR_CUDA.
 */
zl_status zl_apply_left_inverse_batch(zl_batch batch, const void* const* x, void* const* xt, const int* R,
                                      void* stream);

/* zl_destroy_batch -- frees the batch, its plans and its graphs. */
zl_status zl_destroy_batch(zl_batch batch);

#ifdef __cplusplus
}
#endif
#endif /* ZL_H */
