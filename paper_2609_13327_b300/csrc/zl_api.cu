// libzl C ABI: plan lifecycle, argument checking, host-side tables, dispatch.

#include "zl_internal.cuh"

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdio>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <numeric>

namespace {

// ---------------------------------------------------------------------------
// packed real-Fourier basis (one axis of length N)
// ---------------------------------------------------------------------------
int packed_frequency(int N, int p) {
    if (p == 0) return 0;
    if (N % 2 == 0 && p == N - 1) return N / 2;
    return (p + 1) / 2;
}

// b_p(m); the argument 2 pi j m / N is reduced exactly in integers first.
double basis_value(int N, int p, int m) {
    if (p == 0) return 1.0 / std::sqrt((double)N);
    if (N % 2 == 0 && p == N - 1) return ((m & 1) ? -1.0 : 1.0) / std::sqrt((double)N);
    const int j = (p + 1) / 2;
    const long long r = ((long long)j * m) % N;
    const double a = 2.0 * M_PI * (double)r / (double)N;
    return std::sqrt(2.0 / N) * ((p & 1) ? std::cos(a) : std::sin(a));
}

// Eigenvalues of the periodized Gaussian c(d) (normalised to c(0) = 1) for every packed
// basis vector, by Poisson summation:
//   sum_t exp(-t^2 / (2 ell^2)) cos(2 pi f t / N) = sqrt(2 pi) ell sum_q exp(-2 pi^2 ell^2 (f/N - q)^2),
// a sum of positive terms, so the smallest eigenvalues keep full relative accuracy (a direct
// cosine sum over c(d) cancels to about 1e-16 of the largest, i.e. 1e-6..1e-5 relative at
// the mode threshold tau = 1e-10, and the left inverse scales those modes by lambda^{-1/2}).
std::vector<double> gaussian_axis_spectrum(int N, double ell) {
    std::vector<double> lam(N, 1.0);
    if (N == 1) return lam;
    const int P = (int)std::ceil(12.0 * ell / N) + 2;
    double den = 0.0;
    for (int p = -P; p <= P; ++p) {
        const double t = (double)p * N;
        den += std::exp(-t * t / (2.0 * ell * ell));
    }
    const int Q = (int)std::ceil(4.0 / std::max(ell, 1e-3)) + 3;
    for (int p = 0; p < N; ++p) {
        const double fr = (double)packed_frequency(N, p) / N;
        double sum = 0.0;
        for (int q = -Q; q <= Q; ++q) {
            const double u = fr - q;
            sum += std::exp(-2.0 * M_PI * M_PI * ell * ell * u * u);
        }
        lam[p] = std::sqrt(2.0 * M_PI) * ell * sum / den;
    }
    return lam;
}

template <typename T>
cudaError_t upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
    cudaError_t e = zl::dev_malloc((void**)dst, std::max<size_t>(1, src.size()) * sizeof(T));
    if (e != cudaSuccess) return e;
    if (src.empty()) return cudaSuccess;
    e = cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return cudaStreamSynchronize(s);   // src is a temporary host vector
}

template <typename T>
cudaError_t build_tables(zl_plan_s& p, zl::Tables<T>& t, const std::vector<double>& lamS,
                         const std::vector<int>& xfreq, cudaStream_t s) {
    const int nx = p.d.nx, ny = p.d.ny, L = p.L, Px = p.Px;
    std::vector<T> bx((size_t)Px * nx), by((size_t)ny * ny), isl(L), sl(L);
    for (int jx = 0; jx < Px; ++jx)
        for (int x = 0; x < nx; ++x) bx[(size_t)jx * nx + x] = (T)basis_value(nx, xfreq[jx], x);
    for (int q = 0; q < ny; ++q)
        for (int y = 0; y < ny; ++y) by[(size_t)q * ny + y] = (T)basis_value(ny, q, y);
    std::vector<int> py(L), jxv(L);
    std::vector<int> xslot(nx, -1);
    for (int jx = 0; jx < Px; ++jx) xslot[xfreq[jx]] = jx;
    for (int j = 0; j < L; ++j) {
        py[j] = p.modes[j] / nx;
        jxv[j] = xslot[p.modes[j] % nx];
        isl[j] = (T)(1.0 / std::sqrt(lamS[j]));
        sl[j] = (T)std::sqrt(lamS[j]);
    }
    // kept y-frequencies and the transposed table of their basis vectors
    std::vector<int> yslot(ny, -1), pylist;
    for (int j = 0; j < L; ++j) yslot[py[j]] = 1;
    for (int q = 0; q < ny; ++q)
        if (yslot[q] == 1) {
            yslot[q] = (int)pylist.size();
            pylist.push_back(q);
        }
    std::vector<int> ipy(L), yneed(Px, 0);
    for (int j = 0; j < L; ++j) {
        ipy[j] = yslot[py[j]];
        yneed[jxv[j]] = std::max(yneed[jxv[j]], ipy[j] + 1);
    }
    std::vector<T> byk((size_t)ny * p.pys, (T)0);
    for (int y = 0; y < ny; ++y)
        for (size_t i = 0; i < pylist.size(); ++i) byk[(size_t)y * p.pys + i] = (T)basis_value(ny, pylist[i], y);
    std::vector<int> gstart(Px + 1, 0), gmodes(L);
    for (int j = 0; j < L; ++j) gstart[jxv[j] + 1]++;
    for (int q = 0; q < Px; ++q) gstart[q + 1] += gstart[q];
    std::vector<int> fill(gstart.begin(), gstart.end() - 1);
    for (int j = 0; j < L; ++j) gmodes[fill[jxv[j]]++] = j;
    cudaError_t e;
    if ((e = upload(&t.bx, bx, s)) != cudaSuccess) return e;
    if ((e = upload(&t.by, by, s)) != cudaSuccess) return e;
    if ((e = upload(&t.inv_sqrt_lam, isl, s)) != cudaSuccess) return e;
    if ((e = upload(&t.sqrt_lam, sl, s)) != cudaSuccess) return e;
    if ((e = upload(&t.m_py, py, s)) != cudaSuccess) return e;
    if ((e = upload(&t.m_jx, jxv, s)) != cudaSuccess) return e;
    if ((e = upload(&t.grp_start, gstart, s)) != cudaSuccess) return e;
    if ((e = upload(&t.m_ipy, ipy, s)) != cudaSuccess) return e;
    if ((e = upload(&t.byk, byk, s)) != cudaSuccess) return e;
    if ((e = upload(&t.yneed, yneed, s)) != cudaSuccess) return e;
    return upload(&t.grp_modes, gmodes, s);
}

template <typename T>
void free_tables(zl::Tables<T>& t) {
    cudaFree(t.bx);
    cudaFree(t.by);
    cudaFree(t.inv_sqrt_lam);
    cudaFree(t.sqrt_lam);
    cudaFree(t.m_py);
    cudaFree(t.m_jx);
    cudaFree(t.grp_start);
    cudaFree(t.grp_modes);
    cudaFree(t.m_ipy);
    cudaFree(t.byk);
    cudaFree(t.yneed);
    t = zl::Tables<T>();
}

// Staging, streams and events of the host-buffer entry point (any subset may exist).
void release_host_staging(zl_plan_s* p) {
    cudaFree(p->h_x);
    cudaFree(p->h_xt);
    p->h_x = p->h_xt = nullptr;
    if (p->h_in) cudaStreamDestroy(p->h_in);
    if (p->h_out) cudaStreamDestroy(p->h_out);
    p->h_in = p->h_out = nullptr;
    for (cudaEvent_t* ev : {&p->h_start, &p->h_in_done[0], &p->h_in_done[1], &p->h_comp_done[0], &p->h_comp_done[1],
                            &p->h_out_done[0], &p->h_out_done[1]}) {
        if (*ev) cudaEventDestroy(*ev);
        *ev = nullptr;
    }
    p->h_piece = 0;
}

void free_plan(zl_plan_s* p) {
    if (!p) return;
    zl::tc_release(*p);
    cudaFree(p->Zc);
    cudaFree(p->P);
    cudaFree(p->t1);
    release_host_staging(p);
    cudaFree(p->d_status);
    cudaFree(p->d_werr);
    free_tables(p->td);
    free_tables(p->tf);
    delete p;
}

zl_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return ZL_OK;
    if (e == cudaErrorMemoryAllocation) return ZL_ERR_ALLOC;
    return ZL_ERR_CUDA;
}

bool valid_plan(zl_plan p) { return p != nullptr && p->P != nullptr; }

// Operator kinds for the shared forward / inverse passes.
enum class Op { LeftInverse, SqrtAdjoint, Sqrt, Adjoint };

// ZL_LOG (environment, read once): when set and not "0", every apply writes one JSON line
// to stderr with the operator, the sizes and the kernels it runs.
bool log_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("ZL_LOG");
        return v != nullptr && *v != '\0' && std::strcmp(v, "0") != 0;
    }();
    return on;
}

void log_call(const char* op, const zl_plan_s* p, int R, const char* column, const char* ypass) {
    if (!log_enabled()) return;
    static const char* const prec[] = {"fp64", "fp32", "mixed"};
    std::fprintf(stderr,
                 "{\"zl\": \"%s\", \"R\": %d, \"nx\": %d, \"ny\": %d, \"nw\": %d, \"K\": %d, \"L\": %d, "
                 "\"prec\": \"%s\", \"column\": \"%s\", \"ypass\": \"%s\"}\n",
                 op, R, p->d.nx, p->d.ny, p->d.nw, p->d.K, p->L, prec[(int)p->d.prec], column, ypass);
}

zl_status run(zl_plan p, Op op, const void* in, void* out, int R, void* stream) {
    if (!valid_plan(p) || (R > 0 && (in == nullptr || out == nullptr)) || R < 0) return ZL_ERR_ARG;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (R == 0) return ZL_OK;
    if (in == out) return ZL_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const long long n = (long long)p->d.nw * p->nh;
    const long long ns = (long long)p->d.K * p->L;
    const bool fwd = (op == Op::LeftInverse || op == Op::SqrtAdjoint);
    const long long in_len = fwd ? n : ns, out_len = fwd ? ns : n;
    if (log_enabled()) {
        static const char* const names[] = {"left_inverse", "sqrt_adjoint", "sqrt", "adjoint"};
        const bool tc = op == Op::LeftInverse && p->d.prec == ZL_MIXED && p->tc != nullptr && !p->force_plain;
        log_call(names[(int)op], p, R, tc ? "tcgen05" : "cuda-core", tc && p->ytc != nullptr ? "tcgen05" : "cuda-core");
    }
    const int chunk = p->d.max_rhs;
    for (int r0 = 0; r0 < R; r0 += chunk) {
        const int rc = std::min(chunk, R - r0);
        cudaError_t e;
        if (p->d.prec == ZL_FP64) {
            const double* x = (const double*)in + (long long)r0 * in_len;
            double* o = (double*)out + (long long)r0 * out_len;
            const double* M = (const double*)((op == Op::LeftInverse || op == Op::Adjoint) ? p->P : p->Zc);
            const double* sc = (op == Op::LeftInverse || op == Op::Adjoint) ? p->td.inv_sqrt_lam : p->td.sqrt_lam;
            e = fwd ? zl::forward_plain<double>(*p, p->td, M, sc, x, o, rc, s, zl::Rows{0, p->d.ny})
                    : zl::inverse_plain<double>(*p, p->td, M, sc, x, o, rc, s);
        } else {
            const float* x = (const float*)in + (long long)r0 * in_len;
            float* o = (float*)out + (long long)r0 * out_len;
            if (op == Op::LeftInverse && p->d.prec == ZL_MIXED && p->tc != nullptr && !p->force_plain) {
                e = zl::forward_tc(*p, x, o, rc, s, zl::Rows{0, p->d.ny}, p->tf.inv_sqrt_lam);
            } else {
                const float* M = (const float*)((op == Op::LeftInverse || op == Op::Adjoint) ? p->P : p->Zc);
                const float* sc = (op == Op::LeftInverse || op == Op::Adjoint) ? p->tf.inv_sqrt_lam : p->tf.sqrt_lam;
                e = fwd ? zl::forward_plain<float>(*p, p->tf, M, sc, x, o, rc, s, zl::Rows{0, p->d.ny})
                        : zl::inverse_plain<float>(*p, p->tf, M, sc, x, o, rc, s);
            }
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    return ZL_OK;
}

}  // namespace

namespace zl {

namespace {
std::atomic<int> g_alloc_fail_in{0};   // 0: off; n > 0: the n-th allocation from now fails
}

cudaError_t dev_malloc(void** ptr, size_t bytes) {
    int n = g_alloc_fail_in.load();
    while (n > 0) {
        if (g_alloc_fail_in.compare_exchange_weak(n, n - 1)) {
            if (n == 1) {
                *ptr = nullptr;
                return cudaErrorMemoryAllocation;
            }
            break;
        }
    }
    return cudaMalloc(ptr, bytes);
}

cudaEvent_t StageTimer::take() {
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void StageTimer::begin(int stage, cudaStream_t s) {
    if (!on) return;
    Rec r{stage, take(), take()};
    if (r.a == nullptr || r.b == nullptr) return;
    cudaEventRecord(r.a, s);
    recs.push_back(r);
}

void StageTimer::end(cudaStream_t s) {
    if (!on || recs.empty()) return;
    cudaEventRecord(recs.back().b, s);
}

void StageTimer::clear() {
    for (auto& r : recs) {
        cudaEventSynchronize(r.b);
        pool.push_back(r.a);
        pool.push_back(r.b);
    }
    recs.clear();
}

StageTimer::~StageTimer() {
    clear();
    for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

}  // namespace zl

extern "C" {

zl_status zl_set_test_alloc_failure(int n) {
    if (n < 0) return ZL_ERR_ARG;
    zl::g_alloc_fail_in.store(n);
    return ZL_OK;
}

zl_status zl_set_stage_timing(zl_plan p, int enable) {
    if (!valid_plan(p)) return ZL_ERR_ARG;
    if (enable) p->timer.clear();
    p->timer.on = enable != 0;
    return ZL_OK;
}

zl_status zl_get_stage_times(zl_plan p, int stage, int* launches, double* total_ms) {
    if (!valid_plan(p) || stage < 0 || stage >= ZL_NUM_STAGES || launches == nullptr || total_ms == nullptr)
        return ZL_ERR_ARG;
    int n = 0;
    double ms = 0.0;
    for (auto& r : p->timer.recs) {
        if (r.stage != stage) continue;
        if (cudaEventSynchronize(r.b) != cudaSuccess) return ZL_ERR_CUDA;
        float t = 0.f;
        if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) return ZL_ERR_CUDA;
        ms += t;
        ++n;
    }
    *launches = n;
    *total_ms = ms;
    return ZL_OK;
}


const char* zl_status_string(zl_status s) {
    switch (s) {
        case ZL_OK: return "ZL_OK";
        case ZL_ERR_ARG: return "ZL_ERR_ARG: invalid argument";
        case ZL_ERR_SHAPE: return "ZL_ERR_SHAPE: size outside the supported range";
        case ZL_ERR_RANK: return "ZL_ERR_RANK: a column matrix A_m is rank-deficient";
        case ZL_ERR_ALLOC: return "ZL_ERR_ALLOC: device allocation failed";
        case ZL_ERR_CUDA: return "ZL_ERR_CUDA: CUDA runtime error";
        case ZL_ERR_TIMEOUT: return "ZL_ERR_TIMEOUT: a bounded device wait gave up";
        case ZL_ERR_UNSUPPORTED: return "ZL_ERR_UNSUPPORTED: not implemented for this configuration";
    }
    return "unknown zl_status";
}

zl_status zl_gaussian_spectrum(int nx, int ny, double ell, double* out) {
    if (out == nullptr || !(ell > 0.0) || !std::isfinite(ell)) return ZL_ERR_ARG;
    if (nx < 1 || ny < 1 || (long long)nx * ny > (1LL << 30)) return ZL_ERR_SHAPE;
    const std::vector<double> lx = gaussian_axis_spectrum(nx, ell), ly = gaussian_axis_spectrum(ny, ell);
    for (int q = 0; q < ny; ++q)
        for (int p = 0; p < nx; ++p) out[(size_t)q * nx + p] = ly[q] * lx[p];
    return ZL_OK;
}

}  // extern "C"

namespace {

zl_status validate_desc(const zl_desc& d) {
    if (d.prec != ZL_FP64 && d.prec != ZL_FP32 && d.prec != ZL_MIXED) return ZL_ERR_ARG;
    if (!(d.tau >= 0.0) || !std::isfinite(d.tau)) return ZL_ERR_ARG;
    if (d.nx < 1 || d.ny < 1 || d.nw < 1 || d.K < 1 || d.max_rhs < 1 || d.max_rhs > 65535) return ZL_ERR_SHAPE;
    if (d.nx > 65535 || d.ny > 65535) return ZL_ERR_SHAPE;
    const long long nh = (long long)d.nx * d.ny;
    if (nh > (1LL << 30) || (long long)d.nw * d.K > 16384) return ZL_ERR_SHAPE;
    if (zl::setup_smem_bytes(d.nw, d.K) > 200 * 1024) return ZL_ERR_SHAPE;
    return ZL_OK;
}

// The host part of a plan from its kept modes (ascending packed indices) and their
// eigenvalues: sizes, kept x- and y-frequencies, shape limits.  No device work.
zl_status make_plan(const zl_desc& d, std::vector<int> modes, std::vector<double> lamS, zl_plan_s** out) {
    *out = nullptr;
    if (modes.empty()) return ZL_ERR_SHAPE;   // tau >= 1: no eigenvalue exceeds tau * max, nothing to apply
    zl_plan_s* p = new (std::nothrow) zl_plan_s();
    if (!p) return ZL_ERR_ALLOC;
    p->d = d;
    p->nh = (long long)d.nx * d.ny;
    p->g = std::min(d.nw, d.K);
    p->esize = d.prec == ZL_FP64 ? sizeof(double) : sizeof(float);
    p->modes = std::move(modes);
    p->lamS = std::move(lamS);
    p->L = (int)p->modes.size();
    std::vector<char> used(d.nx, 0);
    for (int s : p->modes) used[s % d.nx] = 1;
    for (int q = 0; q < d.nx; ++q)
        if (used[q]) p->xfreq.push_back(q);
    p->Px = (int)p->xfreq.size();
    std::vector<char> yused(d.ny, 0);
    for (int s2 : p->modes) yused[s2 / d.nx] = 1;
    p->Py = 0;
    for (char c : yused) p->Py += c;
    p->pys = (p->Py + 15) / 16 * 16;
    // forward y-pass keeps the L accumulators in shared memory
    if ((size_t)p->L * p->esize + (size_t)p->Px * p->esize > 96 * 1024 ||
        (size_t)d.K * (p->Px + 32) * p->esize > 160 * 1024) {
        delete p;
        return ZL_ERR_SHAPE;
    }
    *out = p;
    return ZL_OK;
}

// The device part: the plan's copy of Z (from the caller's device buffer, or a host
// buffer), the tables, the pseudo-inverse P (formed by the setup kernel, or copied from a
// host buffer of a saved plan, with its recorded rank status), the tensor-core operands
// and the allocation-free entry point's preparation.  Frees the plan on any error except
// ZL_ERR_RANK.
zl_status finish_plan(zl_plan_s* p, const void* Z, bool Z_on_host, const void* P_host, int bad_column,
                      cudaStream_t s, zl_plan* out) {
    const zl_desc& d = p->d;
    if (cudaGetDevice(&p->device) != cudaSuccess) {
        delete p;
        return ZL_ERR_CUDA;
    }
    const size_t mbytes = (size_t)d.K * d.nw * p->nh * p->esize;
    const size_t tbytes = (size_t)d.max_rhs * d.K * d.ny * p->Px * p->esize;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->Zc, mbytes);
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->P, mbytes);
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->t1, std::max<size_t>(tbytes, 16));
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->d_status, sizeof(int));
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->d_werr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->d_werr, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(p->Zc, Z, mbytes, Z_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        static const int kNone = INT_MAX;
        e = cudaMemcpyAsync(p->d_status, &kNone, sizeof(int), cudaMemcpyHostToDevice, s);
    }
    if (e == cudaSuccess) {
        e = d.prec == ZL_FP64 ? build_tables<double>(*p, p->td, p->lamS, p->xfreq, s)
                              : build_tables<float>(*p, p->tf, p->lamS, p->xfreq, s);
    }
    int status = INT_MAX;
    if (P_host == nullptr) {
        if (e == cudaSuccess) e = zl::launch_setup_columns(d, p->nh, Z_on_host ? p->Zc : Z, p->P, p->d_status, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost, s);
    } else {
        if (e == cudaSuccess) e = cudaMemcpyAsync(p->P, P_host, mbytes, cudaMemcpyHostToDevice, s);
        if (bad_column >= 0) status = bad_column;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        free_plan(p);
        return cuda_status(e);
    }
    if (status != INT_MAX) {
        p->bad_column = status;
        *out = p;
        return ZL_ERR_RANK;
    }
    if (d.prec == ZL_MIXED) {
        const zl_status ts = zl::tc_prepare(*p, s);
        if (ts != ZL_OK && ts != ZL_ERR_UNSUPPORTED) {
            free_plan(p);
            return ts;
        }
    }
    // the allocation-free entry point: its scratch array's address on this device (which
    // loads the module that holds the array) and the kernels it launches, so that it loads
    // and allocates nothing itself
    const zl_status ss = zl::static_scratch_prepare(*p);
    if (ss != ZL_OK) {
        free_plan(p);
        return ss;
    }
    *out = p;
    return ZL_OK;
}

constexpr char kPlanMagic[8] = {'Z', 'L', 'P', 'L', 'A', 'N', '1', '\0'};

}  // namespace

extern "C" {

zl_status zl_setup(const zl_desc* desc, const void* Z, const double* spectrum, void* stream, zl_plan* out) {
    if (out == nullptr) return ZL_ERR_ARG;
    *out = nullptr;
    if (desc == nullptr || Z == nullptr || spectrum == nullptr) return ZL_ERR_ARG;
    const zl_desc d = *desc;
    const zl_status vs = validate_desc(d);
    if (vs != ZL_OK) return vs;
    const long long nh = (long long)d.nx * d.ny;
    double lmax = -INFINITY;
    for (long long s = 0; s < nh; ++s) {
        if (!std::isfinite(spectrum[s])) return ZL_ERR_ARG;
        lmax = std::max(lmax, spectrum[s]);
    }
    if (!(lmax > 0.0)) return ZL_ERR_ARG;
    std::vector<int> modes;
    std::vector<double> lamS;
    for (long long s = 0; s < nh; ++s)
        if (spectrum[s] > d.tau * lmax) {
            modes.push_back((int)s);
            lamS.push_back(spectrum[s]);
        }
    zl_plan_s* p = nullptr;
    const zl_status ms = make_plan(d, std::move(modes), std::move(lamS), &p);
    if (ms != ZL_OK) return ms;
    return finish_plan(p, Z, false, nullptr, -1, (cudaStream_t)stream, out);
}

zl_status zl_plan_save(zl_plan p, const char* path) {
    if (p == nullptr || p->P == nullptr || path == nullptr) return ZL_ERR_ARG;
    const size_t mbytes = (size_t)p->d.K * p->d.nw * p->nh * p->esize;
    std::vector<char> zc(mbytes), pc(mbytes);
    if (cudaMemcpy(zc.data(), p->Zc, mbytes, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(pc.data(), p->P, mbytes, cudaMemcpyDeviceToHost) != cudaSuccess)
        return ZL_ERR_CUDA;
    FILE* f = std::fopen(path, "wb");
    if (f == nullptr) return ZL_ERR_ARG;
    const int32_t L = p->L, bad = p->bad_column;
    const uint64_t mb = mbytes;
    bool ok = std::fwrite(kPlanMagic, 1, sizeof(kPlanMagic), f) == sizeof(kPlanMagic) &&
              std::fwrite(&p->d, sizeof(zl_desc), 1, f) == 1 && std::fwrite(&L, sizeof(L), 1, f) == 1 &&
              std::fwrite(&bad, sizeof(bad), 1, f) == 1 && std::fwrite(&mb, sizeof(mb), 1, f) == 1 &&
              std::fwrite(p->modes.data(), sizeof(int), (size_t)L, f) == (size_t)L &&
              std::fwrite(p->lamS.data(), sizeof(double), (size_t)L, f) == (size_t)L &&
              std::fwrite(zc.data(), 1, mbytes, f) == mbytes && std::fwrite(pc.data(), 1, mbytes, f) == mbytes;
    ok = (std::fclose(f) == 0) && ok;
    return ok ? ZL_OK : ZL_ERR_ARG;
}

zl_status zl_plan_load(const char* path, void* stream, zl_plan* out) {
    if (out == nullptr) return ZL_ERR_ARG;
    *out = nullptr;
    if (path == nullptr) return ZL_ERR_ARG;
    FILE* f = std::fopen(path, "rb");
    if (f == nullptr) return ZL_ERR_ARG;
    char magic[sizeof(kPlanMagic)];
    zl_desc d;
    int32_t L = 0, bad = -1;
    uint64_t mb = 0;
    bool ok = std::fread(magic, 1, sizeof(magic), f) == sizeof(magic) &&
              std::memcmp(magic, kPlanMagic, sizeof(magic)) == 0 && std::fread(&d, sizeof(d), 1, f) == 1 &&
              std::fread(&L, sizeof(L), 1, f) == 1 && std::fread(&bad, sizeof(bad), 1, f) == 1 &&
              std::fread(&mb, sizeof(mb), 1, f) == 1;
    ok = ok && validate_desc(d) == ZL_OK;
    const long long nh = ok ? (long long)d.nx * d.ny : 0;
    const size_t esize = d.prec == ZL_FP64 ? sizeof(double) : sizeof(float);
    ok = ok && L >= 1 && L <= nh && mb == (uint64_t)d.K * d.nw * nh * esize && bad >= -1 && bad < nh;
    std::vector<int> modes;
    std::vector<double> lamS;
    std::vector<char> zc, pc;
    if (ok) {
        modes.resize(L);
        lamS.resize(L);
        ok = std::fread(modes.data(), sizeof(int), (size_t)L, f) == (size_t)L &&
             std::fread(lamS.data(), sizeof(double), (size_t)L, f) == (size_t)L;
    }
    for (int i = 0; ok && i < L; ++i)   // ascending mode indices inside the grid, positive eigenvalues
        ok = modes[i] >= 0 && modes[i] < nh && (i == 0 || modes[i] > modes[i - 1]) && lamS[i] > 0.0 &&
             std::isfinite(lamS[i]);
    if (ok) {
        zc.resize(mb);
        pc.resize(mb);
        ok = std::fread(zc.data(), 1, mb, f) == mb && std::fread(pc.data(), 1, mb, f) == mb;
    }
    std::fclose(f);
    if (!ok) return ZL_ERR_ARG;
    zl_plan_s* p = nullptr;
    const zl_status ms = make_plan(d, std::move(modes), std::move(lamS), &p);
    if (ms != ZL_OK) return ms;
    return finish_plan(p, zc.data(), true, pc.data(), bad, (cudaStream_t)stream, out);
}

zl_status zl_get_desc(zl_plan p, zl_desc* desc) {
    if (!valid_plan(p) || desc == nullptr) return ZL_ERR_ARG;
    *desc = p->d;
    return ZL_OK;
}

zl_status zl_get_info(zl_plan p, int* L, int* nw, int* K, long long* nh, int* bad_column) {
    if (!valid_plan(p)) return ZL_ERR_ARG;
    if (L) *L = p->L;
    if (nw) *nw = p->d.nw;
    if (K) *K = p->d.K;
    if (nh) *nh = p->nh;
    if (bad_column) *bad_column = p->bad_column;
    return ZL_OK;
}

zl_status zl_get_runtime_info(zl_plan p, int* tensor_core_path, int* device_error) {
    if (!valid_plan(p)) return ZL_ERR_ARG;
    if (tensor_core_path) *tensor_core_path = (p->tc != nullptr && !p->force_plain) ? 1 : 0;
    if (device_error) {
        int code = 0;
        if (zl::tc_read_error(*p, &code) != cudaSuccess) return ZL_ERR_CUDA;
        *device_error = code;
        if (code != 0) return ZL_ERR_TIMEOUT;
    }
    return ZL_OK;
}

zl_status zl_set_test_wait_timeout(zl_plan p, int enable) {
    if (!valid_plan(p) || (enable != 0 && enable != 1)) return ZL_ERR_ARG;
    if (p->tc == nullptr && !(p->d.prec != ZL_FP64 && zl::f32_column_supported(*p, p->d.max_rhs)))
        return ZL_ERR_UNSUPPORTED;
    if (cudaDeviceSynchronize() != cudaSuccess) return ZL_ERR_CUDA;
    p->test_wait_timeout = enable;
    if (!enable && zl::tc_clear_error(*p) != cudaSuccess) return ZL_ERR_CUDA;
    return ZL_OK;
}

zl_status zl_get_modes(zl_plan p, int* modes) {
    if (!valid_plan(p) || modes == nullptr) return ZL_ERR_ARG;
    std::copy(p->modes.begin(), p->modes.end(), modes);
    return ZL_OK;
}

zl_status zl_apply_left_inverse(zl_plan p, const void* x, void* xt, int R, void* stream) {
    return run(p, Op::LeftInverse, x, xt, R, stream);
}

zl_status zl_apply_sqrt_adjoint(zl_plan p, const void* x, void* t, int R, void* stream) {
    return run(p, Op::SqrtAdjoint, x, t, R, stream);
}

zl_status zl_apply_sqrt(zl_plan p, const void* xt, void* x, int R, void* stream) {
    return run(p, Op::Sqrt, xt, x, R, stream);
}

zl_status zl_apply_adjoint(zl_plan p, const void* y, void* g, int R, void* stream) {
    return run(p, Op::Adjoint, y, g, R, stream);
}

// Right-hand sides per piece of the host-buffer entry point: about a quarter of max_rhs,
// in multiples of the tensor-core kernel's 16-rhs unit, at least 16 and at most max_rhs.
static int host_piece(int max_rhs) {
    const int q = ((max_rhs + 3) / 4 + 15) / 16 * 16;
    return std::min(max_rhs, std::max(16, q));
}

static cudaError_t host_staging(zl_plan_s* p, size_t in_b, size_t out_b) {
    if (p->h_x != nullptr) return cudaSuccess;
    const int piece = host_piece(p->d.max_rhs);
    cudaError_t e = zl::dev_malloc((void**)&p->h_x, 2 * piece * in_b);
    if (e == cudaSuccess) e = zl::dev_malloc((void**)&p->h_xt, 2 * piece * out_b);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->h_in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->h_out, cudaStreamNonBlocking);
    for (cudaEvent_t* ev : {&p->h_start, &p->h_in_done[0], &p->h_in_done[1], &p->h_comp_done[0], &p->h_comp_done[1],
                            &p->h_out_done[0], &p->h_out_done[1]})
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        release_host_staging(p);
        return e;
    }
    p->h_piece = piece;
    return cudaSuccess;
}

zl_status zl_apply_left_inverse_host(zl_plan p, const void* x, void* xt, int R, void* stream) {
    if (!valid_plan(p) || R < 0 || (R > 0 && (x == nullptr || xt == nullptr))) return ZL_ERR_ARG;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (R == 0) return ZL_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t in_b = (size_t)p->d.nw * p->nh * p->esize, out_b = (size_t)p->d.K * p->L * p->esize;
    cudaError_t e = host_staging(p, in_b, out_b);
    if (e != cudaSuccess) return cuda_status(e);
    const int piece = p->h_piece;
    // Piece i uses staging slot i % 2: its copy-in (h_in) overlaps the kernels of piece i - 1
    // (on `stream`) and the copy-out of piece i - 2 (h_out).  The copies of a call start after
    // the work queued on `stream` before it.
    zl_status st = ZL_OK;
    e = cudaEventRecord(p->h_start, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h_in, p->h_start, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h_out, p->h_start, 0);
    for (int r0 = 0, i = 0; r0 < R && e == cudaSuccess && st == ZL_OK; r0 += piece, ++i) {
        const int rc = std::min(piece, R - r0), b = i & 1;
        char* dx = (char*)p->h_x + (size_t)b * piece * in_b;
        char* dxt = (char*)p->h_xt + (size_t)b * piece * out_b;
        // slot b of x was last read by the kernels of piece i - 2, slot b of x~ last copied out
        // by piece i - 2
        if (i >= 2) e = cudaStreamWaitEvent(p->h_in, p->h_comp_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dx, (const char*)x + (size_t)r0 * in_b, rc * in_b, cudaMemcpyHostToDevice, p->h_in);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_in_done[b], p->h_in);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, p->h_in_done[b], 0);
        if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(s, p->h_out_done[b], 0);
        if (e != cudaSuccess) break;
        st = run(p, Op::LeftInverse, dx, dxt, rc, stream);
        if (st != ZL_OK) break;
        e = cudaEventRecord(p->h_comp_done[b], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(p->h_out, p->h_comp_done[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((char*)xt + (size_t)r0 * out_b, dxt, rc * out_b, cudaMemcpyDeviceToHost, p->h_out);
        if (e == cudaSuccess) e = cudaEventRecord(p->h_out_done[b], p->h_out);
    }
    // on every path, nothing queued by this call is still running when it returns
    const cudaError_t e_in = cudaStreamSynchronize(p->h_in);
    const cudaError_t e_s = cudaStreamSynchronize(s);
    const cudaError_t e_out = cudaStreamSynchronize(p->h_out);
    if (st != ZL_OK) return st;
    if (e != cudaSuccess) return cuda_status(e);
    if (e_in != cudaSuccess) return cuda_status(e_in);
    if (e_s != cudaSuccess) return cuda_status(e_s);
    return cuda_status(e_out);
}

zl_status zl_apply_left_inverse_rows(zl_plan p, int y0, int y1, const void* x, void* partial, int R, void* stream) {
    if (!valid_plan(p) || R < 0 || (R > 0 && (x == nullptr || partial == nullptr))) return ZL_ERR_ARG;
    if (y0 < 0 || y1 <= y0 || y1 > p->d.ny) return ZL_ERR_SHAPE;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (R == 0) return ZL_OK;
    if (x == partial) return ZL_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const zl::Rows rows{y0, y1 - y0};
    const long long in_len = (long long)p->d.nw * rows.ny * p->d.nx, out_len = (long long)p->d.K * p->L;
    for (int r0 = 0; r0 < R; r0 += p->d.max_rhs) {
        const int rc = std::min(p->d.max_rhs, R - r0);
        cudaError_t e;
        if (p->d.prec == ZL_FP64) {
            e = zl::forward_plain<double>(*p, p->td, (const double*)p->P, nullptr, (const double*)x + r0 * in_len,
                                          (double*)partial + r0 * out_len, rc, s, rows);
        } else if (p->d.prec == ZL_MIXED && p->tc != nullptr && !p->force_plain) {
            e = zl::forward_tc(*p, (const float*)x + r0 * in_len, (float*)partial + r0 * out_len, rc, s, rows, nullptr);
        } else {
            e = zl::forward_plain<float>(*p, p->tf, (const float*)p->P, nullptr, (const float*)x + r0 * in_len,
                                         (float*)partial + r0 * out_len, rc, s, rows);
        }
        if (e != cudaSuccess) return cuda_status(e);
    }
    return ZL_OK;
}

zl_status zl_scale_modes(zl_plan p, const void* partial, void* xt, int R, void* stream) {
    if (!valid_plan(p) || R < 0 || (R > 0 && (partial == nullptr || xt == nullptr))) return ZL_ERR_ARG;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (R == 0) return ZL_OK;
    const cudaError_t e = p->d.prec == ZL_FP64
        ? zl::launch_scale_modes<double>((const double*)partial, p->td.inv_sqrt_lam, (double*)xt,
                                         (long long)R * p->d.K, p->L, (cudaStream_t)stream)
        : zl::launch_scale_modes<float>((const float*)partial, p->tf.inv_sqrt_lam, (float*)xt,
                                        (long long)R * p->d.K, p->L, (cudaStream_t)stream);
    return cuda_status(e);
}

zl_status zl_column_svd(zl_plan p, double* E, double* lam, double* F, void* stream) {
    if (!valid_plan(p) || E == nullptr || lam == nullptr || F == nullptr) return ZL_ERR_ARG;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (p->g > 64 || zl::column_svd_smem_per_warp(p->d.nw, p->d.K) > 200 * 1024) return ZL_ERR_SHAPE;
    return cuda_status(zl::launch_column_svd(*p, E, lam, F, (cudaStream_t)stream));
}

zl_status zl_xi_indicators(const double* M, int n, double* out, void* stream) {
    if (M == nullptr || out == nullptr || n < 1) return ZL_ERR_ARG;
    if (n > (1 << 20)) return ZL_ERR_SHAPE;
    return cuda_status(zl::launch_xi(M, n, out, (cudaStream_t)stream));
}

zl_status zl_delta(zl_plan p, const void* xt, const void* back, void* d, double* norms, int R, void* stream) {
    if (!valid_plan(p) || R < 0 || (R > 0 && (xt == nullptr || back == nullptr || d == nullptr || norms == nullptr)))
        return ZL_ERR_ARG;
    if (R == 0) return ZL_OK;
    const long long len = (long long)p->d.K * p->L;
    cudaStream_t s = (cudaStream_t)stream;
    const cudaError_t e = p->d.prec == ZL_FP64
        ? zl::launch_delta<double>((const double*)xt, (const double*)back, (double*)d, norms, len, R, s)
        : zl::launch_delta<float>((const float*)xt, (const float*)back, (float*)d, norms, len, R, s);
    return cuda_status(e);
}

zl_status zl_destroy(zl_plan p) {
    if (p == nullptr) return ZL_OK;
    free_plan(p);
    return ZL_OK;
}

}  // extern "C"
