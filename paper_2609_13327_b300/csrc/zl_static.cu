// zl_apply_left_inverse_static: the left inverse on the CUDA-core kernels with its
// scratch in a fixed device array compiled into the library, for callers that
// must not allocate device memory when they apply the operator.
//
// The scratch holds the intermediate of the separable transform (the x-pass
// output, R * K * ny * Px elements per pass).  It is a file-scope device array
// of kStaticScratchBytes.  Host code cannot use the array's name as a device
// address: zl_setup looks the address up with cudaGetSymbolAddress on the
// plan's device (that device current), which also makes the driver load the
// module holding the array there (under lazy module loading, the array takes
// device memory from that moment until the process exits).  zl_setup also
// loads every kernel this entry point may launch, so the entry point itself
// loads and allocates nothing: it only launches kernels.

#include "zl_internal.cuh"

#include <algorithm>
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = size_t(16) << 20;   // 16 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

namespace zl {

zl_status static_scratch_prepare(const zl_plan_s& p) {
    if (p.device < 0 || p.device >= kMaxDevices) return ZL_ERR_UNSUPPORTED;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (g_scratch_addr[p.device] == nullptr) {
            void* a = nullptr;
            const cudaError_t e = cudaGetSymbolAddress(&a, g_static_scratch);
            if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ZL_ERR_ALLOC : ZL_ERR_CUDA;
            g_scratch_addr[p.device] = a;
        }
    }
    const cudaError_t e = p.d.prec == ZL_FP64 ? preload_forward_plain<double>() : preload_forward_plain<float>();
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ZL_ERR_ALLOC : ZL_ERR_CUDA;
    return ZL_OK;
}

}  // namespace zl

extern "C" zl_status zl_apply_left_inverse_static(zl_plan p, const void* x, void* xt, int R, void* stream) {
    if (p == nullptr || p->P == nullptr || R < 0 || (R > 0 && (x == nullptr || xt == nullptr))) return ZL_ERR_ARG;
    if (p->bad_column >= 0) return ZL_ERR_RANK;
    if (R == 0) return ZL_OK;
    if (x == xt) return ZL_ERR_ARG;
    // every element of the scratch is written by the x-pass before the y-pass reads it: nothing to clear
    const size_t per_rhs = (size_t)p->d.K * p->d.ny * p->Px * p->esize;
    if (per_rhs == 0 || per_rhs > kStaticScratchBytes) return ZL_ERR_SHAPE;
    const int chunk = (int)std::min<size_t>({kStaticScratchBytes / per_rhs, (size_t)p->d.max_rhs, (size_t)65535});
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        if (p->device >= 0 && p->device < kMaxDevices) scratch = g_scratch_addr[p->device];
    }
    if (scratch == nullptr) return ZL_ERR_CUDA;   // zl_setup resolves it for every plan it returns
    cudaStream_t s = (cudaStream_t)stream;
    const long long in_len = (long long)p->d.nw * p->nh, out_len = (long long)p->d.K * p->L;
    for (int r0 = 0; r0 < R; r0 += chunk) {
        const int rc = std::min(chunk, R - r0);
        cudaError_t e;
        if (p->d.prec == ZL_FP64) {
            e = zl::forward_plain_on<double>(*p, p->td, (const double*)p->P, p->td.inv_sqrt_lam,
                                             (const double*)x + r0 * in_len, (double*)xt + r0 * out_len, rc, s,
                                             (double*)scratch);
        } else {
            e = zl::forward_plain_on<float>(*p, p->tf, (const float*)p->P, p->tf.inv_sqrt_lam,
                                            (const float*)x + r0 * in_len, (float*)xt + r0 * out_len, rc, s,
                                            (float*)scratch);
        }
        if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? ZL_ERR_ALLOC : ZL_ERR_CUDA;
    }
    return ZL_OK;
}
