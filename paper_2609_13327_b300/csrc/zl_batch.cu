// Batched left inverse over many independent instances with uneven grids,
// level counts, ensemble sizes and right-hand-side counts (the paper's
// algorithm applies to each instance unchanged, Sec. 3.10; the instances share
// nothing).
//
// The batch owns one plan per instance.  An apply with a given set of buffers
// is captured once into a CUDA graph whose branches are the instances (each on
// its own capture stream, forked from and joined back into one origin), so that
// the small instances run concurrently and fill the GPU, and every later apply
// with the same buffers is a single cudaGraphLaunch.  At setup an autotuner
// times, per instance, the kernel variants that meet the plan's accuracy (the
// tcgen05 path and the CUDA-core path with 8, 4, 2 or 1 right-hand sides per
// CTA) on the instance's own shape and keeps the fastest; choices are cached
// per shape in the process and, when ZL_AUTOTUNE_CACHE names a file, across
// processes.

#include "zl_internal.cuh"

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

struct zl_batch_s {
    std::vector<zl_plan> plans;
    std::vector<int> choice;            // autotuned variant per instance (see apply_variant)
    cudaStream_t origin = nullptr;      // capture origin
    std::vector<cudaStream_t> branch;   // capture branches, one per instance
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    struct Graph {
        std::vector<const void*> x;
        std::vector<void*> xt;
        std::vector<int> R;
        cudaGraphExec_t exec = nullptr;
        unsigned long long last_use = 0;
    };
    std::vector<Graph> graphs;          // a few captured applies, least recently used replaced
    unsigned long long uses = 0;
};

namespace {

constexpr int kMaxGraphs = 4;
constexpr int kTuneReps = 3;

// variant v: 0 = default heuristics (tcgen05 for supported mixed plans, else the
// register-tiled FP32 column kernel where its tile fits), 1..4 = CUDA-core path with 8, 4,
// 2, 1 right-hand sides per CTA of the per-column kernel, 5 = CUDA-core path with the
// default heuristics (for a mixed plan: the register-tiled FP32 kernel instead of tcgen05)
constexpr int kVariants = 6;
const int kRcOf[kVariants] = {0, 8, 4, 2, 1, 0};

void apply_variant(zl_plan p, int v) {
    p->force_plain = v != 0;
    p->force_rc = kRcOf[v];
}

std::string shape_key(const zl_plan_s& p) {
    char b[160];
    std::snprintf(b, sizeof(b), "nx=%d ny=%d nw=%d K=%d L=%d Px=%d prec=%d rhs=%d tc=%d", p.d.nx, p.d.ny, p.d.nw, p.d.K,
                  p.L, p.Px, (int)p.d.prec, p.d.max_rhs, p.tc != nullptr ? 1 : 0);
    return b;
}

std::mutex g_tune_mutex;
std::map<std::string, int> g_tune_cache;
bool g_tune_file_read = false;

void read_tune_file() {
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char* path = std::getenv("ZL_AUTOTUNE_CACHE");
    if (path == nullptr) return;
    FILE* f = std::fopen(path, "r");
    if (f == nullptr) return;
    char line[256];
    while (std::fgets(line, sizeof(line), f) != nullptr) {
        std::string s(line);
        const size_t bar = s.rfind('|');
        if (bar == std::string::npos) continue;
        const int v = std::atoi(s.c_str() + bar + 1);
        if (v >= 0 && v < kVariants) g_tune_cache[s.substr(0, bar)] = v;
    }
    std::fclose(f);
}

void append_tune_file(const std::string& key, int v) {
    const char* path = std::getenv("ZL_AUTOTUNE_CACHE");
    if (path == nullptr) return;
    FILE* f = std::fopen(path, "a");
    if (f == nullptr) return;
    std::fprintf(f, "%s|%d\n", key.c_str(), v);
    std::fclose(f);
}

// Time variant v of plan p on R right-hand sides (median of kTuneReps after one warm-up).
float time_variant(zl_plan p, int v, const void* x, void* xt, int R, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1) {
    apply_variant(p, v);
    if (zl_apply_left_inverse(p, x, xt, R, s) != ZL_OK) return -1.f;
    float t[kTuneReps];
    for (int i = 0; i < kTuneReps; ++i) {
        cudaEventRecord(e0, s);
        if (zl_apply_left_inverse(p, x, xt, R, s) != ZL_OK) return -1.f;
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
        cudaEventElapsedTime(&t[i], e0, e1);
    }
    for (int i = 1; i < kTuneReps; ++i)
        for (int j = i; j > 0 && t[j] < t[j - 1]; --j) std::swap(t[j], t[j - 1]);
    return t[kTuneReps / 2];
}

zl_status autotune(zl_batch b, cudaStream_t s) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    read_tune_file();
    size_t in_max = 0, out_max = 0;
    for (zl_plan p : b->plans) {
        in_max = std::max(in_max, (size_t)p->d.max_rhs * (size_t)p->d.nw * (size_t)p->nh * p->esize);
        out_max = std::max(out_max, (size_t)p->d.max_rhs * (size_t)p->d.K * (size_t)p->L * p->esize);
    }
    void *x = nullptr, *xt = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    zl_status st = ZL_OK;
    if (zl::dev_malloc((void**)&x, in_max) != cudaSuccess || zl::dev_malloc((void**)&xt, out_max) != cudaSuccess) st = ZL_ERR_ALLOC;
    if (st == ZL_OK && (cudaMemsetAsync(x, 0, in_max, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                        cudaEventCreate(&e1) != cudaSuccess))
        st = ZL_ERR_CUDA;
    for (size_t i = 0; i < b->plans.size() && st == ZL_OK; ++i) {
        zl_plan p = b->plans[i];
        const std::string key = shape_key(*p);
        auto it = g_tune_cache.find(key);
        int best = 0;
        if (it != g_tune_cache.end()) {
            best = it->second;
        } else {
            float tbest = -1.f;
            for (int v = 0; v < kVariants; ++v) {
                if (v == 0 && p->d.prec == ZL_MIXED && p->tc == nullptr) continue;   // same as variant 5
                if (v == 5 && p->d.prec != ZL_MIXED) continue;                       // same as variant 0
                const float t = time_variant(p, v, x, xt, p->d.max_rhs, s, e0, e1);
                if (t < 0.f) { st = ZL_ERR_CUDA; break; }
                if (tbest < 0.f || t < tbest) { tbest = t; best = v; }
            }
            if (st != ZL_OK) break;
            g_tune_cache[key] = best;
            append_tune_file(key, best);
        }
        apply_variant(p, best);
        b->choice[i] = best;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(x);
    cudaFree(xt);
    return st;
}

void destroy_batch(zl_batch b) {
    for (auto& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (zl_plan p : b->plans) zl_destroy(p);
    for (cudaStream_t s : b->branch) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->origin) cudaStreamDestroy(b->origin);
    delete b;
}

// Capture one apply of every instance into a graph: fork from the origin stream, one
// branch per instance, join back.
zl_status capture(zl_batch b, const void* const* x, void* const* xt, const int* R, cudaGraphExec_t* exec) {
    const int n = (int)b->plans.size();
    if (cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return ZL_ERR_CUDA;
    zl_status st = ZL_OK;
    if (cudaEventRecord(b->fork, b->origin) != cudaSuccess) st = ZL_ERR_CUDA;
    for (int i = 0; i < n && st == ZL_OK; ++i) {
        if (cudaStreamWaitEvent(b->branch[i], b->fork, 0) != cudaSuccess) { st = ZL_ERR_CUDA; break; }
        if (R[i] > 0) st = zl_apply_left_inverse(b->plans[i], x[i], xt[i], R[i], b->branch[i]);
        if (st == ZL_OK && (cudaEventRecord(b->join[i], b->branch[i]) != cudaSuccess ||
                            cudaStreamWaitEvent(b->origin, b->join[i], 0) != cudaSuccess))
            st = ZL_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(b->origin, &graph);
    if (st == ZL_OK && ec != cudaSuccess) st = ZL_ERR_CUDA;
    if (st == ZL_OK && cudaGraphInstantiate(exec, graph, 0) != cudaSuccess) st = ZL_ERR_CUDA;
    if (graph) cudaGraphDestroy(graph);
    return st;
}

}  // namespace

extern "C" {

zl_status zl_setup_batch(int n, const zl_desc* descs, const void* const* Z, const double* const* spectra, void* stream,
                         zl_batch* out, int* failed_instance) {
    if (failed_instance) *failed_instance = -1;
    if (out == nullptr) return ZL_ERR_ARG;
    *out = nullptr;
    if (n <= 0 || descs == nullptr || Z == nullptr || spectra == nullptr) return ZL_ERR_ARG;
    for (int i = 0; i < n; ++i)
        if (Z[i] == nullptr || spectra[i] == nullptr) {
            if (failed_instance) *failed_instance = i;
            return ZL_ERR_ARG;
        }
    cudaStream_t s = (cudaStream_t)stream;
    zl_batch b = new zl_batch_s();
    b->choice.assign(n, 0);
    zl_status st = ZL_OK;
    for (int i = 0; i < n; ++i) {
        zl_plan p = nullptr;
        st = zl_setup(&descs[i], Z[i], spectra[i], stream, &p);
        if (st != ZL_OK) {
            if (p) zl_destroy(p);
            if (failed_instance) *failed_instance = i;
            break;
        }
        b->plans.push_back(p);
    }
    if (st == ZL_OK) {
        if (cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
            st = ZL_ERR_CUDA;
        for (int i = 0; i < n && st == ZL_OK; ++i) {
            cudaStream_t bs = nullptr;
            cudaEvent_t e = nullptr;
            if (cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking) != cudaSuccess) { st = ZL_ERR_CUDA; break; }
            b->branch.push_back(bs);
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { st = ZL_ERR_CUDA; break; }
            b->join.push_back(e);
        }
    }
    if (st == ZL_OK) st = autotune(b, s);
    if (st == ZL_OK && cudaStreamSynchronize(s) != cudaSuccess) st = ZL_ERR_CUDA;
    if (st != ZL_OK) {
        destroy_batch(b);
        return st;
    }
    *out = b;
    return ZL_OK;
}

zl_status zl_batch_get_info(zl_batch b, int i, zl_plan* plan, int* variant) {
    if (b == nullptr || i < 0 || i >= (int)b->plans.size()) return ZL_ERR_ARG;
    if (plan) *plan = b->plans[i];
    if (variant) *variant = b->choice[i];
    return ZL_OK;
}

zl_status zl_apply_left_inverse_batch(zl_batch b, const void* const* x, void* const* xt, const int* R, void* stream) {
    if (b == nullptr || x == nullptr || xt == nullptr || R == nullptr) return ZL_ERR_ARG;
    const int n = (int)b->plans.size();
    for (int i = 0; i < n; ++i) {
        if (R[i] < 0) return ZL_ERR_ARG;
        if (R[i] > 0 && (x[i] == nullptr || xt[i] == nullptr || x[i] == xt[i])) return ZL_ERR_ARG;
        if (b->plans[i]->bad_column >= 0) return ZL_ERR_RANK;
    }
    zl_batch_s::Graph* hit = nullptr;
    for (auto& g : b->graphs) {
        bool same = true;
        for (int i = 0; i < n && same; ++i) same = g.x[i] == x[i] && g.xt[i] == xt[i] && g.R[i] == R[i];
        if (same) { hit = &g; break; }
    }
    if (hit == nullptr) {
        zl_batch_s::Graph g;
        g.x.assign(x, x + n);
        g.xt.assign(xt, xt + n);
        g.R.assign(R, R + n);
        const zl_status st = capture(b, x, xt, R, &g.exec);
        if (st != ZL_OK) return st;
        if ((int)b->graphs.size() >= kMaxGraphs) {
            size_t lru = 0;
            for (size_t k = 1; k < b->graphs.size(); ++k)
                if (b->graphs[k].last_use < b->graphs[lru].last_use) lru = k;
            cudaGraphExecDestroy(b->graphs[lru].exec);
            b->graphs[lru] = g;
            hit = &b->graphs[lru];
        } else {
            b->graphs.push_back(g);
            hit = &b->graphs.back();
        }
    }
    hit->last_use = ++b->uses;
    return cudaGraphLaunch(hit->exec, (cudaStream_t)stream) == cudaSuccess ? ZL_OK : ZL_ERR_CUDA;
}

zl_status zl_destroy_batch(zl_batch b) {
    if (b == nullptr) return ZL_ERR_ARG;
    destroy_batch(b);
    return ZL_OK;
}

}  // extern "C"
