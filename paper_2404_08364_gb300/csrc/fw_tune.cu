// CUDA-graph launches and the engine autotuner.
//
// A multi-request walk launch (requests of mixed algorithms and very uneven
// lengths, e.g. PPR's geometric stops next to fixed-length MetaPath) is
// captured once into a CUDA graph and replayed: the cursor reset and the
// persistent engine launch become one graph launch.  The autotuner times the
// engine on a caller-given sample of the workload over a small grid of
// tunings (CTA size, hub threshold d_t, walk slots), keeps the fastest, and
// caches the choice by (GPU name, algorithm mix, degree-histogram bucket).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "fw_internal.cuh"

using namespace fw;

namespace {

int fail_t(int status, const char* fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(status, buf);
}

std::mutex g_cache_mu;
std::map<std::string, fw_tuning> g_cache;

std::string cache_key(const fw_graph* g, const fw_request* reqs, int n_req) {
    GraphDev gd;
    int dev = 0;
    Tuning tu;
    graph_device_view(g, &gd, &dev, &tu);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    unsigned algos = 0;
    for (int i = 0; i < n_req; ++i) algos |= 1u << (reqs[i].algo & 7) | (reqs[i].params.mode ? 0x100u : 0u);
    // degree-histogram bucket: log2 of the mean degree and of the maximum degree
    int64_t n = 0, m = 0, dmax = 0;
    int32_t a, b, c;
    fw_graph_info(g, &n, &m, &dmax, &a, &b, &c);
    int lmean = 0, lmax = 0;
    for (int64_t x = m / (n > 0 ? n : 1); x > 1; x >>= 1) ++lmean;
    for (int64_t x = dmax; x > 1; x >>= 1) ++lmax;
    char buf[512];
    snprintf(buf, sizeof buf, "%.256s|algos=%x|mean2^%d|max2^%d", prop.name, algos, lmean, lmax);
    return buf;
}

}  // namespace

struct fw_exec {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" int fw_capture_multi(fw_graph* g, const fw_request* reqs, int32_t n_req, fw_exec** out) {
    if (!g || !reqs || !out) return fail_t(FW_EINVAL, "fw_capture_multi: NULL argument");
    *out = nullptr;
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return fail_t(FW_ECUDA, "fw_capture_multi: stream creation failed");
    fw_exec* X = new fw_exec();
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
    int rc = e == cudaSuccess ? fw_walk_multi(g, reqs, n_req, st) : FW_ECUDA;
    cudaError_t e2 = cudaStreamEndCapture(st, &X->graph);
    if (rc == FW_OK && e2 == cudaSuccess) e2 = cudaGraphInstantiate(&X->exec, X->graph, 0);
    cudaStreamDestroy(st);
    if (rc != FW_OK || e != cudaSuccess || e2 != cudaSuccess) {
        fw_exec_destroy(X);
        if (rc != FW_OK) return rc;
        return fail_t(FW_ECUDA, "fw_capture_multi: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    *out = X;
    return FW_OK;
}

extern "C" int fw_exec_launch(fw_exec* X, void* stream) {
    if (!X || !X->exec) return fail_t(FW_EINVAL, "fw_exec_launch: NULL exec");
    cudaError_t e = cudaGraphLaunch(X->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail_t(FW_ECUDA, "fw_exec_launch: %s", cudaGetErrorString(e));
    return FW_OK;
}

extern "C" void fw_exec_destroy(fw_exec* X) {
    if (!X) return;
    if (X->exec) cudaGraphExecDestroy(X->exec);
    if (X->graph) cudaGraphDestroy(X->graph);
    delete X;
}

extern "C" int fw_autotune(fw_graph* g, const fw_request* reqs, int32_t n_req, int32_t reps, fw_tuning* best,
                           double* best_steps_per_s) {
    if (!g || !reqs || !best) return fail_t(FW_EINVAL, "fw_autotune: NULL argument");
    if (n_req < 1 || n_req > 16) return fail_t(FW_EINVAL, "fw_autotune: n_req must be in [1, 16]");
    if (reps < 1) reps = 2;
    const std::string key = cache_key(g, reqs, n_req);
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            *best = it->second;
            if (best_steps_per_s) *best_steps_per_s = 0.0;
            return fw_set_tuning(g, best);
        }
    }
    fw_tuning saved;
    fw_get_tuning(g, &saved);
    const int threads[] = {128, 256, 512};
    const int dts[] = {2048, 8192, 32768, 1 << 20};
    const int slots_per_warp[] = {1, 2, 4};
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess)
        return fail_t(FW_ECUDA, "fw_autotune: stream creation failed");
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    double best_rate = -1.0;
    fw_tuning best_t = saved;
    int rc = FW_OK;
    for (int nt : threads)
        for (int dt : dts)
            for (int spw : slots_per_warp) {
                fw_tuning t = {nt, spw * (nt / 32), dt, 0};
                fw_set_tuning(g, &t);
                fw_stats_reset(g, st);
                rc = fw_walk_multi(g, reqs, n_req, st);  // warm-up
                if (rc != FW_OK) break;
                fw_stats_reset(g, st);
                cudaEventRecord(e0, st);
                for (int r = 0; r < reps && rc == FW_OK; ++r) rc = fw_walk_multi(g, reqs, n_req, st);
                cudaEventRecord(e1, st);
                if (rc != FW_OK) break;
                fw_stats_t s;
                rc = fw_stats(g, &s);
                if (rc != FW_OK) break;
                cudaEventSynchronize(e1);
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                const double rate = ms > 0 ? (double)s.steps / (ms * 1e-3) : 0.0;
                if (rate > best_rate) {
                    best_rate = rate;
                    fw_get_tuning(g, &best_t);
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaStreamDestroy(st);
    if (rc != FW_OK) {
        fw_set_tuning(g, &saved);
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        g_cache[key] = best_t;
    }
    *best = best_t;
    if (best_steps_per_s) *best_steps_per_s = best_rate;
    return fw_set_tuning(g, &best_t);
}

extern "C" int fw_autotune_clear_cache(void) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache.clear();
    return FW_OK;
}
