// Walks whose results exceed device memory: batches in two streams with
// ping-pong result pools (Section 5.2, Fig. 8 and Eq. 3).
//
// The queries are cut into batches of |P_G| queries so that two batches'
// result pools fit in the caller's byte budget; batch k runs on stream k mod 2
// with that stream's own pools, query cursor and counters, so while batch k
// walks, batch k-1's paths travel to the host.  Stream order alone keeps a
// pool from being refilled before its copy to the host has finished.  A query
// keeps its global id (q_id0 + its index) as its random counter, so the
// paths are the same as one launch over all queries would give.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "fw_internal.cuh"

using namespace fw;

namespace {

int fail_b(int status, const char* fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(status, buf);
}

// dst counters += src counters (the cursor is not a counter).
__global__ void add_counters_kernel(Scratch* dst, const Scratch* a, const Scratch* b) {
    const int i = threadIdx.x;
    if (i < C_NUM) dst->counters[i] += a->counters[i] + b->counters[i];
}

// Bytes one query needs in one pool: its path (L + 1 vertices), its start
// and its path length, 4 bytes each.
int64_t query_bytes(int32_t max_len) { return ((int64_t)max_len + 3) * 4; }

}  // namespace

extern "C" int64_t fw_batch_size(uint64_t budget_bytes, int32_t max_len) {
    if (max_len < 0) return 0;
    return (int64_t)(budget_bytes / (2ull * (uint64_t)query_bytes(max_len)));
}

extern "C" int fw_walk_batched(fw_graph* g, int32_t algo, const fw_params* p, const int32_t* h_starts, int64_t n_q,
                               const int32_t* h_lengths, int32_t max_len, uint64_t seed, int64_t q_id0,
                               uint64_t budget_bytes, int32_t* h_paths, int32_t* h_path_len, int64_t* batch_q) {
    if (!g || !p) return fail_b(FW_EINVAL, "fw_walk_batched: NULL graph or params");
    if (n_q < 0 || max_len < 0) return fail_b(FW_EINVAL, "fw_walk_batched: n_q or max_len < 0");
    if (n_q > 0 && (!h_starts || !h_paths || !h_path_len))
        return fail_b(FW_EINVAL, "fw_walk_batched: NULL starts/paths/path_len");
    GraphDev gd;
    int dev = 0;
    Tuning tu;
    graph_device_view(g, &gd, &dev, &tu);
    std::lock_guard<std::mutex> lock(graph_mutex(g));
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    cudaSetDevice(dev);
    struct DevGuard {
        int d;
        ~DevGuard() { cudaSetDevice(d); }
    } guard{cur_dev};

    // request template: parameters checked once
    fw_request rq;
    memset(&rq, 0, sizeof rq);
    rq.algo = algo;
    rq.params = *p;
    rq.max_len = max_len;
    rq.seed = seed;
    ReqDev base;
    int rc = make_request(g, rq, &base);
    if (rc != FW_OK) return rc;
    if (n_q == 0) {
        if (batch_q) *batch_q = 0;
        return FW_OK;
    }

    // Eq. 3: |P_G| = floor((M - M_G) / (2 (L_max + 1) M_v)); the budget
    // stands for M - M_G (0: the free device memory less 256 MiB)
    if (budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail_b(FW_ECUDA, "fw_walk_batched: cudaMemGetInfo failed");
        budget_bytes = fr > (256ull << 20) ? fr - (256ull << 20) : 0;
    }
    int64_t P = fw_batch_size(budget_bytes, max_len);
    if (P < 1) return fail_b(FW_ENOMEM, "fw_walk_batched: the budget holds no query (need %lld bytes per query pair)",
                             (long long)(2 * query_bytes(max_len)));
    if (P > n_q) P = n_q;
    if (batch_q) *batch_q = P;
    const int64_t width = (int64_t)max_len + 1;

    struct Pool {
        int32_t* starts = nullptr;
        int32_t* lengths = nullptr;
        int32_t* paths = nullptr;
        int32_t* len = nullptr;
        Scratch* scratch = nullptr;
        cudaStream_t st = nullptr;
    } pool[2];
    unsigned long long* h_zero = nullptr;
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    for (Pool& q : pool) {
        chk(cudaMalloc(&q.starts, (size_t)P * 4));
        if (h_lengths) chk(cudaMalloc(&q.lengths, (size_t)P * 4));
        chk(cudaMalloc(&q.paths, (size_t)(P * width) * 4));
        chk(cudaMalloc(&q.len, (size_t)P * 4));
        chk(cudaMalloc(&q.scratch, sizeof(Scratch)));
        chk(cudaStreamCreateWithFlags(&q.st, cudaStreamNonBlocking));
        if (e == cudaSuccess) chk(cudaMemsetAsync(q.scratch, 0, sizeof(Scratch), q.st));
    }
    chk(cudaHostAlloc(&h_zero, sizeof(unsigned long long), cudaHostAllocDefault));
    if (h_zero) *h_zero = 0;

    const int64_t nb = (n_q + P - 1) / P;
    for (int64_t b = 0; b < nb && e == cudaSuccess; ++b) {
        Pool& q = pool[b & 1];
        const int64_t q0 = b * P, nbq = n_q - q0 < P ? n_q - q0 : P;
        // this stream's previous batch copied out before these writes (stream order)
        chk(cudaMemcpyAsync(q.starts, h_starts + q0, (size_t)nbq * 4, cudaMemcpyHostToDevice, q.st));
        if (h_lengths) chk(cudaMemcpyAsync(q.lengths, h_lengths + q0, (size_t)nbq * 4, cudaMemcpyHostToDevice, q.st));
        chk(cudaMemcpyAsync(&q.scratch->cursor, h_zero, sizeof(unsigned long long), cudaMemcpyHostToDevice, q.st));
        ReqTable tab;
        memset(&tab, 0, sizeof tab);
        ReqDev& r = tab.r[0];
        r = base;
        r.starts = q.starts;
        r.lengths = q.lengths;
        r.paths = q.paths;
        r.path_len = q.len;
        r.n_q = nbq;
        r.q_begin = 0;
        r.q_id0 = q_id0 + q0;
        if (e == cudaSuccess) chk(launch_walk(gd, rq.params.mode, tab, 1, nbq, q.scratch, tu, q.st));
        chk(cudaMemcpyAsync(h_paths + q0 * width, q.paths, (size_t)(nbq * width) * 4, cudaMemcpyDeviceToHost, q.st));
        chk(cudaMemcpyAsync(h_path_len + q0, q.len, (size_t)nbq * 4, cudaMemcpyDeviceToHost, q.st));
    }
    for (Pool& q : pool)
        if (q.st) chk(cudaStreamSynchronize(q.st));
    // the work shows in the graph's counters (fw_stats)
    unsigned long long cnt[C_NUM];
    memset(cnt, 0, sizeof cnt);
    if (e == cudaSuccess) {
        add_counters_kernel<<<1, 32, 0, pool[0].st>>>(graph_scratch(g), pool[0].scratch, pool[1].scratch);
        chk(cudaGetLastError());
        chk(cudaStreamSynchronize(pool[0].st));
    }
    for (Pool& q : pool) {
        unsigned long long c[C_NUM];
        if (e == cudaSuccess && cudaMemcpy(c, q.scratch->counters, sizeof c, cudaMemcpyDeviceToHost) == cudaSuccess)
            for (int i = 0; i < C_NUM; ++i) cnt[i] += c[i];
        cudaFree(q.starts);
        cudaFree(q.lengths);
        cudaFree(q.paths);
        cudaFree(q.len);
        cudaFree(q.scratch);
        if (q.st) cudaStreamDestroy(q.st);
    }
    if (h_zero) cudaFreeHost(h_zero);
    if (e != cudaSuccess)
        return fail_b(e == cudaErrorMemoryAllocation ? FW_ENOMEM : FW_ECUDA, "fw_walk_batched: %s",
                      cudaGetErrorString(e));
    if (cnt[C_TIMEOUT]) return fail_b(FW_ETIMEOUT, "fw_walk_batched: a device wait timed out");
    if (cnt[C_BAD_INPUT])
        return fail_b(FW_EINVAL, "fw_walk_batched: %llu queries had an out-of-range start (written as empty paths)",
                      (unsigned long long)cnt[C_BAD_INPUT]);
    return FW_OK;
}
