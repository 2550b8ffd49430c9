// C ABI of the walk library: graph residency and validation, walk entry
// points (device or host buffers), tuning and counters.  See include/fw.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <new>

#include "fw_internal.cuh"

using namespace fw;

// ------------------------------------------------------------------ errors

static thread_local char g_last_error[512] = "";

static int fail(int status, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return status;
}

#define FW_CUDA_TRY(expr)                                                                    \
    do {                                                                                     \
        cudaError_t _e = (expr);                                                             \
        if (_e != cudaSuccess) {                                                             \
            if (_e == cudaErrorMemoryAllocation)                                             \
                return fail(FW_ENOMEM, "%s: %s", #expr, cudaGetErrorString(_e));            \
            return fail(FW_ECUDA, "%s: %s", #expr, cudaGetErrorString(_e));                 \
        }                                                                                    \
    } while (0)

extern "C" const char* fw_strerror(int s) {
    switch (s) {
        case FW_OK: return "ok";
        case FW_EINVAL: return "invalid argument";
        case FW_ENOMEM: return "out of memory";
        case FW_ECUDA: return "CUDA error";
        case FW_EUNSORTED: return "CSR row not strictly ascending";
        case FW_ETIMEOUT: return "bounded device wait timed out";
        case FW_EBUSY: return "busy";
        default: return "unknown status";
    }
}

extern "C" const char* fw_last_error(void) { return g_last_error; }

extern "C" int fw_version(void) { return (1 << 16) | 0; }

// ------------------------------------------------------------------- graph

struct fw_graph {
    int device;
    GraphDev g;
    bool owned;
    int64_t d_max;
    uint32_t max_w_u32;
    Scratch* scratch;          // device: cursor + counters
    Tuning tuning;
    cudaStream_t last_stream;
    cudaEvent_t ev0, ev1;
    bool timed;
    std::mutex mu;
};

namespace {

// Validation flags raised by the check kernels.
enum : int { V_ROWPTR = 1, V_COLRANGE = 2, V_UNSORTED = 4, V_WF32 = 8, V_WU32 = 16 };

struct CheckOut {
    int flags;
    int pad;
    unsigned long long d_max;
    unsigned int max_w_u32;
};

__global__ void check_rows_kernel(const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                                  int64_t n, int64_t m, CheckOut* out) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    unsigned long long dmax = 0;
    int flags = 0;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += warps) {
        const int64_t b = row_ptr[v], e = row_ptr[v + 1];
        if (b < 0 || e < b || e > m) {
            flags |= V_ROWPTR;
            continue;
        }
        dmax = max(dmax, (unsigned long long)(e - b));
        for (int64_t i = b + lane; i < e; i += 32) {
            const int32_t c = col[i];
            if (c < 0 || c >= n) flags |= V_COLRANGE;
            if (i + 1 < e && !(c < col[i + 1])) flags |= V_UNSORTED;
        }
    }
    if (flags) atomicOr(&out->flags, flags);
    if (dmax) atomicMax(&out->d_max, dmax);
}

__global__ void check_weights_kernel(const float* __restrict__ wf, const uint32_t* __restrict__ wu,
                                     int64_t m, CheckOut* out) {
    int flags = 0;
    unsigned int wmax = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (wf) {
            const float w = wf[i];
            if (!(w > 0.0f) || !isfinite(w)) flags |= V_WF32;
        }
        if (wu) {
            const uint32_t w = wu[i];
            if (w == 0) flags |= V_WU32;
            wmax = max(wmax, w);
        }
    }
    if (flags) atomicOr(&out->flags, flags);
    if (wmax) atomicMax(&out->max_w_u32, wmax);
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int dev_copy(T** dst, const T* src, int64_t count, bool from_host) {
    *dst = nullptr;
    if (!src || count == 0) return FW_OK;
    // pad to a multiple of 4 elements so 16-byte vector loads of a row's last
    // quad stay inside the allocation
    const size_t bytes = (size_t)((count + 3) & ~3ll) * sizeof(T);
    FW_CUDA_TRY(cudaMalloc((void**)dst, bytes));
    cudaError_t e = cudaMemcpy(*dst, src, (size_t)count * sizeof(T),
                               from_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice);
    if (e == cudaSuccess && bytes > (size_t)count * sizeof(T))
        e = cudaMemset((char*)*dst + (size_t)count * sizeof(T), 0, bytes - (size_t)count * sizeof(T));
    if (e != cudaSuccess) {
        cudaFree(*dst);
        *dst = nullptr;
        return fail(FW_ECUDA, "graph copy: %s", cudaGetErrorString(e));
    }
    return FW_OK;
}

void release(fw_graph* G) {
    if (!G) return;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(G->device);
    if (G->owned) {
        cudaFree((void*)G->g.row_ptr);
        cudaFree((void*)G->g.col);
        cudaFree((void*)G->g.w_f32);
        cudaFree((void*)G->g.w_u32);
        cudaFree((void*)G->g.etype);
    }
    if (G->scratch) cudaFree(G->scratch);
    if (G->ev0) cudaEventDestroy(G->ev0);
    if (G->ev1) cudaEventDestroy(G->ev1);
    cudaSetDevice(cur);
    delete G;
}

}  // namespace

extern "C" int fw_load_csr(fw_graph** out, int64_t n, int64_t m, const int64_t* row_ptr,
                           const int32_t* col, const float* w_f32, const uint32_t* w_u32,
                           const int8_t* etype, uint32_t flags) {
    if (!out) return fail(FW_EINVAL, "fw_load_csr: out is NULL");
    *out = nullptr;
    if (n < 1 || n >= (int64_t)1 << 31 || m < 0) return fail(FW_EINVAL, "fw_load_csr: bad sizes n=%lld m=%lld", (long long)n, (long long)m);
    if (!row_ptr || (m > 0 && !col)) return fail(FW_EINVAL, "fw_load_csr: row_ptr/col is NULL");
    const bool borrow = (flags & FW_BORROW) != 0;
    const bool dev_in = borrow || (flags & FW_DEVICE_PTRS) != 0;
    if (dev_in && (!is_device_ptr(row_ptr) || (m > 0 && !is_device_ptr(col))))
        return fail(FW_EINVAL, "fw_load_csr: device flag set but row_ptr/col are not device memory");
    if (borrow) {
        const void* ps[] = {row_ptr, col, w_f32, w_u32, etype};
        for (const void* p : ps)
            if (p && ((uintptr_t)p & 15)) return fail(FW_EINVAL, "fw_load_csr: borrowed array not 16-byte aligned");
    }

    fw_graph* G = new (std::nothrow) fw_graph();
    if (!G) return fail(FW_ENOMEM, "fw_load_csr: host allocation");
    cudaGetDevice(&G->device);
    G->owned = !borrow;
    G->g.n = n;
    G->g.m = m;
    G->tuning = default_tuning();
    int rc = FW_OK;
    if (borrow) {
        G->g.row_ptr = row_ptr;
        G->g.col = col;
        G->g.w_f32 = w_f32;
        G->g.w_u32 = w_u32;
        G->g.etype = etype;
    } else {
        int64_t* rp = nullptr;
        int32_t* c = nullptr;
        float* wf = nullptr;
        uint32_t* wu = nullptr;
        int8_t* et = nullptr;
        if ((rc = dev_copy(&rp, row_ptr, n + 1, !dev_in)) == FW_OK &&
            (rc = dev_copy(&c, col, m, !dev_in)) == FW_OK &&
            (rc = dev_copy(&wf, w_f32, m, !dev_in)) == FW_OK &&
            (rc = dev_copy(&wu, w_u32, m, !dev_in)) == FW_OK)
            rc = dev_copy(&et, etype, m, !dev_in);
        G->g.row_ptr = rp;
        G->g.col = c;
        G->g.w_f32 = wf;
        G->g.w_u32 = wu;
        G->g.etype = et;
        if (rc != FW_OK) {
            release(G);
            return rc;
        }
    }
    if (cudaMalloc(&G->scratch, sizeof(Scratch)) != cudaSuccess || cudaMemset(G->scratch, 0, sizeof(Scratch)) != cudaSuccess) {
        release(G);
        return fail(FW_ENOMEM, "fw_load_csr: scratch allocation");
    }
    if (cudaEventCreate(&G->ev0) != cudaSuccess || cudaEventCreate(&G->ev1) != cudaSuccess) {
        release(G);
        return fail(FW_ECUDA, "fw_load_csr: event creation");
    }

    // ---- checks (and the max degree / max integer weight) on the device ----
    CheckOut* dco = nullptr;
    CheckOut co = {};
    if (cudaMalloc(&dco, sizeof(CheckOut)) != cudaSuccess) {
        release(G);
        return fail(FW_ENOMEM, "fw_load_csr: check buffer");
    }
    cudaMemset(dco, 0, sizeof(CheckOut));
    int64_t ends[2] = {0, 0};
    cudaMemcpy(&ends[0], G->g.row_ptr, sizeof(int64_t), cudaMemcpyDeviceToHost);
    cudaMemcpy(&ends[1], G->g.row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, G->device);
    check_rows_kernel<<<sms * 8, 256>>>(G->g.row_ptr, G->g.col, n, m, dco);
    if (m > 0 && (G->g.w_f32 || G->g.w_u32))
        check_weights_kernel<<<sms * 8, 256>>>(G->g.w_f32, G->g.w_u32, m, dco);
    cudaError_t e = cudaMemcpy(&co, dco, sizeof co, cudaMemcpyDeviceToHost);
    cudaFree(dco);
    if (e != cudaSuccess) {
        release(G);
        return fail(FW_ECUDA, "fw_load_csr: checks: %s", cudaGetErrorString(e));
    }
    G->d_max = (int64_t)co.d_max;
    G->max_w_u32 = co.max_w_u32;
    // offsets and column ranges are always enforced: the kernels index by them
    if (ends[0] != 0 || ends[1] != m || (co.flags & V_ROWPTR)) rc = fail(FW_EINVAL, "fw_load_csr: row_ptr not monotone from 0 to m");
    else if (co.flags & V_COLRANGE) rc = fail(FW_EINVAL, "fw_load_csr: column index out of [0, n)");
    else if (!(flags & FW_NO_VALIDATE)) {
        if (co.flags & V_UNSORTED) rc = fail(FW_EUNSORTED, "fw_load_csr: a row is not strictly ascending");
        else if (co.flags & V_WF32) rc = fail(FW_EINVAL, "fw_load_csr: w_f32 has a non-positive or non-finite weight");
        else if (co.flags & V_WU32) rc = fail(FW_EINVAL, "fw_load_csr: w_u32 has a zero weight");
    }
    if (rc != FW_OK) {
        release(G);
        return rc;
    }
    *out = G;
    return FW_OK;
}

extern "C" void fw_free(fw_graph* g) { release(g); }

extern "C" int fw_graph_info(const fw_graph* g, int64_t* n, int64_t* m, int64_t* d_max, int32_t* has_f32,
                             int32_t* has_u32, int32_t* has_type) {
    if (!g) return fail(FW_EINVAL, "fw_graph_info: NULL graph");
    if (n) *n = g->g.n;
    if (m) *m = g->g.m;
    if (d_max) *d_max = g->d_max;
    if (has_f32) *has_f32 = g->g.w_f32 != nullptr;
    if (has_u32) *has_u32 = g->g.w_u32 != nullptr;
    if (has_type) *has_type = g->g.etype != nullptr;
    return FW_OK;
}

extern "C" int fw_set_tuning(fw_graph* g, const fw_tuning* t) {
    if (!g) return fail(FW_EINVAL, "fw_set_tuning: NULL graph");
    Tuning tu = default_tuning();
    if (t) tu = Tuning{t->block_threads, t->slots, t->d_warp, t->ctas_per_sm};
    g->tuning = sanitize_tuning(tu);
    return FW_OK;
}

extern "C" int fw_get_tuning(const fw_graph* g, fw_tuning* out) {
    if (!g || !out) return fail(FW_EINVAL, "fw_get_tuning: NULL argument");
    out->block_threads = g->tuning.block_threads;
    out->slots = g->tuning.slots;
    out->d_warp = g->tuning.d_warp;
    out->ctas_per_sm = g->tuning.ctas_per_sm;
    return FW_OK;
}

// ------------------------------------------------------------------- walks

namespace {

// Fill the parameter part of a device request; FW_EINVAL on bad parameters.
int make_req(const fw_graph* G, int32_t algo, const fw_params* p, int32_t max_len, uint64_t seed,
             ReqDev* r) {
    if (algo < FW_WEIGHTED || algo > FW_PPR) return fail(FW_EINVAL, "unknown algo %d", algo);
    if (!p) return fail(FW_EINVAL, "params is NULL");
    if (p->mode != FW_EXACT && p->mode != FW_FAST) return fail(FW_EINVAL, "unknown mode %d", p->mode);
    if (max_len < 0) return fail(FW_EINVAL, "max_len < 0");
    const bool exact = p->mode == FW_EXACT;
    if (exact && !G->g.w_u32) return fail(FW_EINVAL, "exact mode needs w_u32");
    if (!exact && !G->g.w_f32) return fail(FW_EINVAL, "fast mode needs w_f32");
    memset(r, 0, sizeof *r);
    r->max_len = max_len;
    r->algo = algo;
    r->seed = seed;
    r->fac_i[0] = r->fac_i[1] = r->fac_i[2] = 1;
    r->fac_f[0] = r->fac_f[1] = r->fac_f[2] = 1.0f;
    if (algo == FW_NODE2VEC) {
        if (!(p->n2v_p > 0.0f) || !(p->n2v_q > 0.0f) || !isfinite(p->n2v_p) || !isfinite(p->n2v_q))
            return fail(FW_EINVAL, "node2vec p, q must be positive");
        r->fac_f[0] = 1.0f / p->n2v_p;
        r->fac_f[1] = 1.0f;
        r->fac_f[2] = 1.0f / p->n2v_q;
        if (exact) {
            const double S = p->n2v_scale > 0 ? p->n2v_scale : 2;
            const double f[3] = {S / (double)p->n2v_p, S, S / (double)p->n2v_q};
            uint64_t fmax = 0;
            for (int j = 0; j < 3; ++j) {
                if (f[j] < 1.0 || f[j] > 65536.0 || f[j] != floor(f[j]))
                    return fail(FW_EINVAL, "exact node2vec factors S/p, S, S/q must be integers in [1, 65536]");
                r->fac_i[j] = (uint32_t)f[j];
                fmax = fmax > r->fac_i[j] ? fmax : r->fac_i[j];
            }
            if ((uint64_t)G->max_w_u32 * fmax > 0xFFFFFFFFull)
                return fail(FW_EINVAL, "exact node2vec: max w_u32 x factor exceeds 32 bits");
        }
    }
    if (algo == FW_METAPATH) {
        if (!G->g.etype) return fail(FW_EINVAL, "MetaPath needs edge labels");
        if (p->schema_len < 1 || p->schema_len > 16) return fail(FW_EINVAL, "schema_len must be in [1, 16]");
        r->schema_len = p->schema_len;
        memcpy(r->schema, p->schema, 16);
    } else {
        r->schema_len = 1;
    }
    if (algo == FW_PPR) {
        if (!(p->ppr_stop >= 0.0 && p->ppr_stop <= 1.0)) return fail(FW_EINVAL, "ppr_stop must be in [0, 1]");
        const double t = p->ppr_stop * 4294967296.0;
        r->t_stop = t >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)t;
    }
    return FW_OK;
}

int launch(fw_graph* G, int mode, const ReqTable& tab, int n_req, int64_t total, cudaStream_t st) {
    FW_CUDA_TRY(cudaMemsetAsync(&G->scratch->cursor, 0, sizeof(unsigned long long), st));
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool timed = cap == cudaStreamCaptureStatusNone;
    if (timed) FW_CUDA_TRY(cudaEventRecord(G->ev0, st));
    cudaError_t e = launch_walk(G->g, mode, tab, n_req, total, G->scratch, G->tuning, st);
    if (e != cudaSuccess) return fail(FW_ECUDA, "walk launch: %s", cudaGetErrorString(e));
    if (timed) FW_CUDA_TRY(cudaEventRecord(G->ev1, st));
    G->timed = timed;
    G->last_stream = st;
    return FW_OK;
}

}  // namespace

namespace fw {

int set_error(int status, const char* msg) { return fail(status, "%s", msg); }

int graph_device_view(const fw_graph* g, GraphDev* out, int* device, Tuning* tuning) {
    *out = g->g;
    *device = g->device;
    *tuning = g->tuning;
    return FW_OK;
}

int make_request(const fw_graph* g, const fw_request& q, ReqDev* out) {
    return make_req(g, q.algo, &q.params, q.max_len, q.seed, out);
}

Scratch* graph_scratch(const fw_graph* g) { return g->scratch; }

std::mutex& graph_mutex(fw_graph* g) { return g->mu; }

}  // namespace fw

extern "C" int fw_walk_ex(fw_graph* G, int32_t algo, const fw_params* p, const int32_t* starts, int64_t n_q,
                          const int32_t* lengths, int32_t max_len, uint64_t seed, int64_t q_id0,
                          const int32_t* prev, const int32_t* step0, int32_t* paths, int32_t* path_len,
                          void* stream) {
    if (!G) return fail(FW_EINVAL, "fw_walk: NULL graph");
    if (n_q < 0) return fail(FW_EINVAL, "fw_walk: n_q < 0");
    if (n_q > 0 && (!starts || !paths || !path_len)) return fail(FW_EINVAL, "fw_walk: NULL starts/paths/path_len");
    std::lock_guard<std::mutex> lock(G->mu);
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    if (cur_dev != G->device) FW_CUDA_TRY(cudaSetDevice(G->device));
    struct DevGuard {
        int d;
        ~DevGuard() { cudaSetDevice(d); }
    } guard{cur_dev};

    ReqTable tab;
    memset(&tab, 0, sizeof tab);
    ReqDev& r = tab.r[0];
    int rc = make_req(G, algo, p, max_len, seed, &r);
    if (rc != FW_OK) return rc;
    if (n_q == 0) return FW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    r.n_q = n_q;
    r.q_begin = 0;
    r.q_id0 = q_id0;

    // classify buffers; host ones are staged through device memory
    const int64_t width = (int64_t)max_len + 1;
    struct Buf {
        const void* host;
        size_t bytes;
        bool in;
        void* dev;
    };
    Buf bufs[6] = {{starts, (size_t)n_q * 4, true, nullptr},
                   {lengths, (size_t)n_q * 4, true, nullptr},
                   {prev, (size_t)n_q * 4, true, nullptr},
                   {step0, (size_t)n_q * 4, true, nullptr},
                   {paths, (size_t)n_q * (size_t)width * 4, false, nullptr},
                   {path_len, (size_t)n_q * 4, false, nullptr}};
    bool any_host = false;
    for (Buf& b : bufs) {
        if (!b.host) continue;
        if (is_device_ptr(b.host)) {
            b.dev = (void*)b.host;
            b.host = nullptr;
        } else {
            any_host = true;
        }
    }
    if (any_host) {
        // host-side checks are cheap here: the inputs are in host memory
        const int32_t* hs = bufs[0].host ? starts : nullptr;
        const int32_t* hp = bufs[2].host ? prev : nullptr;
        for (int64_t i = 0; hs && i < n_q; ++i)
            if (hs[i] < 0 || hs[i] >= G->g.n) return fail(FW_EINVAL, "fw_walk: start vertex %d out of range", hs[i]);
        for (int64_t i = 0; hp && i < n_q; ++i)
            if (hp[i] < -1 || hp[i] >= G->g.n) return fail(FW_EINVAL, "fw_walk: prev vertex %d out of range", hp[i]);
        for (Buf& b : bufs) {
            if (!b.host) continue;
            cudaError_t e = cudaMallocAsync(&b.dev, b.bytes, st);
            if (e != cudaSuccess) {
                for (Buf& c : bufs)
                    if (c.host && c.dev) cudaFreeAsync(c.dev, st);
                return fail(FW_ENOMEM, "fw_walk: staging buffer: %s", cudaGetErrorString(e));
            }
            if (b.in) FW_CUDA_TRY(cudaMemcpyAsync(b.dev, b.host, b.bytes, cudaMemcpyHostToDevice, st));
        }
    }
    r.starts = (const int32_t*)bufs[0].dev;
    r.lengths = (const int32_t*)bufs[1].dev;
    r.prev = (const int32_t*)bufs[2].dev;
    r.step0 = (const int32_t*)bufs[3].dev;
    r.paths = (int32_t*)bufs[4].dev;
    r.path_len = (int32_t*)bufs[5].dev;
    rc = launch(G, p->mode, tab, 1, n_q, st);
    if (any_host) {
        for (Buf& b : bufs) {
            if (!b.host) continue;
            if (!b.in && rc == FW_OK) {
                cudaError_t e = cudaMemcpyAsync((void*)b.host, b.dev, b.bytes, cudaMemcpyDeviceToHost, st);
                if (e != cudaSuccess) rc = fail(FW_ECUDA, "fw_walk: copy-out: %s", cudaGetErrorString(e));
            }
            cudaFreeAsync(b.dev, st);
        }
        cudaError_t e = cudaStreamSynchronize(st);
        if (rc == FW_OK && e != cudaSuccess) rc = fail(FW_ECUDA, "fw_walk: %s", cudaGetErrorString(e));
    }
    return rc;
}

extern "C" int fw_walk(fw_graph* g, int32_t algo, const fw_params* p, const int32_t* starts, int64_t n_q,
                       const int32_t* lengths, int32_t max_len, uint64_t seed, const int32_t* prev,
                       const int32_t* step0, int32_t* paths, int32_t* path_len, void* stream) {
    return fw_walk_ex(g, algo, p, starts, n_q, lengths, max_len, seed, 0, prev, step0, paths, path_len,
                      stream);
}

extern "C" int fw_walk_multi(fw_graph* G, const fw_request* reqs, int32_t n_req, void* stream) {
    if (!G || !reqs) return fail(FW_EINVAL, "fw_walk_multi: NULL argument");
    if (n_req < 1 || n_req > kMaxInlineReqs) return fail(FW_EINVAL, "fw_walk_multi: n_req must be in [1, %d]", kMaxInlineReqs);
    std::lock_guard<std::mutex> lock(G->mu);
    ReqTable tab;
    memset(&tab, 0, sizeof tab);
    int64_t total = 0;
    const int mode = reqs[0].params.mode;
    for (int i = 0; i < n_req; ++i) {
        const fw_request& q = reqs[i];
        if (q.params.mode != mode) return fail(FW_EINVAL, "fw_walk_multi: requests must share one mode");
        if (q.n_q < 0) return fail(FW_EINVAL, "fw_walk_multi: n_q < 0");
        if (q.n_q > 0 && (!q.starts || !q.paths || !q.path_len))
            return fail(FW_EINVAL, "fw_walk_multi: NULL starts/paths/path_len");
        const void* ps[] = {q.starts, q.lengths, q.prev, q.step0, q.paths, q.path_len};
        for (const void* pp : ps)
            if (pp && !is_device_ptr(pp)) return fail(FW_EINVAL, "fw_walk_multi: buffers must be device memory");
        ReqDev& r = tab.r[i];
        int rc = make_req(G, q.algo, &q.params, q.max_len, q.seed, &r);
        if (rc != FW_OK) return rc;
        r.starts = q.starts;
        r.lengths = q.lengths;
        r.prev = q.prev;
        r.step0 = q.step0;
        r.paths = q.paths;
        r.path_len = q.path_len;
        r.n_q = q.n_q;
        r.q_begin = total;
        r.q_id0 = q.q_id0;
        total += q.n_q;
    }
    if (total == 0) return FW_OK;
    return launch(G, mode, tab, n_req, total, (cudaStream_t)stream);
}

extern "C" int fw_sync(void* stream) {
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return fail(FW_ECUDA, "fw_sync: %s", cudaGetErrorString(e));
    return FW_OK;
}

extern "C" int fw_stats(fw_graph* G, fw_stats_t* out) {
    if (!G || !out) return fail(FW_EINVAL, "fw_stats: NULL argument");
    std::lock_guard<std::mutex> lock(G->mu);
    cudaError_t e = cudaStreamSynchronize(G->last_stream);
    if (e != cudaSuccess) return fail(FW_ECUDA, "fw_stats: %s", cudaGetErrorString(e));
    Scratch s;
    e = cudaMemcpy(&s, G->scratch, sizeof s, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(FW_ECUDA, "fw_stats: %s", cudaGetErrorString(e));
    memset(out, 0, sizeof *out);
    out->walks = s.counters[C_WALKS];
    out->steps = s.counters[C_STEPS];
    out->rows_scanned = s.counters[C_ROWS];
    out->warp_steps = s.counters[C_WARP_STEPS];
    out->block_steps = s.counters[C_BLOCK_STEPS];
    out->n2v_tests = s.counters[C_PROBES];
    out->algo_bytes = s.counters[C_ALGO_BYTES];
    out->aux_device_bytes = sizeof(Scratch);
    out->last_kernel_ms = 0.0;
    if (G->timed) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, G->ev0, G->ev1) == cudaSuccess) out->last_kernel_ms = ms;
        else cudaGetLastError();
    }
    if (s.counters[C_TIMEOUT])
        return fail(FW_ETIMEOUT, "fw_stats: a walk kernel stopped after a bounded wait ran out (%llu CTAs)",
                    (unsigned long long)s.counters[C_TIMEOUT]);
    if (s.counters[C_BAD_INPUT])
        return fail(FW_EINVAL, "fw_stats: %llu queries had an out-of-range start/prev or negative step0 (written as empty paths)",
                    (unsigned long long)s.counters[C_BAD_INPUT]);
    return FW_OK;
}

extern "C" int fw_stats_reset(fw_graph* G, void* stream) {
    if (!G) return fail(FW_EINVAL, "fw_stats_reset: NULL graph");
    std::lock_guard<std::mutex> lock(G->mu);
    FW_CUDA_TRY(cudaMemsetAsync(G->scratch, 0, sizeof(Scratch), (cudaStream_t)stream));
    G->last_stream = (cudaStream_t)stream;
    return FW_OK;
}

// -------------------------------------------------------- Philox cross-check

namespace {
__global__ void philox_kernel(const uint32_t* __restrict__ in, uint32_t* __restrict__ out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t* a = in + 6 * i;
        const uint4 o = philox4x32_10(make_uint4(a[0], a[1], a[2], a[3]), make_uint2(a[4], a[5]));
        out[4 * i + 0] = o.x;
        out[4 * i + 1] = o.y;
        out[4 * i + 2] = o.z;
        out[4 * i + 3] = o.w;
    }
}
}  // namespace

extern "C" int fw_philox(const uint32_t* in, uint32_t* out, int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!in || !out))) return fail(FW_EINVAL, "fw_philox: bad arguments");
    if (n == 0) return FW_OK;
    if (!is_device_ptr(in) || !is_device_ptr(out)) return fail(FW_EINVAL, "fw_philox: device pointers required");
    const int64_t blocks = (n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096;
    philox_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(in, out, n);
    FW_CUDA_TRY(cudaGetLastError());
    return FW_OK;
}

// ------------------------------------------------------ no-allocation launch
//
// For callers that cannot allocate device memory when they walk: the request
// table and query cursor of the launch live in this one file-scope device
// array instead of freshly allocated memory.  The launch's counts go to the
// graph's own counters (allocated when the graph was loaded), so fw_stats
// reports them, bad starts and timed-out waits included.  Host code may not
// pass the symbol itself to a kernel (in host code it names a host stand-in),
// so its device address is looked up once per device.

namespace {
struct NoAllocScratch {
    Scratch s;                          // s.cursor: reset every call (s.counters unused)
    ReqDev reqs[FW_NOALLOC_MAX_REQS];   // the launch's request table
};
}  // namespace

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

namespace {
std::mutex g_noalloc_mu;
constexpr int kMaxDevices = 64;
NoAllocScratch* g_noalloc_addr[kMaxDevices];  // device address per device, looked up once
ReqDev g_noalloc_host[FW_NOALLOC_MAX_REQS];   // host staging of the table (under the mutex)
}  // namespace

extern "C" int fw_walk_noalloc(fw_graph* G, const fw_request* reqs, int32_t n_req, void* stream) {
    if (!G || !reqs) return fail(FW_EINVAL, "fw_walk_noalloc: NULL argument");
    if (n_req < 1 || n_req > FW_NOALLOC_MAX_REQS)
        return fail(FW_EINVAL, "fw_walk_noalloc: n_req = %d, must be in [1, %d]", n_req, FW_NOALLOC_MAX_REQS);
    if (G->device < 0 || G->device >= kMaxDevices) return fail(FW_EINVAL, "fw_walk_noalloc: device ordinal too large");
    std::lock_guard<std::mutex> glock(G->mu);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    int cur_dev = 0;
    cudaGetDevice(&cur_dev);
    if (cur_dev != G->device) FW_CUDA_TRY(cudaSetDevice(G->device));
    struct DevGuard {
        int d;
        ~DevGuard() { cudaSetDevice(d); }
    } guard{cur_dev};
    NoAllocScratch* dev = g_noalloc_addr[G->device];
    if (!dev) {
        // set-up, once per device, with that device current
        cudaError_t e = cudaGetSymbolAddress((void**)&dev, g_noalloc_scratch);
        if (e != cudaSuccess || !dev)
            return fail(FW_ECUDA, "fw_walk_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_addr[G->device] = dev;
    }
    int64_t total = 0;
    const int mode = reqs[0].params.mode;
    for (int i = 0; i < n_req; ++i) {
        const fw_request& q = reqs[i];
        if (q.params.mode != mode) return fail(FW_EINVAL, "fw_walk_noalloc: requests must share one mode");
        if (q.n_q < 0) return fail(FW_EINVAL, "fw_walk_noalloc: n_q < 0");
        if (q.n_q > 0 && (!q.starts || !q.paths || !q.path_len))
            return fail(FW_EINVAL, "fw_walk_noalloc: NULL starts/paths/path_len");
        const void* ps[] = {q.starts, q.lengths, q.prev, q.step0, q.paths, q.path_len};
        for (const void* pp : ps)
            if (pp && !is_device_ptr(pp)) return fail(FW_EINVAL, "fw_walk_noalloc: buffers must be device memory");
        ReqDev& r = g_noalloc_host[i];
        int rc = make_req(G, q.algo, &q.params, q.max_len, q.seed, &r);
        if (rc != FW_OK) return rc;
        r.starts = q.starts;
        r.lengths = q.lengths;
        r.prev = q.prev;
        r.step0 = q.step0;
        r.paths = q.paths;
        r.path_len = q.path_len;
        r.n_q = q.n_q;
        r.q_begin = total;
        r.q_id0 = q.q_id0;
        total += q.n_q;
    }
    if (total == 0) return FW_OK;
    cudaStream_t st = (cudaStream_t)stream;
    // The table comes from pageable host memory.  Such a copy waits for the
    // work already queued on the stream and has taken the data by the time
    // cudaMemcpyAsync returns, so the staging array may be reused at once.
    FW_CUDA_TRY(cudaMemcpyAsync(dev->reqs, g_noalloc_host, sizeof(ReqDev) * (size_t)n_req,
                                cudaMemcpyHostToDevice, st));
    FW_CUDA_TRY(cudaMemsetAsync(&dev->s.cursor, 0, sizeof(unsigned long long), st));  // starts at zero
    ReqTable tab;
    memset(&tab, 0, sizeof tab);
    tab.ext = dev->reqs;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cap);
    const bool timed = cap == cudaStreamCaptureStatusNone;
    if (timed) FW_CUDA_TRY(cudaEventRecord(G->ev0, st));
    cudaError_t e = launch_walk(G->g, mode, tab, n_req, total, &dev->s.cursor, G->scratch->counters, G->tuning, st);
    if (e != cudaSuccess) return fail(FW_ECUDA, "fw_walk_noalloc: launch: %s", cudaGetErrorString(e));
    if (timed) FW_CUDA_TRY(cudaEventRecord(G->ev1, st));
    G->timed = timed;
    G->last_stream = st;
    return FW_OK;
}
