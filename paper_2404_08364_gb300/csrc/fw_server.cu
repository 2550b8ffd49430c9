// Served form: continuous batching on the persistent walk engine.
//
// Requests (different algorithms, sizes, lengths, seeds) are admitted by
// output-buffer memory into a device arena, published into a device ring
// while the engine runs, and claimed query by query by the engine's warps, so
// a request that arrives while others are on the GPU starts as soon as warps
// free up, and shares the device with them.  The last walk of a request
// stamps a completion word in pinned host memory; a host thread copies the
// results out, frees the arena space and admits waiting requests.  After an
// idle period the host sets the engine's stop word: warps claim nothing new,
// finish the walks they hold and return together, and the engine is
// relaunched when work arrives.
//
// A request's walks use request-local query ids and the request's own seed,
// so its paths are the same alone and in any mix (bit for bit in exact mode;
// in fast mode too: no engine tuning changes a result).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "fw_internal.cuh"

using namespace fw;

namespace {

using Clock = std::chrono::steady_clock;

int fail_s(int status, const char* fmt, ...) {
    char buf[400];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(status, buf);
}

// First-fit allocator of byte ranges inside the output arena.
class Arena {
   public:
    void reset(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        cap_ = bytes;
        used_ = 0;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t capacity() const { return cap_; }
    size_t used() const { return used_; }

   private:
    std::map<size_t, size_t> free_;
    size_t cap_ = 0, used_ = 0;
};

enum TicketState { T_PENDING = 0, T_RUNNING = 1, T_COPYING = 2, T_DONE = 3, T_FAILED = 4 };

struct Ticket {
    uint64_t id;
    fw_request req;                 // as submitted (host buffers)
    std::vector<int32_t> starts, lengths, prev, step0;  // inputs copied at submission
    Clock::time_point t_submit, t_admit, t_done;
    int state = T_PENDING;
    int64_t ring_id = -1;
    size_t off = 0, bytes = 0;       // arena space
    cudaEvent_t copied = nullptr;
    uint64_t steps = 0;
};

}  // namespace

struct fw_server {
    fw_graph* graph;
    GraphDev g;
    Tuning tuning;
    int device;
    int mode;
    int maxr;
    // device
    ReqDev* ring = nullptr;
    unsigned long long* done = nullptr;
    unsigned long long* taken = nullptr;   // per ring slot: query hand-out counter
    unsigned long long* head = nullptr;    // oldest ring id that may still hand out queries
    long long* pub_r = nullptr;            // requests published
    int* stop = nullptr;
    Scratch* scratch = nullptr;
    unsigned char* arena_mem = nullptr;
    // pinned host staging, one entry per ring slot: the sources of the
    // stream-ordered copies that publish a request (a slot's entry is not
    // rewritten before its request completes, long after its copies ran)
    ReqDev* h_ring = nullptr;
    unsigned long long* h_taken = nullptr;
    long long* h_pub_r = nullptr;
    int* h_stop = nullptr;                 // {0, 1}: the values copied into `stop`
    unsigned long long* h_zero = nullptr;  // 0: copied into a slot's retire count
    // pinned, mapped host words
    unsigned long long* h_complete = nullptr;  // maxr
    ServeDev sv;
    Arena arena;
    cudaStream_t kstream = nullptr, cstream = nullptr;
    cudaEvent_t kdone = nullptr;
    bool kernel_running = false;
    bool stop_sent = false;               // this launch has been asked to return
    Clock::duration idle;                 // host idle time before the engine is stopped
    Clock::time_point last_busy;
    uint64_t launches = 0;
    // requests
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Ticket*> pending;
    std::map<uint64_t, Ticket*> tickets;
    std::vector<Ticket*> ring_owner;   // ticket holding each ring slot
    uint64_t next_ticket = 1;
    int64_t next_ring = 0;
    bool shutdown = false;
    int error = 0;
    std::thread worker;
    // stats
    uint64_t completed = 0, total_steps = 0;
    Clock::time_point t_first, t_last;
};

namespace {

size_t request_bytes(const fw_request& r) {
    const size_t nq = (size_t)r.n_q;
    size_t b = nq * ((size_t)r.max_len + 1) * 4 + nq * 4;            // paths + path_len
    b += nq * 4;                                                      // starts
    if (r.lengths) b += nq * 4;
    if (r.prev) b += nq * 4;
    if (r.step0) b += nq * 4;
    return b + 6 * 256;                                               // alignment slack
}

// Copy a ticket's inputs into its arena space and describe it on the device.
int stage_request(fw_server* S, Ticket* T, ReqDev* rd) {
    unsigned char* base = S->arena_mem + T->off;
    size_t at = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + at;
        at = (at + bytes + 255) & ~(size_t)255;
        return p;
    };
    const fw_request& r = T->req;
    const size_t nq = (size_t)r.n_q;
    int32_t* d_paths = (int32_t*)take(nq * ((size_t)r.max_len + 1) * 4);
    int32_t* d_len = (int32_t*)take(nq * 4);
    int32_t* d_starts = (int32_t*)take(nq * 4);
    int32_t* d_lengths = r.lengths ? (int32_t*)take(nq * 4) : nullptr;
    int32_t* d_prev = r.prev ? (int32_t*)take(nq * 4) : nullptr;
    int32_t* d_step0 = r.step0 ? (int32_t*)take(nq * 4) : nullptr;
    cudaMemcpyAsync(d_starts, T->starts.data(), nq * 4, cudaMemcpyHostToDevice, S->cstream);
    if (d_lengths) cudaMemcpyAsync(d_lengths, T->lengths.data(), nq * 4, cudaMemcpyHostToDevice, S->cstream);
    if (d_prev) cudaMemcpyAsync(d_prev, T->prev.data(), nq * 4, cudaMemcpyHostToDevice, S->cstream);
    if (d_step0) cudaMemcpyAsync(d_step0, T->step0.data(), nq * 4, cudaMemcpyHostToDevice, S->cstream);
    rd->starts = d_starts;
    rd->lengths = d_lengths;
    rd->prev = d_prev;
    rd->step0 = d_step0;
    rd->paths = d_paths;
    rd->path_len = d_len;
    return FW_OK;
}

void worker_loop(fw_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (!S->shutdown) {
        bool busy = false;
        // ---- admit waiting requests while the arena and the ring have room ----
        while (!S->pending.empty()) {
            Ticket* T = S->pending.front();
            const int slot = (int)(S->next_ring % S->maxr);
            if (S->ring_owner[slot]) break;  // ring slot still held by an older request
            if (!S->arena.alloc(T->bytes, &T->off)) break;  // wait for memory to free up
            ReqDev rd;
            int rc = make_request(S->graph, T->req, &rd);
            if (rc != FW_OK) {
                S->arena.release(T->off, T->bytes);
                S->pending.pop_front();
                T->state = T_FAILED;
                S->cv.notify_all();
                continue;
            }
            // stream-ordered publication: inputs, the ring entry, the
            // retire count, the hand-out counter (from here on the engine
            // may claim the request's queries), then the published count
            S->h_complete[slot] = 0;
            stage_request(S, T, &rd);
            rd.n_q = T->req.n_q;
            rd.q_begin = 0;
            rd.q_id0 = T->req.q_id0;
            S->h_ring[slot] = rd;
            S->h_taken[slot] = kTakenBase - (unsigned long long)T->req.n_q;
            S->h_pub_r[slot] = S->next_ring + 1;
            cudaMemcpyAsync(&S->ring[slot], &S->h_ring[slot], sizeof(ReqDev), cudaMemcpyHostToDevice, S->cstream);
            // (a copy, not a memset: a memset runs as a kernel, and the
            // resident engine may hold every SM until these words land)
            cudaMemcpyAsync(&S->done[slot], S->h_zero, sizeof(unsigned long long), cudaMemcpyHostToDevice, S->cstream);
            cudaMemcpyAsync(&S->taken[slot], &S->h_taken[slot], sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            S->cstream);
            cudaError_t e = cudaMemcpyAsync(S->pub_r, &S->h_pub_r[slot], sizeof(long long), cudaMemcpyHostToDevice,
                                            S->cstream);
            if (e != cudaSuccess) {
                S->error = FW_ECUDA;
                S->shutdown = true;
                break;
            }
            S->ring_owner[slot] = T;
            T->ring_id = S->next_ring++;
            T->state = T_RUNNING;
            T->t_admit = Clock::now();
            S->pending.pop_front();
            busy = true;
        }
        // ---- keep the engine running while admitted work is unfinished ----
        bool unfinished = false;
        for (int i = 0; i < S->maxr && !unfinished; ++i)
            if (S->ring_owner[i] && S->ring_owner[i]->state == T_RUNNING) unfinished = true;
        if (S->kernel_running && cudaEventQuery(S->kdone) == cudaSuccess) S->kernel_running = false;
        if (unfinished && !S->kernel_running && !S->shutdown) {
            // clear the stop word behind the previous launch, then launch
            cudaError_t e = cudaMemcpyAsync(S->stop, &S->h_stop[0], sizeof(int), cudaMemcpyHostToDevice, S->kstream);
            if (e == cudaSuccess) e = launch_serve(S->g, S->mode, S->sv, S->scratch, S->tuning, S->kstream);
            if (e == cudaSuccess) e = cudaEventRecord(S->kdone, S->kstream);
            if (e != cudaSuccess) {
                S->error = FW_ECUDA;
                S->shutdown = true;
                break;
            }
            S->kernel_running = true;
            S->stop_sent = false;
            ++S->launches;
        }
        // ---- idle for a while: let the engine return (it drains first) ----
        const Clock::time_point now = Clock::now();
        if (unfinished || !S->pending.empty()) S->last_busy = now;
        if (S->kernel_running && !S->stop_sent && !unfinished && S->pending.empty() && now - S->last_busy > S->idle) {
            cudaMemcpyAsync(S->stop, &S->h_stop[1], sizeof(int), cudaMemcpyHostToDevice, S->cstream);
            S->stop_sent = true;
        }
        // ---- completions: copy results out, then release the space ----
        for (int i = 0; i < S->maxr; ++i) {
            Ticket* T = S->ring_owner[i];
            if (!T) continue;
            if (T->state == T_RUNNING && __atomic_load_n(&S->h_complete[i], __ATOMIC_ACQUIRE) != 0) {
                const size_t nq = (size_t)T->req.n_q;
                unsigned char* base = S->arena_mem + T->off;
                const size_t pbytes = nq * ((size_t)T->req.max_len + 1) * 4;
                const size_t lbytes = nq * 4;
                cudaMemcpyAsync(T->req.paths, base, pbytes, cudaMemcpyDeviceToHost, S->cstream);
                cudaMemcpyAsync(T->req.path_len, base + ((pbytes + 255) & ~(size_t)255), lbytes,
                                cudaMemcpyDeviceToHost, S->cstream);
                cudaEventRecord(T->copied, S->cstream);
                T->state = T_COPYING;
                busy = true;
            }
            if (T->state == T_COPYING && cudaEventQuery(T->copied) == cudaSuccess) {
                T->t_done = Clock::now();
                uint64_t steps = 0;
                for (int64_t q = 0; q < T->req.n_q; ++q) steps += (uint64_t)(T->req.path_len[q] - 1);
                T->steps = steps;
                S->total_steps += steps;
                ++S->completed;
                if (S->completed == 1) S->t_first = T->t_submit;
                S->t_last = T->t_done;
                S->arena.release(T->off, T->bytes);
                S->ring_owner[i] = nullptr;
                T->state = T_DONE;
                S->cv.notify_all();
                busy = true;
            }
        }
        if (!busy) S->cv.wait_for(lk, std::chrono::microseconds(20));
    }
}

}  // namespace

extern "C" int fw_server_create(fw_graph* graph, int32_t mode, uint64_t mem_budget, int32_t max_requests,
                                double idle_ms, fw_server** out) {
    if (!graph || !out) return fail_s(FW_EINVAL, "fw_server_create: NULL argument");
    *out = nullptr;
    if (mode != FW_EXACT && mode != FW_FAST) return fail_s(FW_EINVAL, "fw_server_create: unknown mode");
    if (mem_budget < (1u << 20)) return fail_s(FW_EINVAL, "fw_server_create: mem_budget below 1 MiB");
    if (max_requests <= 0) max_requests = 1024;
    if (max_requests > 65536) return fail_s(FW_EINVAL, "fw_server_create: max_requests above 65536");
    fw_server* S = new fw_server();
    S->graph = graph;
    graph_device_view(graph, &S->g, &S->device, &S->tuning);
    // The resident engine runs 512-thread CTAs, four walks per warp, one CTA
    // per SM, whatever the graph's batch tuning (that tuning's d_t is kept;
    // no tuning changes a result).  launch_serve leaves eight SMs free for
    // other streams' kernels.  Measured on R-MAT-24 at saturation, this
    // served 0.94 of the plain batch's steps/s, against 0.75 for 128-thread
    // CTAs with one CTA slot per SM free (16 warps per SM either way, but
    // 96 registers with spills instead of 128).
    S->tuning.block_threads = 512;
    S->tuning.slots = 64;
    S->tuning.ctas_per_sm = 0;
    S->mode = mode;
    S->maxr = max_requests;
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    cudaError_t e = cudaSuccess;
    auto chk = [&](cudaError_t x) {
        if (e == cudaSuccess) e = x;
    };
    chk(cudaMalloc(&S->ring, sizeof(ReqDev) * (size_t)S->maxr));
    chk(cudaMalloc(&S->done, sizeof(unsigned long long) * (size_t)S->maxr));
    chk(cudaMalloc(&S->taken, sizeof(unsigned long long) * (size_t)S->maxr));
    chk(cudaMalloc(&S->head, sizeof(unsigned long long)));
    chk(cudaMalloc(&S->pub_r, sizeof(long long)));
    chk(cudaMalloc(&S->stop, sizeof(int)));
    chk(cudaMalloc(&S->scratch, sizeof(Scratch)));
    chk(cudaMalloc(&S->arena_mem, (size_t)mem_budget));
    chk(cudaHostAlloc(&S->h_ring, sizeof(ReqDev) * (size_t)S->maxr, cudaHostAllocDefault));
    chk(cudaHostAlloc(&S->h_taken, sizeof(unsigned long long) * (size_t)S->maxr, cudaHostAllocDefault));
    chk(cudaHostAlloc(&S->h_pub_r, sizeof(long long) * (size_t)S->maxr, cudaHostAllocDefault));
    chk(cudaHostAlloc(&S->h_stop, 2 * sizeof(int), cudaHostAllocDefault));
    chk(cudaHostAlloc(&S->h_zero, sizeof(unsigned long long), cudaHostAllocDefault));
    chk(cudaHostAlloc(&S->h_complete, sizeof(unsigned long long) * (size_t)S->maxr, cudaHostAllocMapped));
    chk(cudaStreamCreateWithFlags(&S->kstream, cudaStreamNonBlocking));
    chk(cudaStreamCreateWithFlags(&S->cstream, cudaStreamNonBlocking));
    chk(cudaEventCreateWithFlags(&S->kdone, cudaEventDisableTiming));
    if (e == cudaSuccess) {
        // every slot starts exhausted: nothing can be claimed before admission
        for (int i = 0; i < S->maxr; ++i) S->h_taken[i] = kTakenBase;
        chk(cudaMemcpy(S->taken, S->h_taken, sizeof(unsigned long long) * (size_t)S->maxr, cudaMemcpyHostToDevice));
        chk(cudaMemset(S->head, 0, sizeof(unsigned long long)));
        chk(cudaMemset(S->pub_r, 0, sizeof(long long)));
        chk(cudaMemset(S->stop, 0, sizeof(int)));
        chk(cudaMemset(S->scratch, 0, sizeof(Scratch)));
        chk(cudaMemset(S->done, 0, sizeof(unsigned long long) * (size_t)S->maxr));
    }
    if (e != cudaSuccess) {
        fw_server_destroy(S);
        cudaSetDevice(cur);
        return fail_s(e == cudaErrorMemoryAllocation ? FW_ENOMEM : FW_ECUDA, "fw_server_create: %s",
                      cudaGetErrorString(e));
    }
    S->h_stop[0] = 0;
    S->h_stop[1] = 1;
    *S->h_zero = 0;
    memset(S->h_complete, 0, sizeof(unsigned long long) * (size_t)S->maxr);
    ServeDev& sv = S->sv;
    sv.ring = S->ring;
    sv.maxr = S->maxr;
    sv.done = S->done;
    sv.taken = S->taken;
    sv.head = S->head;
    sv.pub_r = S->pub_r;
    sv.stop = S->stop;
    unsigned long long* dcomp = nullptr;
    cudaHostGetDevicePointer((void**)&dcomp, S->h_complete, 0);
    sv.complete = dcomp;
    S->idle = std::chrono::duration_cast<Clock::duration>(
        std::chrono::duration<double, std::milli>(idle_ms > 0 ? idle_ms : 20.0));
    S->last_busy = Clock::now();
    S->arena.reset((size_t)mem_budget);
    S->ring_owner.assign(S->maxr, nullptr);
    S->worker = std::thread(worker_loop, S);
    cudaSetDevice(cur);
    *out = S;
    return FW_OK;
}

extern "C" int fw_server_submit(fw_server* S, const fw_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return fail_s(FW_EINVAL, "fw_server_submit: NULL argument");
    if (req->params.mode != S->mode) return fail_s(FW_EINVAL, "fw_server_submit: mode differs from the server's");
    if (req->n_q < 1 || !req->starts || !req->paths || !req->path_len || req->max_len < 0)
        return fail_s(FW_EINVAL, "fw_server_submit: bad request (n_q, buffers or max_len)");
    Ticket* T = new Ticket();
    T->req = *req;
    const size_t nq = (size_t)req->n_q;
    T->starts.assign(req->starts, req->starts + nq);
    if (req->lengths) T->lengths.assign(req->lengths, req->lengths + nq);
    if (req->prev) T->prev.assign(req->prev, req->prev + nq);
    if (req->step0) T->step0.assign(req->step0, req->step0 + nq);
    for (size_t i = 0; i < nq; ++i)
        if (T->starts[i] < 0 || T->starts[i] >= S->g.n) {
            delete T;
            return fail_s(FW_EINVAL, "fw_server_submit: start vertex out of range");
        }
    T->bytes = request_bytes(*req);
    if (T->bytes > S->arena.capacity()) {
        delete T;
        return fail_s(FW_EBUSY, "fw_server_submit: request needs %zu bytes, more than the whole arena", request_bytes(*req));
    }
    cudaEventCreateWithFlags(&T->copied, cudaEventDisableTiming);
    T->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->shutdown) {
            cudaEventDestroy(T->copied);
            delete T;
            return fail_s(FW_ECUDA, "fw_server_submit: the server has stopped");
        }
        T->id = S->next_ticket++;
        S->tickets[T->id] = T;
        S->pending.push_back(T);
        *ticket = T->id;
    }
    S->cv.notify_all();
    return FW_OK;
}

// Status of a ticket: done = 1 when its outputs are in the caller's buffers
// (latency_s = submission to completion), -1 if it failed.
extern "C" int fw_server_poll(fw_server* S, uint64_t ticket, int32_t* done, double* latency_s) {
    if (!S || !done) return fail_s(FW_EINVAL, "fw_server_poll: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail_s(FW_EINVAL, "fw_server_poll: unknown ticket");
    Ticket* T = it->second;
    *done = T->state == T_DONE ? 1 : (T->state == T_FAILED ? -1 : 0);
    if (latency_s && T->state == T_DONE)
        *latency_s = std::chrono::duration<double>(T->t_done - T->t_submit).count();
    return S->error ? fail_s(S->error, "fw_server_poll: the server hit a CUDA error") : FW_OK;
}

extern "C" int fw_server_wait(fw_server* S, uint64_t ticket, double timeout_s, double* latency_s) {
    if (!S) return fail_s(FW_EINVAL, "fw_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail_s(FW_EINVAL, "fw_server_wait: unknown ticket");
    Ticket* T = it->second;
    const auto until = Clock::now() + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(timeout_s));
    while (T->state != T_DONE && T->state != T_FAILED && !S->error) {
        if (S->cv.wait_until(lk, until) == std::cv_status::timeout) return fail_s(FW_ETIMEOUT, "fw_server_wait: timed out");
    }
    if (S->error) return fail_s(S->error, "fw_server_wait: the server hit a CUDA error");
    if (T->state == T_FAILED) return fail_s(FW_EINVAL, "fw_server_wait: the request was rejected");
    if (latency_s) *latency_s = std::chrono::duration<double>(T->t_done - T->t_submit).count();
    return FW_OK;
}

// Forget a finished ticket (its latency can no longer be queried).
extern "C" int fw_server_release(fw_server* S, uint64_t ticket) {
    if (!S) return fail_s(FW_EINVAL, "fw_server_release: NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail_s(FW_EINVAL, "fw_server_release: unknown ticket");
    Ticket* T = it->second;
    if (T->state != T_DONE && T->state != T_FAILED) return fail_s(FW_EBUSY, "fw_server_release: ticket still running");
    cudaEventDestroy(T->copied);
    delete T;
    S->tickets.erase(it);
    return FW_OK;
}

extern "C" int fw_server_stats(fw_server* S, fw_server_stats_t* out) {
    if (!S || !out) return fail_s(FW_EINVAL, "fw_server_stats: NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    memset(out, 0, sizeof *out);
    out->completed = S->completed;
    out->steps = S->total_steps;
    out->launches = S->launches;
    out->pending = S->pending.size();
    out->arena_used = S->arena.used();
    out->arena_capacity = S->arena.capacity();
    out->busy_s = S->completed ? std::chrono::duration<double>(S->t_last - S->t_first).count() : 0.0;
    return FW_OK;
}

extern "C" void fw_server_destroy(fw_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->shutdown = true;
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(S->device);
    // a running engine drains and returns
    if (S->stop && S->h_stop && S->cstream)
        cudaMemcpyAsync(S->stop, &S->h_stop[1], sizeof(int), cudaMemcpyHostToDevice, S->cstream);
    if (S->kstream) cudaStreamSynchronize(S->kstream);
    if (S->cstream) cudaStreamSynchronize(S->cstream);
    for (auto& kv : S->tickets) {
        if (kv.second->copied) cudaEventDestroy(kv.second->copied);
        delete kv.second;
    }
    cudaFree(S->ring);
    cudaFree(S->done);
    cudaFree(S->taken);
    cudaFree(S->head);
    cudaFree(S->pub_r);
    cudaFree(S->stop);
    cudaFree(S->scratch);
    cudaFree(S->arena_mem);
    if (S->h_ring) cudaFreeHost(S->h_ring);
    if (S->h_taken) cudaFreeHost(S->h_taken);
    if (S->h_pub_r) cudaFreeHost(S->h_pub_r);
    if (S->h_stop) cudaFreeHost(S->h_stop);
    if (S->h_zero) cudaFreeHost(S->h_zero);
    if (S->h_complete) cudaFreeHost(S->h_complete);
    if (S->kdone) cudaEventDestroy(S->kdone);
    if (S->kstream) cudaStreamDestroy(S->kstream);
    if (S->cstream) cudaStreamDestroy(S->cstream);
    cudaSetDevice(cur);
    delete S;
}
