/*
 * fw.h — C ABI of the GB300 dynamic-graph random-walk library.
 *
 * The library implements the per-step hot path of FlowWalker (arXiv
 * 2404.08364): at every step of every walk query it computes the
 * state-dependent weight of each neighbour of the current vertex
 * (Alg. 1's initialisation phase: weighted, MetaPath Eq. 1, node2vec Eq. 2,
 * PPR) and draws one neighbour (the selection phase) without any per-vertex
 * preprocessing buffer in global memory (Section 5.3, "Memory Consumption").
 *
 * Conventions for every call:
 *   - Return value: FW_OK (0) or a negative fw_status; no exceptions cross
 *     the ABI.  fw_strerror() names a status; fw_last_error() gives a
 *     one-line message for the calling thread's last failure.
 *   - The caller owns every input and output buffer; the library owns its
 *     copy of the graph (unless FW_BORROW) and a few bytes of device state
 *     per graph (query cursor and counters).
 *   - Device work is enqueued on the caller's CUDA stream (cudaStream_t
 *     passed as void*, NULL = legacy default stream) and returns before it
 *     finishes; an asynchronous device error surfaces at the next
 *     synchronising call (fw_stats, fw_sync) as FW_ECUDA.
 *   - Vertex ids are int32; row offsets int64.  One graph, one device: the
 *     device current at fw_load_csr is used for every later call on it.
 *   - Calls on the same graph must be ordered on one stream (they share the
 *     graph's query cursor); different graphs are independent.
 */
#ifndef FW_H_
#define FW_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FW_OK = 0,
    FW_EINVAL = -1,     /* bad argument (null pointer, size, range, params) */
    FW_ENOMEM = -2,     /* device or host allocation failed */
    FW_ECUDA = -3,      /* a CUDA call or a kernel failed */
    FW_EUNSORTED = -4,  /* a CSR row is not strictly ascending */
    FW_ETIMEOUT = -5,   /* a bounded device wait ran out (a copy or a hub task never completed) */
    FW_EBUSY = -6       /* resource in use (served form: no admission room) */
} fw_status;

/* Weight rule of a walk (Section 2.1). */
typedef enum {
    FW_WEIGHTED = 0,  /* p(u) ∝ w(v,u): DeepWalk-style first-order walk */
    FW_NODE2VEC = 1,  /* Eq. 2 weighted: w(v,u) × {1/p, 1, 1/q} by dist(v',u) */
    FW_METAPATH = 2,  /* Eq. 1 weighted: w(v,u) × [l(v,u) = schema[t mod len]] */
    FW_PPR = 3        /* weighted step, then stop with probability ppr_stop */
} fw_algo;

/* Sampling mode. */
typedef enum {
    FW_EXACT = 0,  /* integer weights (w_u32) and integer node2vec factors; one
                      Philox-4x32-10 block per (seed, query, step) and an exact
                      inverse-transform pick: bit-identical to the CPU oracle */
    FW_FAST = 1    /* FP32 weights (w_f32); single-pass weighted reservoir
                      sampling (exponential race with exponential jumps).  A
                      row is cut into segments of 16384 entries (counted from
                      its first 16-entry-aligned group; more per segment past
                      64 segments), segment j draws from random stream j and
                      the smallest race time wins, whichever sampler scans the
                      row: fast-mode paths do not depend on fw_tuning */
} fw_mode;

/* fw_load_csr flags */
#define FW_HOST_PTRS 0u     /* inputs are host pointers; the library copies */
#define FW_DEVICE_PTRS 1u   /* inputs are device pointers; the library copies */
#define FW_BORROW 2u        /* inputs are device pointers the caller keeps alive
                               until fw_free; nothing is copied.  Each must be
                               16-byte aligned. */
#define FW_NO_VALIDATE 4u   /* accept unsorted rows and invalid weights (results
                               are then undefined, but every access stays in
                               bounds); offsets and column ranges are always
                               checked, since the kernels index by them */

typedef struct fw_graph fw_graph;

/*
 * Walk parameters.
 *   mode            FW_EXACT or FW_FAST.
 *   n2v_p, n2v_q    node2vec return (paper's a) and in-out (paper's b)
 *                   parameters of Eq. 2.  Fast mode uses the factors 1/p, 1,
 *                   1/q in FP32.  Exact mode uses the integers S/p, S, S/q
 *                   with S = n2v_scale (must all be positive integers in
 *                   [1, 65536], else FW_EINVAL); p = 2, q = 0.5, S = 2 gives
 *                   1, 2, 4.  Exact mode multiplies weight by factor in 32
 *                   bits, so max(w_u32) × the largest factor must stay below
 *                   2^32, else the walk call returns FW_EINVAL.
 *   schema          MetaPath labels, schema[t mod schema_len] is required
 *                   at move t (0-based); schema_len in [1, 16].
 *   ppr_stop        PPR stop probability in [0, 1]; the walk stops after a
 *                   move when word 2 of the step's Philox block is below
 *                   floor(ppr_stop · 2^32).
 */
typedef struct {
    int32_t mode;
    float n2v_p, n2v_q;
    int32_t n2v_scale;
    int32_t schema_len;
    int8_t schema[16];
    double ppr_stop;
} fw_params;

/*
 * Engine tuning (Section 5.1's |P_L| and d_t and the launch shape).
 *   block_threads   threads per CTA: 128, 256 or 512 (anything else: the
 *                   default, 512).
 *   slots           walks resident per CTA: the local task pool P_L, at most
 *                   8 per warp (default 4 per warp).
 *   d_warp          degree threshold d_t: rows with d <= d_warp are sampled
 *                   by one warp, larger rows by the whole CTA (default 65536;
 *                   exact mode caps it at 8184).
 *   ctas_per_sm     persistent CTAs per SM (0 = as many as fit).
 * Zero fields mean "default".  No field changes a walk's result: exact mode is
 * bit-identical to the CPU oracle under every tuning, and fast mode draws each
 * row with the same segment streams whichever sampler takes it.
 */
typedef struct {
    int32_t block_threads;
    int32_t slots;
    int32_t d_warp;
    int32_t ctas_per_sm;
} fw_tuning;

/* Device counters accumulated since the last fw_stats_reset. */
typedef struct {
    uint64_t walks;          /* queries finished */
    uint64_t steps;          /* moves made (sum over queries of path_len - 1) */
    uint64_t rows_scanned;   /* sum over moves of d(cur): neighbour entries read */
    uint64_t warp_steps;     /* moves sampled by a warp sampler */
    uint64_t block_steps;    /* moves sampled by a CTA sampler */
    uint64_t n2v_tests;      /* node2vec membership tests against N(prev) */
    uint64_t algo_bytes;     /* algorithmic bytes: per move 8·d (+1·d labels)
                                + 16 (row offsets) + 4 (path write) */
    uint64_t aux_device_bytes; /* device memory the library holds beyond the
                                  graph copy and caller buffers */
    double last_kernel_ms;   /* duration of the last walk launch (events) */
} fw_stats_t;

/*
 * Load a CSR graph (Section 2.1: G = (V, E) with w(u,v), l(u,v)).
 *   n, m        vertex and entry counts (n >= 1, m >= 0, n < 2^31).
 *   row_ptr     int64[n+1], row_ptr[0] = 0, non-decreasing, row_ptr[n] = m.
 *   col         int32[m], each row strictly ascending (sorted, no duplicates:
 *               node2vec's dist(v',u) = 1 test is a search in the sorted row).
 *   w_f32       float[m] weights for FW_FAST (finite, > 0), or NULL.
 *   w_u32       uint32[m] weights for FW_EXACT (> 0), or NULL.
 *   etype       int8[m] edge labels for FW_METAPATH, or NULL.
 *   flags       FW_HOST_PTRS / FW_DEVICE_PTRS / FW_BORROW, | FW_NO_VALIDATE.
 * Errors: FW_EINVAL (sizes, null row_ptr/col, bad offsets, column out of
 * range, non-positive or non-finite weight), FW_EUNSORTED (a row not strictly
 * ascending), FW_ENOMEM, FW_ECUDA.  On error *g is NULL and nothing is held.
 */
int fw_load_csr(fw_graph** g, int64_t n, int64_t m, const int64_t* row_ptr, const int32_t* col,
                const float* w_f32, const uint32_t* w_u32, const int8_t* etype, uint32_t flags);

/* Release the graph and every device buffer the library holds for it. */
void fw_free(fw_graph* g);

/*
 * Run n_q walk queries (Alg. 1) on the graph; enqueued on `stream`.
 *   algo, p      weight rule and parameters (see above).
 *   starts       int32[n_q] start vertices.
 *   lengths      int32[n_q] per-query move limits, or NULL (all max_len).
 *   max_len      maximum moves; each output row holds max_len + 1 vertices.
 *   seed         64-bit Philox key.  Query i uses query id q_id0 + i in the
 *                random-number counter (see fw_walk_ex), so a query's path
 *                depends only on (graph, algo, params, seed, its id, its
 *                start state) and not on batching or on the device tuning.
 *   prev, step0  int32[n_q] or NULL: resume a walk whose previous vertex is
 *                prev[i] (-1 = none) at move index step0[i]; the walk then
 *                makes moves step0[i] .. limit-1.
 *   paths        int32[n_q × (max_len+1)] output, row i = start vertex then
 *                one vertex per move, padded with -1 (Section 5.2's result
 *                pool, Eq. 3's L_max + 1 entries per query).
 *   path_len     int32[n_q] output: vertices written (moves + 1).
 * Pointers may be device or host memory (each is classified separately);
 * host buffers are staged through device memory, and then the call returns
 * only when the outputs are back on the host.
 * Errors: FW_EINVAL (null, n_q < 0, max_len < 0, start or prev out of range,
 * params, algo needs a missing array), FW_ENOMEM, FW_ECUDA.
 */
int fw_walk(fw_graph* g, int32_t algo, const fw_params* p, const int32_t* starts, int64_t n_q,
            const int32_t* lengths, int32_t max_len, uint64_t seed, const int32_t* prev,
            const int32_t* step0, int32_t* paths, int32_t* path_len, void* stream);

/* One walk request inside a multi-request launch (fw_walk_multi). */
typedef struct {
    int32_t algo;
    fw_params params;
    const int32_t* starts;
    int64_t n_q;
    const int32_t* lengths;
    int32_t max_len;
    uint64_t seed;
    int64_t q_id0;           /* query id of starts[0] in the random counter */
    const int32_t* prev;
    const int32_t* step0;
    int32_t* paths;
    int32_t* path_len;
} fw_request;

/*
 * Run several requests (different algorithms, parameters, lengths, seeds) in
 * ONE persistent launch: the CTAs claim queries from all requests through one
 * cursor, so short and long walks (PPR's geometric lengths next to fixed-length
 * MetaPath) share the GPU without a batch barrier.  All requests must use the
 * same mode.  Device pointers only.  Errors as fw_walk.
 */
int fw_walk_multi(fw_graph* g, const fw_request* reqs, int32_t n_req, void* stream);

/*
 * fw_walk_noalloc — the multi-request launch of fw_walk_multi for callers
 * that must not allocate device memory at call time: code that runs while a
 * latency-critical server loop holds the device (a cudaMalloc there can
 * synchronise the whole device), callers whose allocator owns all device
 * memory, and callers in environments that forbid runtime allocation.  The
 * paper has no counterpart; this is a deployment convenience.
 *
 *   g, reqs, n_req, stream   as fw_walk_multi; every buffer is device memory
 *                            the caller owns; 1 <= n_req <= FW_NOALLOC_MAX_REQS.
 * Scratch: the request table and the query cursor of the launch live in one
 * static device array compiled into the library (about FW_NOALLOC_MAX_REQS ×
 * 168 bytes + 128 bytes), which every GPU that loads the library holds until
 * the process exits.  Nothing is allocated: no cudaMalloc, no cudaFree, no
 * host heap.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current: make that first call
 * before any stream capture.  The array is shared by all calls and keeps the
 * last call's contents; each call resets the cursor it uses.  Two calls whose
 * launches overlap on the GPU (different streams, no ordering between them)
 * race on the array: order them on one stream.
 * The request table is copied from pageable host memory, and such a copy
 * waits for the work already queued on `stream`: the call returns only after
 * the stream's earlier work has finished (the walk itself is then queued and
 * runs asynchronously).
 * The launch adds its counts to the graph's counters, which the graph holds
 * from fw_load_csr on: fw_stats reports them like those of fw_walk, and
 * returns FW_EINVAL when a start or prev was out of range (written as an
 * empty path) and FW_ETIMEOUT when a bounded device wait ran out.
 * Errors: FW_EINVAL (n_req outside [1, FW_NOALLOC_MAX_REQS], host buffers,
 * bad parameters), FW_ECUDA.
 */
#define FW_NOALLOC_MAX_REQS 1024
int fw_walk_noalloc(fw_graph* g, const fw_request* reqs, int32_t n_req, void* stream);

/*
 * fw_walk_batched — walks whose results exceed device memory (Section 5.2,
 * Fig. 8 and Eq. 3).  The n_q queries are cut into batches of
 *     |P_G| = floor(budget_bytes / (2 * (max_len + 3) * 4))
 * queries: Eq. 3 with budget_bytes standing for M - M_G, its (L_max + 1)
 * result words per query plus each query's start and path length.  Batches
 * alternate between two streams, each with its own result pool, query cursor
 * and counters, so one batch's paths are copied to the host while the next
 * batch walks.  budget_bytes = 0 takes the free device memory less 256 MiB.
 *   h_starts [n_q], h_lengths [n_q] or NULL, h_paths [n_q][max_len + 1],
 *   h_path_len [n_q]: host memory (pinned memory lets the copies overlap the
 *   walks; pageable memory works without overlap).  Output layout, padding
 *   and random counters (q_id0 + query index) are those of fw_walk_ex, so the
 *   paths equal one launch over all queries.
 *   batch_q (may be NULL) receives |P_G| as used (at most n_q).
 * Synchronous; the work is added to the graph's counters (fw_stats).
 * Errors: FW_EINVAL (arguments, parameters; or, after the run, starts out of
 * range, whose paths are written empty), FW_ENOMEM (the budget does not hold
 * one query in each pool, or an allocation failed), FW_ECUDA, FW_ETIMEOUT (a
 * device wait gave up).
 */
int fw_walk_batched(fw_graph* g, int32_t algo, const fw_params* p, const int32_t* h_starts, int64_t n_q,
                    const int32_t* h_lengths, int32_t max_len, uint64_t seed, int64_t q_id0,
                    uint64_t budget_bytes, int32_t* h_paths, int32_t* h_path_len, int64_t* batch_q);

/* Eq. 3's batch size for a byte budget (host arithmetic only; no GPU needed). */
int64_t fw_batch_size(uint64_t budget_bytes, int32_t max_len);

/*
 * fw_sampler_run — the parallel weighted samplers side by side (Section 4):
 *   method 0  the engine's exponential-jump reservoir (its fast mode),
 *   method 1  DPRS, direct parallel reservoir sampling (Alg. 3),
 *   method 2  ZPRS, zig-zag parallel reservoir sampling (Alg. 4),
 * each run by a group of `width` threads (32: a warp; 256: a CTA).  `reps`
 * independent draws from the same weights d_w [n] (device, n in [1, 2^31),
 * weights >= 0) run at once, one per group; d_out [reps] (device) receives the
 * drawn indices (-1 if every weight is 0).  Draw r uses random counters of
 * its own (seed, r), so the draws are independent, each with law
 * w_i / sum(w).  If ms is not NULL the call waits and stores the launch time
 * (CUDA events on `stream`).  Errors: FW_EINVAL (arguments), FW_ECUDA.
 */
int fw_sampler_run(int32_t method, int32_t width, const float* d_w, int64_t n, int64_t reps, uint64_t seed,
                   int32_t* d_out, void* stream, float* ms);

/* Same as fw_walk with an explicit query-id offset q_id0 (for sharding one
 * query range over several calls or devices with identical results). */
int fw_walk_ex(fw_graph* g, int32_t algo, const fw_params* p, const int32_t* starts, int64_t n_q,
               const int32_t* lengths, int32_t max_len, uint64_t seed, int64_t q_id0,
               const int32_t* prev, const int32_t* step0, int32_t* paths, int32_t* path_len,
               void* stream);

/*
 * Served form: continuous batching on a resident graph.
 *
 * A server owns a device output arena of mem_budget bytes and a ring of up to
 * max_requests live requests.  fw_server_submit copies a request's inputs
 * (host starts / lengths / prev / step0) and queues it; a server thread
 * admits queued requests in arrival order as soon as the arena has room for
 * their outputs (admission by output-buffer memory) and publishes them to the
 * running engine, whose warps pick them up between steps of the walks already
 * on the GPU (no batch barrier).  When a request's last walk ends its paths
 * and path_len are copied to the request's HOST buffers (paths, path_len,
 * which must stay valid until then) and its arena space is freed.
 *   mode         FW_EXACT or FW_FAST for every request of this server.
 *   idle_ms      the engine returns after this long without work and is
 *                relaunched when work arrives (<= 0: 20 ms).
 * A request's random counters use its own seed and its own query ids
 * (q_id0 + i), so its paths equal those of the same request run alone, bit
 * for bit in both modes (no engine tuning changes a result).
 * The engine's warps also return by themselves after 2 s without work (a
 * bounded device wait); the server then relaunches the engine for the next
 * request.
 * Latency = submission to outputs in the caller's buffers.
 * Errors: FW_EINVAL (arguments, mode mismatch, start out of range), FW_EBUSY
 * (a request larger than the whole arena), FW_ETIMEOUT (wait), FW_ENOMEM,
 * FW_ECUDA.
 */
typedef struct fw_server fw_server;

typedef struct {
    uint64_t completed;      /* requests finished */
    uint64_t steps;          /* moves of the finished requests */
    uint64_t launches;       /* engine launches (relaunches after idle) */
    uint64_t pending;        /* requests waiting for admission */
    uint64_t arena_used;     /* bytes of the output arena in use */
    uint64_t arena_capacity;
    double busy_s;           /* first submission to last completion */
} fw_server_stats_t;

int fw_server_create(fw_graph* g, int32_t mode, uint64_t mem_budget, int32_t max_requests, double idle_ms,
                     fw_server** out);
int fw_server_submit(fw_server* s, const fw_request* req, uint64_t* ticket);
int fw_server_poll(fw_server* s, uint64_t ticket, int32_t* done, double* latency_s);
int fw_server_wait(fw_server* s, uint64_t ticket, double timeout_s, double* latency_s);
int fw_server_release(fw_server* s, uint64_t ticket);
int fw_server_stats(fw_server* s, fw_server_stats_t* out);
void fw_server_destroy(fw_server* s);

/*
 * CUDA-graph form of a multi-request launch: fw_capture_multi records the
 * cursor reset and the persistent engine launch of fw_walk_multi(reqs) into
 * a CUDA graph; fw_exec_launch replays it on `stream` (the same buffers: the
 * caller may rewrite starts, lengths, prev and step0 in place between
 * replays).  Device buffers only; errors as fw_walk_multi, FW_ECUDA.
 */
typedef struct fw_exec fw_exec;
int fw_capture_multi(fw_graph* g, const fw_request* reqs, int32_t n_req, fw_exec** out);
int fw_exec_launch(fw_exec* x, void* stream);
void fw_exec_destroy(fw_exec* x);

/*
 * Engine autotuner (Section 5.1's |P_L| and d_t, and the CTA size): runs
 * fw_walk_multi(reqs) — a representative sample of the workload, device
 * buffers — over a grid of tunings (128/256/512 threads, d_t 2^11 .. 2^20,
 * 1..4 walk slots per warp), `reps` timed launches each, keeps the fastest in
 * walk steps per second, sets it on g and returns it in *best (and its rate in
 * *best_steps_per_s when not NULL).  The choice is cached by (GPU name,
 * algorithms and mode of the sample, log2 mean and max degree of g); a cache
 * hit returns at once with rate 0.  1 <= n_req <= 16.
 */
int fw_autotune(fw_graph* g, const fw_request* reqs, int32_t n_req, int32_t reps, fw_tuning* best,
                double* best_steps_per_s);
int fw_autotune_clear_cache(void);

/* Set / get the engine tuning used by later walks on g (NULL = defaults). */
int fw_set_tuning(fw_graph* g, const fw_tuning* t);
int fw_get_tuning(const fw_graph* g, fw_tuning* out);

/* Synchronise the graph's last stream and copy the counters to *out. */
int fw_stats(fw_graph* g, fw_stats_t* out);
int fw_stats_reset(fw_graph* g, void* stream);

/* Wait for all work enqueued by the library on `stream`; FW_ECUDA on a
 * device error. */
int fw_sync(void* stream);

/* Graph facts: n, m, max degree, and which weight/label arrays are present. */
int fw_graph_info(const fw_graph* g, int64_t* n, int64_t* m, int64_t* d_max, int32_t* has_f32,
                  int32_t* has_u32, int32_t* has_type);

/*
 * Philox-4x32-10 blocks from the device generator the walk kernels use, for
 * cross-checking it against other implementations (Salmon et al., SC'11).
 *   in   device uint32[n × 6]: ctr0 ctr1 ctr2 ctr3 key0 key1 per block.
 *   out  device uint32[n × 4].
 * Enqueued on `stream`.  Errors: FW_EINVAL (n < 0, NULL, host pointers).
 */
int fw_philox(const uint32_t* in, uint32_t* out, int64_t n, void* stream);

const char* fw_strerror(int status);
const char* fw_last_error(void);

/* Library version as (major << 16) | minor. */
int fw_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FW_H_ */
