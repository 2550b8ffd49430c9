// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "fw.h"

namespace fw {

// ---------------------------------------------------------------------------
// Philox-4x32-10 (Salmon et al., SC'11): ten rounds of two 32x32 -> 64 bit
// multiplications whose high halves are xored with the other two counter
// words and the round key; the key advances by the Weyl increments between
// rounds.  Stateless: a block is a pure function of (counter, key), so no
// generator state lives anywhere (the paper keeps cuRAND states in shared
// memory, Section 4.3; a counter-based generator needs none).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
#ifdef __CUDA_ARCH__
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
#else
        const uint32_t hi0 = (uint32_t)(((uint64_t)0xD2511F53u * c.x) >> 32);
        const uint32_t hi1 = (uint32_t)(((uint64_t)0xCD9E8D57u * c.z) >> 32);
#endif
        const uint32_t lo0 = 0xD2511F53u * c.x;
        const uint32_t lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// Per-step block: counter (t, q_lo, q_hi, 0), key (seed_lo, seed_hi).
// Words x|y<<32 give the exact-mode 64-bit draw, word z the PPR stop test.
__host__ __device__ __forceinline__ uint4 step_block(uint64_t seed, uint64_t qid, uint32_t t) {
    return philox4x32_10(make_uint4(t, (uint32_t)qid, (uint32_t)(qid >> 32), 0u),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// Fast-mode reservoir draws: counter word 3 = 0x80000000 | lane << 16 | k.
// `lane` numbers the sampler's lanes over all segments of a row (< 2^15), k
// the lane's draws (< 2^16), so no two streams of one step meet each other or
// the per-step block.
__device__ __forceinline__ uint4 lane_block(uint64_t seed, uint64_t qid, uint32_t t, uint32_t lane,
                                            uint32_t k) {
    return philox4x32_10(make_uint4(t, (uint32_t)qid, (uint32_t)(qid >> 32),
                                    0x80000000u | ((lane & 0x7FFFu) << 16) | (k & 0xFFFFu)),
                         make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ---------------------------------------------------------------------------
// Device-side request: one contiguous range of the launch's query space.
// ---------------------------------------------------------------------------
struct ReqDev {
    const int32_t* starts;
    const int32_t* lengths;
    const int32_t* prev;
    const int32_t* step0;
    int32_t* paths;
    int32_t* path_len;
    int64_t n_q;
    int64_t q_begin;   // first launch-global query index of this request
    int64_t q_id0;     // random-counter id of local query 0
    uint64_t seed;
    int32_t max_len;
    int32_t algo;
    uint32_t fac_i[3]; // exact node2vec factors (ret, in, out)
    float fac_f[3];    // fast node2vec factors
    uint32_t t_stop;   // PPR threshold on Philox word z
    int32_t schema_len;
    int8_t schema[16];
};

// Graph arrays as the kernels see them.
struct GraphDev {
    const int64_t* row_ptr;
    const int32_t* col;
    const float* w_f32;
    const uint32_t* w_u32;
    const int8_t* etype;
    int64_t n;
    int64_t m;
};

// Counter slots in the device scratch (all uint64).
enum CounterSlot {
    C_WALKS = 0,
    C_STEPS,
    C_ROWS,
    C_WARP_STEPS,
    C_BLOCK_STEPS,
    C_PROBES,
    C_ALGO_BYTES,
    C_BAD_INPUT,
    C_TIMEOUT,
    C_NUM
};

// Device scratch of one launch: the query cursor and the counters.
struct Scratch {
    unsigned long long cursor;
    unsigned long long counters[C_NUM];
    unsigned long long pad[16 - 1 - C_NUM];
};
static_assert(sizeof(Scratch) == 128, "scratch layout");

// Requests handed to one launch.  Up to kMaxInlineReqs travel inside the
// kernel's parameter block (so a launch captured in a CUDA graph carries them);
// longer lists live in device memory at `ext`.
constexpr int kMaxInlineReqs = 16;
struct ReqTable {
    const ReqDev* ext;
    ReqDev r[kMaxInlineReqs];
};

// Served form: requests live in a device ring that the host keeps extending
// (by stream-ordered copies) while the kernel runs; the kernel claims
// published queries, and the last walk of a request stamps its completion
// word in host memory.  The host ends a launch by setting `stop` once it has
// been idle for a while: warps then claim nothing new, finish the walks they
// hold and return.
struct ServeDev {
    ReqDev* ring;                                 // device, maxr entries (null: batch launch)
    int maxr;
    unsigned long long* done;                     // device, per ring slot: walks retired
    // device, per ring slot: the query hand-out counter.  Admission sets it
    // to kTakenBase - n_q; a warp claims query k of the slot's request when
    // atomicAdd returns kTakenBase - n_q + k < kTakenBase.  The counter alone
    // decides whether a claim is valid, so a warp holding a stale ring id
    // can never claim from a slot that is being refilled.
    unsigned long long* taken;
    unsigned long long* head;                     // device: oldest ring id that may still hand out queries
    const volatile long long* pub_r;              // device: requests published (written by host copies)
    const volatile int* stop;                     // device: drain and return (written by a host copy)
    volatile unsigned long long* complete;        // mapped host: per ring slot, nonzero when done
};

constexpr unsigned long long kTakenBase = 1ull << 62;

struct Tuning {
    int block_threads;
    int slots;
    int d_warp;
    int ctas_per_sm;
};

// Launch the persistent walk engine over `n_req` requests (device array
// `reqs`) holding `total` queries; the warps claim queries from `cursor`
// (which must be 0 when the launch starts) and add their counts to
// `counters` (C_NUM words).  Defined in fw_walk.cu.
cudaError_t launch_walk(const GraphDev& g, int mode, const ReqTable& reqs, int n_req, int64_t total,
                        unsigned long long* cursor, unsigned long long* counters, const Tuning& tune,
                        cudaStream_t stream);

inline cudaError_t launch_walk(const GraphDev& g, int mode, const ReqTable& reqs, int n_req, int64_t total,
                               Scratch* scratch, const Tuning& tune, cudaStream_t stream) {
    return launch_walk(g, mode, reqs, n_req, total, &scratch->cursor, scratch->counters, tune, stream);
}

// Launch the engine in served mode (runs until stopped or idle).  Defined in
// fw_walk.cu.
cudaError_t launch_serve(const GraphDev& g, int mode, const ServeDev& sv, Scratch* scratch, const Tuning& tune,
                         cudaStream_t stream);

Tuning default_tuning();
Tuning sanitize_tuning(Tuning t);

// Library-internal helpers shared by the ABI translation units (fw_api.cu).
int set_error(int status, const char* msg);                          // records the message, returns status
int graph_device_view(const fw_graph* g, GraphDev* out, int* device, Tuning* tuning);
int make_request(const fw_graph* g, const fw_request& q, ReqDev* out);  // parameters only
Scratch* graph_scratch(const fw_graph* g);                            // the graph's cursor and counters
std::mutex& graph_mutex(fw_graph* g);                                 // serialises launches on the graph

}  // namespace fw
