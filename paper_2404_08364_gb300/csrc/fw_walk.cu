// Persistent, degree-aware walk engine (FlowWalker Sections 4-5, re-designed
// for sm_103a without block-wide barriers).
//
// Scheduling (Section 5's sampler-centric model and two-level task pools):
//   * Every warp is an independent sampler with a few walk slots of its own
//     in shared memory (its share of the CTA's local task pool P_L).  It
//     claims queries from one global atomic cursor over the callers' request
//     arrays (the global task pool P_G: nothing extra in global memory) and
//     runs one step at a time on whichever of its walks is ready.
//   * A step whose current row holds at most d_t entries is sampled by the
//     warp alone (the warp sampler).  A longer row becomes a CTA hub task:
//     it is cut into segments and every warp of the CTA that has a free
//     moment takes segments through shared-memory atomics (the block
//     sampler, without __syncthreads: warps join and leave freely).  The
//     warp that finishes the last segment merges the result and commits the
//     move; the walk then returns to its owner warp.  So a walk moves between
//     the warp and the block sampler at every step, by the degree of the
//     vertex it stands on, and never leaves its CTA.
//
// Samplers (Section 4's selection phase; no O(d) buffer in global memory):
//   exact mode: W = sum of integer weights, r = floor(x * W / 2^64) from the
//     step's 64-bit Philox draw, pick = smallest i with inclusive prefix > r
//     (inverse transform sampling, two passes: the first keeps one sum per
//     128-entry chunk or per segment in shared memory, the second re-reads
//     only the chunk or segment holding the crossing);
//   fast mode: one pass of weighted reservoir sampling in exponential-race
//     form: the warp keeps one Efraimidis-Spirakis reservoir with
//     exponential jumps per row segment (a warp sum per 256-entry stage
//     against the remaining jump budget; random draws only where a record
//     falls, about ln d per row), and segments are merged by an arg-min over
//     race times (a 64-bit atomicMin of packed (time, index) across the
//     warps of a hub task).
//
// Rows are streamed in 256-entry stages (columns, weights and labels) by TMA
// bulk copies into a two-stage shared-memory ring per warp, the next stage's
// copy in flight while the current one is sampled; a lane reads two aligned
// 16-byte quads per stage.
#include <math.h>
#include <string.h>

#include <type_traits>

#include "fw_internal.cuh"

namespace fw {
namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int INT_BIG = 0x7fffffff;
constexpr int MODE_EXACT = 0, MODE_FAST = 1;
constexpr int WIN = 136;          // node2vec: window of N(prev) (exact re-scans, 128) or 128 padded splitters
constexpr int NSPL = 128;         // node2vec: splitters of a dense window
constexpr int SW_MAX = 8;         // walk slots per warp, upper bound
constexpr int NHUB = 4;           // hub tasks open at once per CTA
constexpr int NSEG_MAX = 64;      // segments per hub task
// A row is cut into segments of kSegQuads quads (16384 entries, counted from
// its first aligned 16-entry group), or more for rows past NSEG_MAX such
// segments.  In fast mode segment j draws from random stream j and the step
// takes the smallest race time over the segments, whichever sampler (a warp
// alone, or a CTA hub task) scans the row: the pick depends on the row, not
// on the threshold d_t or the launch shape.
constexpr int kSegQuads = 4096;
constexpr int NCHUNK_MAX = 64;    // exact warp sampler: chunk sums (d_t <= 8192)
constexpr int NST = 2;            // TMA ring stages per warp (the next stage lands while one is read)
// node2vec: a stage whose range, at the density of N(prev)'s loaded block,
// would hold more than kDenseBlocks further blocks of N(prev) looks for the
// end of its window; a window of more than kDenseMin entries is searched from
// the stage entries' side.
constexpr float kDenseBlocks = 3.0f;
constexpr int kDenseMin = 256;
constexpr int CHQ = 32;           // quads per chunk (one per lane)
constexpr int SQ = 2 * CHQ;       // quads per stage: two chunks, lane l holds quads l and l + 32
constexpr int ST_COL = 0, ST_W = SQ * 16, ST_ET = SQ * 32;
constexpr int STAGE_BYTES = SQ * 36;  // columns, weights, labels of one stage
constexpr int ST_EMPTY = 0, ST_READY = 1, ST_HUB = 2, ST_FINISH = 3;
// hub task control word: state << 24 | next segment to hand out
constexpr int H_FREE = 0, H_SETUP = 1, H_ACTIVE = 2;
constexpr unsigned H_SEG_MASK = 0xFFFFFFu;

// Per-step view of one walk, held in registers by the lanes of its sampler.
struct StepCtx {
    long long beg;
    long long pbeg;
    int d;
    int pdeg;
    int prev;
    int algo;
    int want;   // MetaPath label for this move
    uint32_t fi0, fi1, fi2;
    float ff0, ff1, ff2;
};

// A CTA hub task: one step of one walk whose row is longer than d_t.
struct HubTask {
    unsigned ctl;     // state << 24 | next_seg; one atomic both claims a
                      // segment and tells whether the task was live
    int slot;         // owner slot (warp * SW_MAX + j)
    int nseg;
    int seg_q;        // quads per segment
    int done_seg;
    unsigned long long best;  // fast: (race-time bits << 32) | row index
    StepCtx c;
    uint64_t seed;
    uint64_t qid;
    uint32_t t;
    unsigned long long seg_sum[NSEG_MAX];  // exact
};

template <int NT>
struct __align__(16) Smem {
    static constexpr int NS = (NT / 32) * SW_MAX;
    ReqDev rq[NS];        // each walk's request, copied in when the walk starts
    long long q[NS];      // local query index inside its request
    long long pbeg[NS];   // row of prev (node2vec)
    int req[NS];
    int cur[NS], prev[NS], t[NS], lim[NS], k[NS], pdeg[NS];
    int state[NS];
    HubTask hub[NHUB];
    unsigned long long cnt[NT / 32][C_NUM];
    int abort_flag;
};

// ------------------------------------------------------------ small helpers

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long n = __shfl_up_sync(FULL, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

__device__ __forceinline__ float unit_open(uint32_t w) {
    // strictly inside (0, 1): 23 random bits centred in their cell, so the
    // largest value is 1 - 2^-24 (exact in FP32) and -log(u) > 0 always
    return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // bounded waits: 2 s

// ------------------------------------------------- TMA bulk copies, mbarriers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(20000u)  // let the thread sleep up to 20 us for the phase
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier; false after kWaitLimitNs (a copy
// that never lands means a bug: the caller then stops cleanly).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > kWaitLimitNs) return false;
    }
}

// 1-D bulk copy global -> shared, completion counted in bytes on `bar`.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// A warp's private ring of NST stage buffers in shared memory, each with its
// mbarrier.  A stage holds SQ quads (256 entries).  Stages go through the
// ring in order; (st, ph) = stage of the next one to consume and the barrier
// phase parity it completes there.  A stage that would read past the end of
// the CSR arrays is not copied (its barrier is just arrived on) and its
// quads are read from global memory instead: stage_direct() says which.
struct WarpPipe {
    unsigned char* buf;
    unsigned long long* bar;
    unsigned* mask;  // node2vec membership of the current stage: one byte per entry (64 words)
    int st;
    uint32_t ph;
};

__device__ __forceinline__ void ring_next(int& st, uint32_t& ph) {
    if (++st == NST) {
        st = 0;
        ph ^= 1u;
    }
}

// --------------------------------------------------------------------------
// node2vec membership: is a neighbour u of cur also in N(prev)?  Both rows are
// sorted, so the entries of one 128-entry chunk of N(cur) can only match the
// contiguous window of N(prev) between the chunk's smallest and largest
// value.  A warp keeps one cursor into N(prev) that only moves forward (the
// chunks ascend), finds each window with ballots over coalesced 32-entry
// blocks (a 32-ary search when it has to skip far), stages it in shared
// memory and lets every lane search its own four entries there.  N(prev) is
// read about once (its part that overlaps N(cur)), instead of a log2 d(prev)
// probe chain per neighbour.
// --------------------------------------------------------------------------

// First index i >= pos with B[i] >= x, or pd.  Warp-collective, uniform result.
__device__ __forceinline__ int lower_bound_from(const int32_t* __restrict__ B, int pd, int pos, int x, int lane) {
    {
        const int idx = pos + lane;
        const int v = idx < pd ? __ldg(B + idx) : INT_BIG;
        const unsigned m = __ballot_sync(FULL, v < x);
        if (m != FULL) return pos + __popc(m);
    }
    int lo = pos + 32, hi = pd;  // the answer lies in [lo, hi]
    while (hi - lo > 32) {
        const int s = (hi - lo + 31) >> 5;
        const long long idx = (long long)lo + (long long)s * (lane + 1) - 1;
        const int v = idx < hi ? __ldg(B + idx) : INT_BIG;
        const int k = __popc(__ballot_sync(FULL, v < x));
        const int nlo = lo + s * k;
        const long long nhi = (long long)lo + (long long)s * (k + 1) - 1;
        lo = nlo;
        hi = nhi < hi ? (int)nhi : hi;
    }
    const int v = lo + lane < hi ? __ldg(B + lo + lane) : INT_BIG;
    return lo + __popc(__ballot_sync(FULL, v < x));
}

// Four 32-entry blocks of B from `base` in one round trip (INT_BIG past pd).
__device__ __forceinline__ void load_b128(const int32_t* __restrict__ B, int pd, int base, int lane, int (&v)[4]) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int idx = base + 32 * i + lane;
        v[i] = idx < pd ? __ldg(B + idx) : INT_BIG;
    }
}

// How many of the 128 loaded entries satisfy the (prefix-closed) predicate.
__device__ __forceinline__ int count_lt(const int (&v)[4], int x) {
    int n = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) n += __popc(__ballot_sync(FULL, v[i] < x));
    return n;
}

// Bit j of the result: entry j of this lane's quad (valid bit j) is in B.
// Warp-collective; `pos` is the warp's forward cursor into B.  The chunk's
// window of B usually lies within the 128 entries after the cursor, which
// one round of loads fetches together with both window bounds.
__device__ __forceinline__ unsigned chunk_members(const int32_t* __restrict__ B, int pd, int& pos,
                                                  const int (&c)[4], unsigned valid, int lane,
                                                  int* __restrict__ win) {
    int lmin = INT_BIG, lmax = -1;
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (valid >> j & 1u) {
            lmin = min(lmin, c[j]);
            lmax = max(lmax, c[j]);
        }
    const int amin = __reduce_min_sync(FULL, lmin);
    const int amax = __reduce_max_sync(FULL, lmax);
    if (amin == INT_BIG || pos >= pd) return 0u;
    int v[4];
    load_b128(B, pd, pos, lane, v);
    int nlt = count_lt(v, amin);
    int lo, hi;
    bool staged = false;
    if (nlt == 128) {
        // the window starts further on: search for it, then load from there
        lo = lower_bound_from(B, pd, pos + 128, amin, lane);
        load_b128(B, pd, lo, lane, v);
        nlt = 0;
    } else {
        lo = pos + nlt;
    }
    const int base = lo - nlt;  // index of v[0] at lane 0
    const int nle = amax == INT_BIG - 1 ? 128 : count_lt(v, amax + 1);
    if (nle < 128) {
        hi = base + nle;
        // stage B[lo, hi) (all inside the loaded 128 entries) in shared memory
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = 32 * i + lane;
            if (e >= nlt && e < nle) win[e - nlt] = v[i];
        }
        staged = true;
    } else {
        hi = lower_bound_from(B, pd, base + 128, amax + 1, lane);
    }
    pos = hi;
    const int len = hi - lo;
    if (len == 0) return 0u;
    unsigned flags = 0;
    if (staged) {
        __syncwarp();
        // this lane's values ascend: one binary search, then short forward steps
        int a = 0;
        bool first = true;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(valid >> j & 1u)) continue;
            if (first) {
                int b = len;
                while (a < b) {
                    const int mid = (a + b) >> 1;
                    if (win[mid] < c[j]) a = mid + 1;
                    else b = mid;
                }
                first = false;
            } else {
                while (a < len && win[a] < c[j]) ++a;
            }
            if (a < len && win[a] == c[j]) flags |= 1u << j;
        }
        __syncwarp();  // the window is rewritten by the next chunk
    } else {
        int from = lo;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!(valid >> j & 1u)) continue;
            int a = from, b = hi;
            while (a < b) {
                const int mid = (a + b) >> 1;
                if (__ldg(B + mid) < c[j]) a = mid + 1;
                else b = mid;
            }
            if (a < hi && __ldg(B + a) == c[j]) flags |= 1u << j;
            from = a;
        }
    }
    return flags;
}

// The warp's view of B = N(prev) across the chunks of one step: the 128
// entries B[base, base + 128) stay loaded in registers (v[i] at lane l is
// B[base + 32 i + l], INT_BIG past the end) until the chunks move past them.
struct BBlock {
    int base;   // -1: nothing loaded yet
    int v[4];
    int nv[4];  // the next block, B[base + 128, base + 256), already requested
};

// Load the block at `base` and request the one after it.
__device__ __forceinline__ void bb_load(const int32_t* __restrict__ B, int pd, int base, int lane, BBlock& bb) {
    bb.base = base;
    load_b128(B, pd, base, lane, bb.v);
    load_b128(B, pd, base + 128, lane, bb.nv);
}

// Move to the next block (its loads were issued a block earlier) and
// request the one after it.
__device__ __forceinline__ void bb_advance(const int32_t* __restrict__ B, int pd, int lane, BBlock& bb) {
    bb.base += 128;
#pragma unroll
    for (int i = 0; i < 4; ++i) bb.v[i] = bb.nv[i];
    load_b128(B, pd, bb.base + 128, lane, bb.nv);
}

// Bits of the warp's stage membership bytes that belong to this lane's eight
// stage entries (positions 4 lane + j and 128 + 4 lane + j).
__device__ __forceinline__ unsigned lane_mask_bits(const unsigned* __restrict__ mask, int lane) {
    // the four bytes of a quad (each 0 or 1) gathered into four bits: the
    // multiplier moves byte j's low bit to bit 24 + j, and no two partial
    // products land on the same bit, so nothing carries into bits 24..27
    const unsigned b0 = mask[lane] & 0x01010101u, b1 = mask[CHQ + lane] & 0x01010101u;
    return ((b0 * 0x01020408u) >> 24) | (((b1 * 0x01020408u) >> 24) << 4);
}

// Dense windows: B holds many more values than the stage inside the stage's
// range, so each stage entry x > `above` searches the window B[from, end)
// instead.  NSPL splitters B[from + (s+1) w - 1] (w = ceil((end - from) / NSPL))
// are staged in `spl`, splitter s at index s + s / 32 so that the search's
// power-of-two strides fall on different shared-memory banks; x's lower
// bound lies in bracket s = the number of splitters below x, found by a
// branch-free search in shared memory, and a binary search of that bracket
// in global memory finishes it (log2 w dependent loads instead of
// log2(end - from)), the lane's eight entries in lockstep.  Returns this
// lane's hit bits in the low word and, in the high word, the largest lower
// bound found (the next stage's window starts at or after it).
// Warp-collective.
__device__ __forceinline__ unsigned long long dense_members(const int32_t* __restrict__ B, int end, int from, int above,
                                                         int4 c_lo, int4 c_hi, unsigned valid, int lane,
                                                         int* __restrict__ spl) {
    const int cv[8] = {c_lo.x, c_lo.y, c_lo.z, c_lo.w, c_hi.x, c_hi.y, c_hi.z, c_hi.w};
    const int w = (end - from + NSPL - 1) / NSPL;
#pragma unroll
    for (int i = 0; i < NSPL / 32; ++i) {
        const int sp = 32 * i + lane;
        spl[sp + i] = __ldg(B + min((long long)from + (long long)(sp + 1) * w - 1, (long long)end - 1));
    }
    __syncwarp();
    int a[8], b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int x = cv[j];
        int lo = 0;
#pragma unroll
        for (int step = NSPL / 2; step > 0; step >>= 1) {
            const int i = lo + step - 1;
            if (spl[i + (i >> 5)] < x) lo += step;
        }
        // lo counts the splitters 0..NSPL-2 below x; when x is above them all
        // the bracket may start past the window's end: clamp it there (x is
        // then not in the window, and its lower bound is the end)
        const bool want = (valid >> j & 1u) && x > above;
        a[j] = want ? min(from + lo * w, end) : 0;
        b[j] = want ? min(a[j] + w, end) : 0;
    }
    for (;;) {
        bool more = false;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (a[j] < b[j]) {
                more = true;
                const int mid = (a[j] + b[j]) >> 1;
                if (__ldg(B + mid) < cv[j]) a[j] = mid + 1;
                else b[j] = mid;
            }
        if (!more) break;
    }
    unsigned f = 0;
    int hi_pos = from;
#pragma unroll
    for (int j = 0; j < 8; ++j)
        if (a[j] > 0) {
            hi_pos = max(hi_pos, a[j]);
            if (a[j] < end && __ldg(B + a[j]) == cv[j]) f |= 1u << j;
        }
    const int top = __reduce_max_sync(FULL, hi_pos);
    __syncwarp();  // the splitters are rewritten by the next dense stage
    return ((unsigned long long)(unsigned)top << 32) | f;
}

// One lane's four consecutive row entries (an aligned quad of the CSR
// arrays) with the state-dependent weight of each (0 outside the row).
template <int MODE>
struct Quad {
    typedef typename std::conditional<MODE == MODE_EXACT, uint32_t, float>::type W;
    int c[4];
    W w[4];
    unsigned valid;
};

template <int MODE>
__device__ __forceinline__ void clear_quad(Quad<MODE>& Q) {
    Q.valid = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        Q.c[j] = INT_BIG;
        Q.w[j] = 0;
    }
}

// Load quad q of the row [beg, end) and apply the weight rule except the
// node2vec factor (which needs the warp-collective membership test).
template <int MODE>
__device__ __forceinline__ void load_quad(const GraphDev& g, const StepCtx& cx, long long q, long long end,
                                          Quad<MODE>& Q) {
    const long long e0 = q << 2;
    clear_quad(Q);
    int et = 0;
    if (e0 + 3 < g.m) {
        const int4 cv = __ldg(reinterpret_cast<const int4*>(g.col + e0));
        Q.c[0] = cv.x; Q.c[1] = cv.y; Q.c[2] = cv.z; Q.c[3] = cv.w;
        if (MODE == MODE_EXACT) {
            const uint4 wv = __ldg(reinterpret_cast<const uint4*>(g.w_u32 + e0));
            Q.w[0] = wv.x; Q.w[1] = wv.y; Q.w[2] = wv.z; Q.w[3] = wv.w;
        } else {
            const float4 wv = __ldg(reinterpret_cast<const float4*>(g.w_f32 + e0));
            Q.w[0] = wv.x; Q.w[1] = wv.y; Q.w[2] = wv.z; Q.w[3] = wv.w;
        }
        if (cx.algo == FW_METAPATH) et = __ldg(reinterpret_cast<const int*>(g.etype + e0));
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long e = e0 + j;
            if (e < g.m) {
                Q.c[j] = __ldg(g.col + e);
                if (MODE == MODE_EXACT) Q.w[j] = __ldg(g.w_u32 + e);
                else Q.w[j] = __ldg(g.w_f32 + e);
                if (cx.algo == FW_METAPATH) et |= ((int)(uint8_t)__ldg(g.etype + e)) << (8 * j);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const long long e = e0 + j;
        if (e >= cx.beg && e < end) {
            Q.valid |= 1u << j;
            if (cx.algo == FW_METAPATH && (int)(int8_t)(et >> (8 * j)) != cx.want) Q.w[j] = 0;
        } else {
            Q.c[j] = INT_BIG;
            Q.w[j] = 0;
        }
    }
}

// Apply the node2vec factors to a loaded quad (warp-collective: every lane
// of the warp must call it).
template <int MODE>
__device__ __forceinline__ void n2v_factors(const StepCtx& cx, Quad<MODE>& Q, unsigned mem) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const bool isprev = Q.c[j] == cx.prev;
        const bool in = mem >> j & 1u;
        if (MODE == MODE_EXACT) Q.w[j] *= isprev ? cx.fi0 : (in ? cx.fi1 : cx.fi2);
        else Q.w[j] *= isprev ? cx.ff0 : (in ? cx.ff1 : cx.ff2);
    }
}

template <int MODE>
__device__ __forceinline__ void n2v_apply(const GraphDev& g, const StepCtx& cx, Quad<MODE>& Q, int& pos, int lane,
                                          int* win) {
    if (cx.algo != FW_NODE2VEC || cx.prev < 0) return;
    n2v_factors<MODE>(cx, Q, chunk_members(g.col + cx.pbeg, cx.pdeg, pos, Q.c, Q.valid, lane, win));
}

// A warp's weighted reservoir (exponential race with exponential jumps),
// run over the warp's entries in row order, 128 at a time.  tau = the current
// minimum race time E_i / w_i (E_i ~ Exp(1)) and sel its entry; X = the
// weight still to pass before some entry beats tau.  An entry of weight w
// beats the minimum with probability 1 - exp(-w tau), so the weight skipped
// before the next record is Exp(1) / tau; the record's own time is the race
// time conditioned to lie below tau.  Every lane holds the same state: a
// chunk costs one warp prefix sum and one comparison unless a record falls
// inside it, and a row of d entries makes about ln d records.  X is kept as
// an unevaluated sum of two FP32 numbers so that subtracting many chunk
// totals does not drift (FP64 is a slow pipe on this part).
struct WarpRes {
    float tau;
    int sel;
    float Xh, Xl;  // X as an unevaluated FP32 sum Xh + Xl
    uint32_t ctr;
    uint32_t spare0, spare1;
    uint32_t has_spare;

    __device__ __forceinline__ void init() {
        tau = __int_as_float(0x7f800000);  // +inf
        sel = -1;
        Xh = 0.0f;
        Xl = 0.0f;
        ctr = 0;
        has_spare = 0;
    }
};

// The order in which segment results compete: the smaller race time wins,
// the smaller row index breaks a tie (race times are positive, so their FP32
// bit patterns order as the values do).
__device__ __forceinline__ unsigned long long race_key(const WarpRes& r) {
    return ((unsigned long long)__float_as_uint(r.tau) << 32) | (unsigned)r.sel;
}

// Quads per segment for a row range of nq quads: seg_q, or more for rows of
// more than NSEG_MAX such segments; a multiple of 32 (one quad per lane).
__device__ __forceinline__ long long seg_quads(long long nq, int seg_q) {
    const long long sq = max((long long)seg_q, (nq + NSEG_MAX - 1) / NSEG_MAX);
    return (sq + 31) & ~31ll;
}

// A new record at row entry idx of weight w (uniform across the warp).
__device__ __forceinline__ WarpRes warp_record(WarpRes r, int idx, float w, uint64_t seed, uint64_t qid, uint32_t t,
                                            uint32_t stream) {
    uint32_t a, b;
    if (r.has_spare) {
        a = r.spare0;
        b = r.spare1;
        r.has_spare = 0;
    } else {
        const uint4 o = lane_block(seed, qid, t, stream, r.ctr++);
        a = o.x;
        b = o.y;
        r.spare0 = o.z;
        r.spare1 = o.w;
        r.has_spare = 1;
    }
    const float u1 = unit_open(a), u2 = unit_open(b);
    // -log u by the fast intrinsic (u is at least 2^-24, well inside its
    // accurate range); the conditioned draw keeps log1pf/expm1f, whose
    // arguments are tiny once many entries have been seen
    float e;
    if (isinf(r.tau)) e = -__logf(u1);
    else e = -log1pf(u1 * expm1f(-w * r.tau));
    r.tau = __fdividef(e, w);
    r.sel = idx;
    r.Xh = __fdividef(-__logf(u2), r.tau);
    r.Xl = 0.0f;
    return r;
}

// A record falls inside a stage: find every record there, in visiting order
// (lane by lane, j ascending), and leave R with the skip budget past the
// stage.  `own` is this lane's weight total.
__device__ __forceinline__ WarpRes stage_records(WarpRes R, float4 wa, float4 wb, float own, int e0, int lane,
                                              uint64_t seed, uint64_t qid, uint32_t t, uint32_t stream) {
    const float w[8] = {wa.x, wa.y, wa.z, wa.w, wb.x, wb.y, wb.z, wb.w};
    float incl = own;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const float n = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += n;
    }
    const float tot = __shfl_sync(FULL, incl, 31);
    // running sums in visiting order
    float cum[8];
    cum[0] = (incl - own) + w[0];
#pragma unroll
    for (int j = 1; j < 8; ++j) cum[j] = cum[j - 1] + w[j];
    float target = R.Xh + R.Xl;  // a record falls on the first entry whose cumulative weight reaches target
    int last = -1;               // visiting position (lane * 8 + j) of the last record: each record lies beyond it
    for (;;) {
        int jj = -1;
#pragma unroll
        for (int j = 7; j >= 0; --j)
            if (lane * 8 + j > last && w[j] > 0.0f && cum[j] >= target) jj = j;
        const unsigned m = __ballot_sync(FULL, jj >= 0);
        if (!m) {
            R.Xh = target - tot;
            R.Xl = 0.0f;
            return R;
        }
        const int L = __ffs(m) - 1;
        float wj = 0.0f, cj = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j)
            if (j == jj) {
                wj = w[j];
                cj = cum[j];
            }
        const float wr = __shfl_sync(FULL, wj, L);
        const float cr = __shfl_sync(FULL, cj, L);
        const int jl = __shfl_sync(FULL, jj, L);
        const int idx = __shfl_sync(FULL, e0, L) + jl + (jl >= 4 ? 124 : 0);
        last = L * 8 + jl;
        R = warp_record(R, idx, wr, seed, qid, t, stream);
        target = cr + R.Xh;
    }
}

// Offer one stage: lane `lane` holds the entries of row indices e0 + j
// (w[j], j < 4) and e0 + 124 + j (w[j], j >= 4), i.e. its quad of each
// chunk of the stage.  Entries are visited lane by lane, j ascending: any
// fixed order gives the same law.  The stage total comes from an xor
// butterfly, whose pairwise sums are the same in every lane (a + b = b + a
// in IEEE arithmetic), so the warp's reservoir state stays uniform.
__device__ __forceinline__ void warp_offer_stage(WarpRes& R, const float (&w)[8], int e0, int lane, uint64_t seed,
                                                 uint64_t qid, uint32_t t, uint32_t stream) {
    const float own = ((w[0] + w[1]) + (w[2] + w[3])) + ((w[4] + w[5]) + (w[6] + w[7]));
    float tot = own;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(FULL, tot, o);
    if (R.Xh - tot + R.Xl > 0.0f) {  // no record in this stage (the common case)
        // X -= tot with the rounding error kept (Fast2Sum: |Xh| > tot here)
        const float sh = R.Xh - tot;
        R.Xl += (R.Xh - sh) - tot;
        R.Xh = sh;
        return;
    }
    R = stage_records(R, make_float4(w[0], w[1], w[2], w[3]), make_float4(w[4], w[5], w[6], w[7]), own, e0, lane,
                      seed, qid, t, stream);
}

// Pick inside one lane's quad: smallest j whose prefix exceeds rr.
__device__ __forceinline__ int pick_in_quad(const uint32_t (&w)[4], unsigned long long rr) {
    unsigned long long acc = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        acc += w[j];
        if (acc > rr) return j;
    }
    return 3;
}

// Whether a stage of nq quads from qs is read from global memory instead of
// being copied (it would run past the end of the CSR arrays).  Uniform.
__device__ __forceinline__ bool stage_direct(const GraphDev& g, long long qs, int nq) {
    return 4 * (qs + ((nq + 3) & ~3)) > g.m;
}

// Lane 0: start loading quads [qs, qs + nq) (qs a multiple of 4, nq <= SQ)
// into stage st of the warp's ring.
template <int MODE>
__device__ __forceinline__ void pipe_issue(const GraphDev& g, WarpPipe& P, int st, long long qs, int nq,
                                           bool labels) {
    unsigned char* b = P.buf + st * STAGE_BYTES;
    if (!stage_direct(g, qs, nq)) {
        const uint32_t nq4 = (uint32_t)((nq + 3) & ~3);
        mbar_arrive_expect_tx(&P.bar[st], nq4 * 32 + (labels ? nq4 * 4 : 0));
        tma_load_1d(b + ST_COL, g.col + 4 * qs, nq4 * 16, &P.bar[st]);
        if (MODE == MODE_EXACT) tma_load_1d(b + ST_W, g.w_u32 + 4 * qs, nq4 * 16, &P.bar[st]);
        else tma_load_1d(b + ST_W, g.w_f32 + 4 * qs, nq4 * 16, &P.bar[st]);
        if (labels) tma_load_1d(b + ST_ET, g.etype + 4 * qs, nq4 * 4, &P.bar[st]);
    } else {
        mbar_arrive(&P.bar[st]);
    }
}

// This lane's quad of chunk h (0 or 1) of a landed stage whose entry 0 is
// row index r0; entries at row indices outside [0, lim) are masked out,
// MetaPath labels applied.
template <int MODE>
__device__ __forceinline__ void stage_quad(const StepCtx& c, const unsigned char* b, int h, int r0, int lim, int lane,
                                           Quad<MODE>& Q) {
    const int o = h * (CHQ * 16) + lane * 16;
    const int4 cv = *reinterpret_cast<const int4*>(b + ST_COL + o);
    Q.c[0] = cv.x; Q.c[1] = cv.y; Q.c[2] = cv.z; Q.c[3] = cv.w;
    if (MODE == MODE_EXACT) {
        const uint4 wv = *reinterpret_cast<const uint4*>(b + ST_W + o);
        Q.w[0] = wv.x; Q.w[1] = wv.y; Q.w[2] = wv.z; Q.w[3] = wv.w;
    } else {
        const float4 wv = *reinterpret_cast<const float4*>(b + ST_W + o);
        Q.w[0] = wv.x; Q.w[1] = wv.y; Q.w[2] = wv.z; Q.w[3] = wv.w;
    }
    const int et = c.algo == FW_METAPATH ? *reinterpret_cast<const int*>(b + ST_ET + h * (CHQ * 4) + lane * 4) : 0;
    Q.valid = 0;
    const int rel = r0 + h * (4 * CHQ) + 4 * lane;  // row index of entry 0 of the quad
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((unsigned)(rel + j) < (unsigned)lim) {
            Q.valid |= 1u << j;
            if (c.algo == FW_METAPATH && (int)(int8_t)(et >> (8 * j)) != c.want) Q.w[j] = 0;
        } else {
            Q.c[j] = INT_BIG;
            Q.w[j] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Fast mode: the lean range scan.  Used for every range whose stages can all
// be copied by TMA (everything but the very end of the CSR arrays).  A stage
// costs: one barrier wait, four 16-byte shared loads per lane, the weight
// rule, the reservoir's skip test (one butterfly sum) and lane 0's copy of a
// later stage.  Rows are masked only in a range's first and last stage.
// node2vec tracks `nb`, the smallest value of N(prev) above every entry seen
// so far (INT_MIN: not known yet), so that a stage with nb > its largest
// entry — no value of N(prev) inside its range — needs no membership work.
// ---------------------------------------------------------------------------

// Lane 0: copy the first ne entries (a multiple of 16, possibly 0) of a
// stage into ring slot st.
__device__ __forceinline__ void issue_stage_fast(WarpPipe& P, int st, const int32_t* cs, const float* ws,
                                                 const int8_t* es, uint32_t ne, bool labels) {
    unsigned char* b = P.buf + st * STAGE_BYTES;
    if (ne == 0) {
        mbar_arrive(&P.bar[st]);
        return;
    }
    mbar_arrive_expect_tx(&P.bar[st], ne * 8 + (labels ? ne : 0));
    tma_load_1d(b + ST_COL, cs, ne * 4, &P.bar[st]);
    tma_load_1d(b + ST_W, ws, ne * 4, &P.bar[st]);
    if (labels) tma_load_1d(b + ST_ET, es, ne, &P.bar[st]);
}

// Entries to copy of stage k of a range: whole 16-entry groups, and for the
// range's last stage, when it runs into the end of the CSR arrays, only the
// groups that lie inside them (stage_tail_fill loads the rest).
__device__ __forceinline__ uint32_t stage_copy_entries(long long m, long long e0, int nq) {
    const long long ne = 4ll * ((nq + 3) & ~3);
    return (uint32_t)(e0 + ne <= m ? ne : ((m - e0) >> 4) << 4);
}

// The end of the CSR arrays: the entries [e0 + from, e0 + to) of a stage
// (to - from < 16 + 4 * SQ) that no copy brought in, by plain loads into the
// stage buffer b.  Out of line: it runs only for the last rows of the graph.
__device__ __noinline__ void stage_tail_fill(const int32_t* __restrict__ col, const float* __restrict__ w,
                                             const int8_t* __restrict__ et, unsigned char* b, long long e0, int from,
                                             int to, int lane) {
    for (int e = from + lane; e < to; e += 32) {
        reinterpret_cast<int*>(b + ST_COL)[e] = __ldg(col + e0 + e);
        reinterpret_cast<float*>(b + ST_W)[e] = __ldg(w + e0 + e);
        if (et) reinterpret_cast<int8_t*>(b + ST_ET)[e] = __ldg(et + e0 + e);
    }
    __syncwarp();
}

// Value at position pos (< 128) of a loaded block of B.  Warp-collective:
// every lane takes part in the shuffles, each with its own pos.
__device__ __forceinline__ int block_value(const BBlock& bb, int pos) {
    const int src = pos & 31, ii = pos >> 5;
    const int x0 = __shfl_sync(FULL, bb.v[0], src), x1 = __shfl_sync(FULL, bb.v[1], src);
    const int x2 = __shfl_sync(FULL, bb.v[2], src), x3 = __shfl_sync(FULL, bb.v[3], src);
    return ii == 0 ? x0 : (ii == 1 ? x1 : (ii == 2 ? x2 : x3));
}

// Stage position of value x among the 256 staged entries colS, or -1.  colS
// ascends over the whole stage: the scan has overwritten the entries outside
// the row with INT_MIN (before it) and INT_BIG (after it), which equal no
// vertex id.  x picks its half by a127 (entry 127), then the first quad of
// that half whose largest entry is >= x by a five-step binary search over
// the quads' last entries in shared memory, and compares x with that quad's
// four entries.  Per lane; x may differ between lanes.
__device__ __forceinline__ int stage_find(int a127, const int* __restrict__ colS, int x) {
    const bool hi = x > a127;
    const int* qmax = colS + (hi ? 4 * CHQ : 0) + 3;  // qmax[4 q] = last entry of quad q of the half
    int q = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
        const int i = q + step - 1;
        if (qmax[4 * i] < x) q += step;
    }
    const int p = (hi ? 4 * CHQ : 0) + 4 * q;
    const int4 v = *reinterpret_cast<const int4*>(colS + p);
    const unsigned hit = (v.x == x ? 1u : 0u) | (v.y == x ? 2u : 0u) | (v.z == x ? 4u : 0u) | (v.w == x ? 8u : 0u);
    return hit ? p + __ffs(hit) - 1 : -1;
}

// Membership of one stage's entries in N(prev) = B when some value of B may
// fall inside the stage's range [amin, amax] (its first and last entry of
// the row).  The values of B inside the range form one run of the loaded
// 128-entry block (and maybe of the blocks after it); the run is handed out
// 32 values per round, one per lane, each located in the stage by stage_find,
// and every hit sets its entry's byte in the warp's 256-byte mask (the values
// of B are distinct, so no two lanes write the same byte).  If the range runs past the block
// and, at the block's density, would hold several more blocks, a search finds
// where it ends, and a window of more than kDenseMin values is answered from
// the entries' side (dense_members).  cv: this lane's entries, ordered as
// stage_find needs them.  Returns this lane's bits (bit j: entry cv[j]) in
// the low word and, in the high word, the first value of B above amax (or a
// value below it, or INT_MIN when not known: the next stage then looks
// again).  Warp-collective.
__device__ __forceinline__ unsigned long long stage_members(const int32_t* __restrict__ B, int pd, BBlock& bb,
                                                         const int* __restrict__ colS, int amin,
                                                         int amax, const int (&cv)[8], unsigned valid, int lane,
                                                         unsigned* __restrict__ mask, int* __restrict__ spl) {
    if (bb.base < 0) bb_load(B, pd, lower_bound_from(B, pd, 0, amin, lane), lane, bb);
    int last = __shfl_sync(FULL, bb.v[3], 31);
    if (last < amin) {
        // the whole block lies below this stage: jump to the stage's range
        bb_load(B, pd, lower_bound_from(B, pd, bb.base + 128, amin, lane), lane, bb);
        last = __shfl_sync(FULL, bb.v[3], 31);
    }
    const int a127 = __shfl_sync(FULL, cv[3], 31);
    reinterpret_cast<uint2*>(mask)[lane] = make_uint2(0u, 0u);
    __syncwarp();
    bool checked = false;
    int nb = INT_BIG;
    while (bb.base < pd) {
        // positions [p0, p1) of the block hold the values inside [amin, amax]
        int nge = 0, nle = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            nge += __popc(__ballot_sync(FULL, bb.v[i] >= amin));
            nle += __popc(__ballot_sync(FULL, bb.v[i] <= amax));
        }
        const int p0 = 128 - nge, p1 = nle;
#pragma unroll 1
        for (int r = p0; r < p1; r += 32) {
            const int pa = r + lane;
            const int ha = stage_find(a127, colS, block_value(bb, pa));
            if (pa < p1 && ha >= 0) reinterpret_cast<unsigned char*>(mask)[ha] = 1;
        }
        if (p1 < 128) {
            nb = block_value(bb, p1);  // the block reaches past the stage: the next value of B
            break;
        }
        // every value of the block is at most amax: the window goes on
        if (bb.base + 128 >= pd) {
            bb.base += 128;
            break;
        }
        const int first = __shfl_sync(FULL, bb.v[0], 0);
        if (!checked && (float)(amax - last) * 128.0f > kDenseBlocks * 128.0f * (float)(last - first + 1)) {
            checked = true;
            const int from = bb.base + 128;
            const int ub = lower_bound_from(B, pd, from, amax + 1, lane);
            if (ub - from > kDenseMin) {
                const unsigned long long dm =
                    dense_members(B, ub, from, last, make_int4(cv[0], cv[1], cv[2], cv[3]),
                                  make_int4(cv[4], cv[5], cv[6], cv[7]), valid, lane, spl);
                const unsigned f = (unsigned)dm;
                bb_load(B, pd, (int)(dm >> 32), lane, bb);
                __syncwarp();
                return ((unsigned long long)(unsigned)INT_MIN << 32) | (f | lane_mask_bits(mask, lane));
            }
        }
        bb_advance(B, pd, lane, bb);
        last = __shfl_sync(FULL, bb.v[3], 31);
    }
    __syncwarp();
    return ((unsigned long long)(unsigned)nb << 32) | lane_mask_bits(mask, lane);
}

// Scan quads [qa, qb) of the row [c.beg, c.beg + c.d) in fast mode: weights
// with the rule's factors, offered to the warp's reservoir R drawing from
// random stream rng_stream.  False if a copy never landed.  Warp-collective.
__device__ __forceinline__ bool scan_range_fast(const GraphDev& g, const StepCtx& c, long long qa, long long qb,
                                                int lane, int* __restrict__ win, WarpPipe& P, WarpRes& R,
                                                uint32_t rng_stream, uint64_t seed, uint64_t qid, uint32_t t) {
    const int nqt = (int)(qb - qa);                       // quads in the range
    const int nst = (nqt + SQ - 1) / SQ;
    const bool labels = c.algo == FW_METAPATH;
    const bool n2v = c.algo == FW_NODE2VEC && c.prev >= 0;
    const int r_a = (int)((qa << 2) - c.beg);             // row index of the range's first staged entry
    const int lim = (int)min((long long)c.d, (qb << 2) - c.beg);  // entries at or past lim are outside
    const int32_t* cs = g.col + (qa << 2);
    const float* ws = g.w_f32 + (qa << 2);
    const int8_t* es = labels ? g.etype + (qa << 2) : nullptr;
    if (lane == 0) {
        int ist = P.st;
        uint32_t iph = P.ph;
        for (int k = 0; k < nst && k < NST; ++k) {
            const int nq = min(SQ, nqt - k * SQ);
            issue_stage_fast(P, ist, cs + k * 4 * SQ, ws + k * 4 * SQ, es ? es + k * 4 * SQ : nullptr,
                             stage_copy_entries(g.m, (qa << 2) + k * 4 * SQ, nq), labels);
            ring_next(ist, iph);
        }
    }
    // whether the last stage runs into the end of the CSR arrays
    const bool tail = (qa + (long long)(nst - 1) * SQ + ((nqt - (nst - 1) * SQ + 3) & ~3)) * 4 > g.m;
    const int32_t* B = g.col + c.pbeg;
    BBlock bb;
    bb.base = -1;
    int nb = INT_MIN;
    if (n2v && qa == ((c.beg >> 2) & ~3ll)) {
        // a whole row (or its first segment): start loading N(prev)'s first
        // block now, while the first stage is still on its way
        bb_load(B, c.pdeg, 0, lane, bb);
    }
    for (int k = 0; k < nst; ++k) {
        const int st = P.st;
        if (!mbar_try_wait(&P.bar[st], P.ph)) {
            const bool ok = mbar_wait_bounded(&P.bar[st], P.ph);
            if (!__all_sync(FULL, ok)) {
                // let the copies already issued land before giving up
                if (lane == 0) {
                    int dst = st;
                    uint32_t dph = P.ph;
                    for (int kk = k + 1; kk < nst && kk < k + NST; ++kk) {
                        ring_next(dst, dph);
                        mbar_wait_bounded(&P.bar[dst], dph);
                    }
                }
                return false;
            }
        }
        unsigned char* b = P.buf + st * STAGE_BYTES;
        if (tail && k == nst - 1) {
            const long long e0 = (qa << 2) + k * 4 * SQ;
            const int nq = nqt - k * SQ;
            stage_tail_fill(g.col, g.w_f32, labels ? g.etype : nullptr, b, e0,
                            (int)stage_copy_entries(g.m, e0, nq), (int)min(4ll * nq, g.m - e0), lane);
        }
        const int4 c0 = *reinterpret_cast<const int4*>(b + ST_COL + lane * 16);
        const int4 c1 = *reinterpret_cast<const int4*>(b + ST_COL + CHQ * 16 + lane * 16);
        const float4 w0 = *reinterpret_cast<const float4*>(b + ST_W + lane * 16);
        const float4 w1 = *reinterpret_cast<const float4*>(b + ST_W + CHQ * 16 + lane * 16);
        int cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
        float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const int r0 = r_a + k * (4 * SQ);
        const bool edge = r0 < 0 || r0 + 4 * SQ > lim;
        unsigned valid = 0xFFu;
        if (edge) {
            // the range's first or last stage: entries outside the row are
            // out; node2vec also overwrites them in the staged copy, which
            // stage_find searches
            valid = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int rel = r0 + 4 * lane + j + (j >= 4 ? 4 * CHQ - 4 : 0);
                if ((unsigned)rel < (unsigned)lim) {
                    valid |= 1u << j;
                } else {
                    cv[j] = rel < 0 ? INT_MIN : INT_BIG;  // keeps the stage's entries in ascending order
                    wv[j] = 0.0f;
                    if (n2v) reinterpret_cast<int*>(b + ST_COL)[4 * lane + (j & 3) + (j >= 4 ? 4 * CHQ : 0)] = cv[j];
                }
            }
        }
        if (labels) {
            const int e0 = *reinterpret_cast<const int*>(b + ST_ET + lane * 4);
            const int e1 = *reinterpret_cast<const int*>(b + ST_ET + CHQ * 4 + lane * 4);
#pragma unroll
            for (int j = 0; j < 8; ++j)
                if ((int)(int8_t)((j < 4 ? e0 : e1) >> (8 * (j & 3))) != c.want) wv[j] = 0.0f;
        }
        if (n2v) {
            const int* colS = reinterpret_cast<const int*>(b + ST_COL);
            int ia = 0, ib = 4 * SQ, amin, amax;
            if (edge) {
                ia = max(0, -r0);
                ib = min(4 * SQ, lim - r0);
                amin = colS[ia];
                amax = colS[ib - 1];
            } else {
                amin = __shfl_sync(FULL, cv[0], 0);
                amax = __shfl_sync(FULL, cv[7], 31);
            }
            unsigned mem = 0;
            if (nb <= amax) {
                const unsigned long long r =
                    stage_members(B, c.pdeg, bb, colS, amin, amax, cv, valid, lane, P.mask, win);
                mem = (unsigned)r;
                nb = (int)(unsigned)(r >> 32);
            }
            if (c.prev >= amin && c.prev <= amax) {
                // prev may sit in this stage: the return factor applies there
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    float f = (mem >> j & 1u) ? c.ff1 : c.ff2;
                    if (cv[j] == c.prev) f = c.ff0;
                    wv[j] *= f;
                }
            } else {
#pragma unroll
                for (int j = 0; j < 8; ++j) wv[j] *= (mem >> j & 1u) ? c.ff1 : c.ff2;
            }
        }
        __syncwarp();  // every lane is done with the stage: it may be refilled
        if (lane == 0 && k + NST < nst) {
            const int kn = k + NST;
            const int nq = min(SQ, nqt - kn * SQ);
            issue_stage_fast(P, st, cs + kn * 4 * SQ, ws + kn * 4 * SQ, es ? es + kn * 4 * SQ : nullptr,
                             stage_copy_entries(g.m, (qa << 2) + kn * 4 * SQ, nq), labels);
        }
        ring_next(P.st, P.ph);
        warp_offer_stage(R, wv, r0 + 4 * lane, lane, seed, qid, t, rng_stream);
    }
    return true;
}


// Stream quads [qa, qb) (qa a multiple of 4) of the row [c.beg, end) through
// the warp's TMA ring, NST - 1 stages ahead: weights with the node2vec
// factors applied, then (fast) the warp's reservoir drawing from random
// stream rng_stream, or (exact) each lane's running sum and, if chunk_sums
// is given, one warp total per 128-entry chunk.  False if a copy never
// landed.
template <int MODE>
__device__ __forceinline__ bool scan_range(const GraphDev& g, const StepCtx& c, long long qa, long long qb,
                                           long long end, int lane, int* __restrict__ win, WarpPipe& P,
                                           WarpRes& res, unsigned long long& lane_sum,
                                           unsigned long long* __restrict__ chunk_sums, uint32_t rng_stream,
                                           uint64_t seed, uint64_t qid, uint32_t t) {
    const int nst = (int)((qb - qa + SQ - 1) / SQ);
    const bool labels = c.algo == FW_METAPATH;
    // row indices: of the range's first staged entry, and the end of the
    // range (entries at or past it are masked out)
    const int r_a = (int)((qa << 2) - c.beg);
    const int lim = (int)min((long long)c.d, (qb << 2) - c.beg);
    if (lane == 0) {
        int ist = P.st;
        uint32_t iph = P.ph;
        for (int k = 0; k < nst && k < NST; ++k) {
            const long long qs = qa + (long long)k * SQ;
            pipe_issue<MODE>(g, P, ist, qs, (int)min((long long)SQ, qb - qs), labels);
            ring_next(ist, iph);
        }
    }
    int pos = 0;
    BBlock bb;
    bb.base = -1;
    int nb = INT_MIN;  // smallest value of N(prev) above the entries seen so far (INT_MIN: not known)
    const bool n2v = c.algo == FW_NODE2VEC && c.prev >= 0;
    if (n2v && qa == ((c.beg >> 2) & ~3ll)) {
        // a whole row (or its first segment): start loading N(prev)'s first
        // block now, while the first stage is still on its way
        bb_load(g.col + c.pbeg, c.pdeg, 0, lane, bb);
    }
    bool ok = true;
    for (int k = 0; k < nst; ++k) {
        const int st = P.st;
        const long long qs = qa + (long long)k * SQ;
        const int nq = (int)min((long long)SQ, qb - qs);
        const int r0 = r_a + k * (4 * SQ);
        if (!mbar_wait_bounded(&P.bar[st], P.ph)) ok = false;
        if (!__all_sync(FULL, ok)) {
            // let the copies already issued land before giving up
            if (lane == 0) {
                int dst = st;
                uint32_t dph = P.ph;
                for (int kk = k + 1; kk < nst && kk < k + NST; ++kk) {
                    ring_next(dst, dph);
                    mbar_wait_bounded(&P.bar[dst], dph);
                }
            }
            return false;
        }
        Quad<MODE> h0, h1;
        if (stage_direct(g, qs, nq)) {
            // the end of the arrays: plain loads, the entries' side membership
            if (lane < nq) load_quad<MODE>(g, c, qs + lane, end, h0);
            else clear_quad(h0);
            if (lane + CHQ < nq) load_quad<MODE>(g, c, qs + CHQ + lane, end, h1);
            else clear_quad(h1);
            n2v_apply<MODE>(g, c, h0, pos, lane, win);
            n2v_apply<MODE>(g, c, h1, pos, lane, win);
        } else {
            unsigned char* b = P.buf + st * STAGE_BYTES;
            stage_quad<MODE>(c, b, 0, r0, lim, lane, h0);
            stage_quad<MODE>(c, b, 1, r0, lim, lane, h1);
            if (n2v) {
                // staged entries [ia, ib) belong to this range of the row
                const int ia = max(0, -r0);
                const int ib = min(4 * SQ, lim - r0);
                // the stage's entries in ascending order: INT_MIN before the row, INT_BIG after it
                int cv[8] = {h0.c[0], h0.c[1], h0.c[2], h0.c[3], h1.c[0], h1.c[1], h1.c[2], h1.c[3]};
                int* colS = reinterpret_cast<int*>(b + ST_COL);
                const unsigned vbits = h0.valid | (h1.valid << 4);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int e = 4 * lane + (j & 3) + (j >= 4 ? 4 * CHQ : 0);
                    if (e < ia) cv[j] = INT_MIN;
                    // entries outside the row take their sentinel in the
                    // staged copy too, which stage_find searches
                    if (!(vbits >> j & 1u)) colS[e] = cv[j];
                }
                unsigned mem = 0;
                if (ia < ib && nb <= colS[ib - 1]) {
                    const unsigned long long rm = stage_members(g.col + c.pbeg, c.pdeg, bb, colS, colS[ia],
                                                                colS[ib - 1], cv, h0.valid | (h1.valid << 4), lane,
                                                                P.mask, win);
                    mem = (unsigned)rm;
                    nb = (int)(unsigned)(rm >> 32);
                }
                n2v_factors<MODE>(c, h0, mem & 0xFu);
                n2v_factors<MODE>(c, h1, mem >> 4);
            }
        }
        __syncwarp();  // every lane is done with the stage: it may be refilled
        if (lane == 0 && k + NST < nst) {
            const long long qn = qa + (long long)(k + NST) * SQ;
            pipe_issue<MODE>(g, P, st, qn, (int)min((long long)SQ, qb - qn), labels);
        }
        ring_next(P.st, P.ph);
        if (MODE == MODE_FAST) {
            const float wf[8] = {(float)h0.w[0], (float)h0.w[1], (float)h0.w[2], (float)h0.w[3],
                                 (float)h1.w[0], (float)h1.w[1], (float)h1.w[2], (float)h1.w[3]};
            warp_offer_stage(res, wf, r0 + 4 * lane, lane, seed, qid, t, rng_stream);
        } else {
            const unsigned long long s0 = (unsigned long long)h0.w[0] + h0.w[1] + h0.w[2] + h0.w[3];
            const unsigned long long s1 = (unsigned long long)h1.w[0] + h1.w[1] + h1.w[2] + h1.w[3];
            lane_sum += s0 + s1;
            if (chunk_sums) {
                const unsigned long long cs0 = warp_sum_u64(s0), cs1 = warp_sum_u64(s1);
                if (lane == 0 && 2 * k < NCHUNK_MAX) chunk_sums[2 * k] = cs0;
                if (lane == 0 && 2 * k + 1 < NCHUNK_MAX) chunk_sums[2 * k + 1] = cs1;
            }
        }
    }
    return ok;
}

// Exact mode: scan quads [qa, qb) chunk by chunk and return the row-relative
// index of the entry where the running prefix (from 0) first exceeds r.
// Warp-collective, uniform result; -1 if the range sums to at most r.
__device__ int exact_find(const GraphDev& g, const StepCtx& cx, long long qa, long long qb, long long end,
                          unsigned long long r, int lane, int* win) {
    int pos = 0;
    unsigned long long run = 0;
    for (long long qc = qa; qc < qb; qc += 32) {
        const long long q = qc + lane;
        Quad<MODE_EXACT> Q;
        if (q < qb) load_quad<MODE_EXACT>(g, cx, q, end, Q);
        else clear_quad(Q);
        n2v_apply<MODE_EXACT>(g, cx, Q, pos, lane, win);
        const unsigned long long s = (unsigned long long)Q.w[0] + Q.w[1] + Q.w[2] + Q.w[3];
        const unsigned long long incl = warp_incl_scan_u64(s, lane);
        const unsigned m = __ballot_sync(FULL, run + incl > r);
        if (m) {
            const int L = __ffs(m) - 1;
            int sel = 0;
            if (lane == L) sel = (int)((q << 2) + pick_in_quad(Q.w, r - (run + incl - s)) - cx.beg);
            return __shfl_sync(FULL, sel, L);
        }
        run += __shfl_sync(FULL, incl, 31);
    }
    return -1;
}

// Find which of the n sums (n <= 64) holds the crossing of r, and r's offset
// inside it.  Warp-collective; sums lives in shared memory.
__device__ __forceinline__ int find_crossing(const unsigned long long* sums, int n, unsigned long long& r, int lane) {
    unsigned long long run = 0;
    for (int base = 0; base < n; base += 32) {
        const int i = base + lane;
        const unsigned long long v = i < n ? sums[i] : 0ull;
        const unsigned long long incl = warp_incl_scan_u64(v, lane);
        const unsigned m = __ballot_sync(FULL, run + incl > r);
        if (m) {
            const int L = __ffs(m) - 1;
            const unsigned long long before = __shfl_sync(FULL, run + incl - v, L);
            r -= before;
            return base + L;
        }
        run += __shfl_sync(FULL, incl, 31);
    }
    return -1;
}

__device__ __forceinline__ int find_req(const ReqDev* __restrict__ reqs, int n_req, long long gq) {
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].q_begin <= gq) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Per-warp counters, kept by lane 0 in the warp's shared-memory row (not in
// registers: the scan loop needs them) and flushed at exit.
struct Counters {
    unsigned long long* v;
    __device__ __forceinline__ void clear() {
#pragma unroll
        for (int i = 0; i < C_NUM; ++i) v[i] = 0;
    }
    __device__ __forceinline__ void step(int d, int algo, bool hub) {
        v[C_STEPS] += 1;
        v[C_ROWS] += (unsigned long long)d;
        v[hub ? C_BLOCK_STEPS : C_WARP_STEPS] += 1;
        if (algo == FW_NODE2VEC) v[C_PROBES] += (unsigned long long)d;
        v[C_ALGO_BYTES] += (unsigned long long)(8ll * d + (algo == FW_METAPATH ? d : 0) + 16 + 4);
    }
};

template <int NT>
__device__ __forceinline__ StepCtx make_ctx(const Smem<NT>& sm, const ReqDev& R, int s, long long beg, int d) {
    StepCtx c;
    c.beg = beg;
    c.d = d;
    c.pbeg = sm.pbeg[s];
    c.pdeg = sm.pdeg[s];
    c.prev = sm.prev[s];
    c.algo = R.algo;
    c.want = (R.algo == FW_METAPATH) ? (int)R.schema[sm.t[s] % R.schema_len] : -1;
    c.fi0 = R.fac_i[0];
    c.fi1 = R.fac_i[1];
    c.fi2 = R.fac_i[2];
    c.ff0 = R.fac_f[0];
    c.ff1 = R.fac_f[1];
    c.ff2 = R.fac_f[2];
    return c;
}

// Commit a move of slot s (one thread): append `next` to the path, advance
// the walk, apply the PPR stop test and the length limit, start fetching the
// next row's offsets into L2, and hand the slot back (READY or FINISH).
template <int NT>
__device__ __forceinline__ void commit(const GraphDev& g, Smem<NT>& sm, const ReqDev& R, int s, const StepCtx& c,
                                       int next, uint32_t oz) {
    const long long width = (long long)R.max_len + 1;
    const int k = sm.k[s];
    R.paths[sm.q[s] * width + k] = next;
    sm.k[s] = k + 1;
    sm.prev[s] = sm.cur[s];
    sm.pbeg[s] = c.beg;
    sm.pdeg[s] = c.d;
    sm.cur[s] = next;
    const int t = sm.t[s] + 1;
    sm.t[s] = t;
    const bool stop = (R.algo == FW_PPR && oz < R.t_stop) || t >= sm.lim[s];
    if (!stop) asm volatile("prefetch.global.L2 [%0];" ::"l"(g.row_ptr + next));
    __threadfence_block();
    *(volatile int*)&sm.state[s] = stop ? ST_FINISH : ST_READY;
}

// Finish the step of a hub task (the warp that completed its last segment).
template <int MODE, int NT>
__device__ void hub_finalize(const GraphDev& g, Smem<NT>& sm, HubTask& H, int lane, int* win, Counters& cnt) {
    const ReqDev& R = sm.rq[H.slot];
    const StepCtx c = H.c;
    int sel = -1;
    uint32_t oz = 0xFFFFFFFFu;
    if (MODE == MODE_FAST) {
        const unsigned long long b = H.best;
        sel = b == ~0ull ? -1 : (int)(b & 0xFFFFFFFFull);
        if (sel >= 0 && R.algo == FW_PPR) oz = step_block(H.seed, H.qid, H.t).z;
    } else {
        unsigned long long W = 0;
        for (int j = lane; j < H.nseg; j += 32) W += H.seg_sum[j];
        W = warp_sum_u64(W);
        if (W != 0) {
            const uint4 o = step_block(H.seed, H.qid, H.t);
            oz = o.z;
            const unsigned long long x = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            unsigned long long r = __umul64hi(x, W);
            const int j = find_crossing(H.seg_sum, H.nseg, r, lane);
            if (j >= 0) {
                const long long Q0a = (c.beg >> 2) & ~3ll, Q1 = (c.beg + c.d + 3) >> 2;
                const long long qa = Q0a + (long long)j * H.seg_q;
                sel = exact_find(g, c, qa, min(Q1, qa + H.seg_q), c.beg + c.d, r, lane, win);
            }
        }
    }
    if (lane == 0) {
        const int s = H.slot;
        if (sel < 0) {
            __threadfence_block();
            *(volatile int*)&sm.state[s] = ST_FINISH;
        } else {
            cnt.step(c.d, c.algo, true);
            commit(g, sm, R, s, c, __ldg(g.col + c.beg + sel), oz);
        }
        __threadfence_block();
        atomicExch(&H.ctl, (unsigned)H_FREE << 24);
    }
    __syncwarp();
}

// Claim one segment of an open hub task: (h, j) = task, segment; false if
// none is open.  Warp-collective, uniform result.
template <int NT>
__device__ __forceinline__ bool hub_claim(Smem<NT>& sm, int lane, int& h, int& j) {
    h = -1;
    j = -1;
    if (lane == 0) {
        for (int i = 0; i < NHUB; ++i) {
            HubTask& H = sm.hub[i];
            const unsigned v = *(volatile unsigned*)&H.ctl;
            if ((v >> 24) != H_ACTIVE || (int)(v & H_SEG_MASK) >= *(volatile int*)&H.nseg) continue;
            const unsigned old = atomicAdd(&H.ctl, 1u);
            // a claim counts only if the task was live then; the task cannot
            // be freed before this segment is done, so its fields stay valid
            if ((old >> 24) == H_ACTIVE) {
                __threadfence_block();
                const int jj = (int)(old & H_SEG_MASK);
                if (jj < H.nseg) {
                    h = i;
                    j = jj;
                    break;
                }
            }
        }
    }
    h = __shfl_sync(FULL, h, 0);
    j = __shfl_sync(FULL, j, 0);
    if (h >= 0) __threadfence_block();
    return h >= 0;
}

// Fold a sampled segment into its hub task; the warp that completes the last
// segment finishes the step.  Warp-collective.
template <int MODE, int NT>
__device__ __forceinline__ void hub_merge(const GraphDev& g, Smem<NT>& sm, HubTask& H, int j, const WarpRes& res,
                                          unsigned long long lane_sum, int lane, int* win, Counters& cnt) {
    if (MODE == MODE_FAST) {
        if (lane == 0 && res.sel >= 0) atomicMin(&H.best, race_key(res));
    } else {
        const unsigned long long s = warp_sum_u64(lane_sum);
        if (lane == 0) H.seg_sum[j] = s;
    }
    int last = 0;
    if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&H.done_seg, 1) == H.nseg - 1;
    }
    last = __shfl_sync(FULL, last, 0);
    if (last) {
        __threadfence_block();
        hub_finalize<MODE, NT>(g, sm, H, lane, win, cnt);
    }
}

// Per-warp dynamic shared memory: the TMA ring, the node2vec window, (exact
// mode) the chunk sums, the ring's barriers and the membership mask.
template <int MODE>
struct WarpSmem {
    static constexpr int WIN_OFF = NST * STAGE_BYTES;
    static constexpr int SUMS_OFF = WIN_OFF + WIN * 4;
    static constexpr int BAR_OFF = SUMS_OFF + (MODE == MODE_EXACT ? NCHUNK_MAX * 8 : 0);
    static constexpr int MASK_OFF = BAR_OFF + NST * 8;
    static constexpr int BYTES = (MASK_OFF + 4 * SQ + 127) & ~127;
};

// ------------------------------------------------------------- the engine

// Resident CTAs per SM the register budget is cut for.  The default
// 512-thread build keeps 128 registers a thread (16 warps per SM, no
// spills); the 256- and 128-thread builds take 24 and 20 warps per SM at 80
// and 96 registers, with spills, and measured slower on node2vec.
constexpr int min_ctas(int nt) { return nt >= 512 ? 1 : (nt >= 256 ? 3 : 5); }

// SERVE: the served form's build (queries claimed from the request ring,
// completion stamps, idle polling); the batch build compiles all of that
// out, which keeps its instruction footprint smaller.
template <int MODE, int NT, bool SERVE>
__global__ void __launch_bounds__(NT, min_ctas(NT)) walk_kernel(GraphDev g, const __grid_constant__ ReqTable tab, int n_req,
                                                  long long total, unsigned long long* cursor,
                                                  unsigned long long* counters, int sw, int d_t, int seg_q,
                                                  ServeDev sv) {
    constexpr bool serving = SERVE;
    const ReqDev* __restrict__ reqs = serving ? sv.ring : (tab.ext ? tab.ext : tab.r);
    __shared__ Smem<NT> sm;
    // dynamic shared memory per warp: the node2vec window (WIN ints) and, in
    // exact mode, the warp sampler's chunk sums
    extern __shared__ __align__(128) unsigned char dyn[];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    unsigned char* mine = dyn + warp * WarpSmem<MODE>::BYTES;
    int* win = reinterpret_cast<int*>(mine + WarpSmem<MODE>::WIN_OFF);
    unsigned long long* chunk_sums = reinterpret_cast<unsigned long long*>(mine + WarpSmem<MODE>::SUMS_OFF);
    WarpPipe P;
    P.buf = mine;
    P.bar = reinterpret_cast<unsigned long long*>(mine + WarpSmem<MODE>::BAR_OFF);
    P.mask = reinterpret_cast<unsigned*>(mine + WarpSmem<MODE>::MASK_OFF);
    P.st = 0;
    P.ph = 0;
    if (lane < NST) mbar_init(&P.bar[lane], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");

    for (int i = tid; i < Smem<NT>::NS; i += NT) sm.state[i] = ST_EMPTY;
    if (tid < NHUB) sm.hub[tid].ctl = (unsigned)H_FREE << 24;
    if (tid == 0) sm.abort_flag = 0;
    __syncthreads();

    Counters cnt;
    cnt.v = sm.cnt[warp];
    if (lane == 0) cnt.clear();
    const int s0 = warp * SW_MAX;
    bool exhausted = false;
    int rr = 0;
    unsigned long long idle_since = 0;
    unsigned nap = 128;  // idle back-off (ns)

    for (;;) {
        // ------------------------------------------------ choose the work
        // Either one segment of an open hub task (their owners are waiting,
        // so they come first) or one step of one of this warp's own walks.
        StepCtx c;
        long long qa, qb;
        uint64_t seed, qid;
        uint32_t t, stream;
        unsigned long long* sums = nullptr;
        int h, j;
        int s = -1;
        const ReqDev* R = nullptr;
        const bool seg = hub_claim<NT>(sm, lane, h, j);
        if (seg) {
            HubTask& H = sm.hub[h];
            c = H.c;
            const long long Q0a = (c.beg >> 2) & ~3ll, Q1 = (c.beg + c.d + 3) >> 2;
            qa = Q0a + (long long)j * H.seg_q;
            qb = min(Q1, qa + H.seg_q);
            seed = H.seed;
            qid = H.qid;
            t = H.t;
            stream = (uint32_t)j;
        } else {
            // ---- pick a walk: refill empty slots, retire finished ones ----
            bool waiting = false;
            for (int i = 0; i < sw; ++i) {
                const int jj = s0 + (rr + i) % sw;
                // another warp may flip a hub-parked slot at any time: let
                // lane 0 read it once for the whole warp
                int st = __shfl_sync(FULL, lane == 0 ? *(volatile int*)&sm.state[jj] : 0, 0);
                if (st == ST_EMPTY && !exhausted) {
                    // claim one query (lane 0): r = its request, qi = its
                    // index inside the request; -1 if none
                    long long qi = -1;
                    int r = 0;
                    if (serving) {
                        // served form: the oldest published request with
                        // queries left hands out its next one; once the host
                        // asks the engine to stop, nothing new is claimed
                        if (lane == 0 && !*sv.stop) {
                            for (int tries = 0; tries < 64; ++tries) {
                                const unsigned long long h = *(volatile unsigned long long*)sv.head;
                                if ((long long)h >= *sv.pub_r) break;
                                const int rs = (int)(h % (unsigned long long)sv.maxr);
                                const unsigned long long old = atomicAdd(&sv.taken[rs], 1ull);
                                if (old < kTakenBase) {
                                    qi = (long long)(old + (unsigned long long)__ldcg(&sv.ring[rs].n_q) - kTakenBase);
                                    r = rs;
                                    break;
                                }
                                atomicCAS(sv.head, h, h + 1);  // exhausted: move the head on
                            }
                        }
                        qi = __shfl_sync(FULL, qi, 0);
                        if (qi < 0) continue;  // nothing published right now: the slot stays empty
                    } else {
                        long long gq = 0;
                        if (lane == 0) gq = (long long)atomicAdd(cursor, 1ull);
                        gq = __shfl_sync(FULL, gq, 0);
                        if (gq >= total) {
                            exhausted = true;
                        } else if (lane == 0) {
                            r = find_req(reqs, n_req, gq);
                            qi = gq - reqs[r].q_begin;
                        }
                    }
                    if (!exhausted) {
                        // the walk's own copy of its request (through L2: a
                        // served ring slot is rewritten between requests)
                        r = __shfl_sync(FULL, r, 0);
                        constexpr int RW = (int)(sizeof(ReqDev) / 8);
                        static_assert(sizeof(ReqDev) % 8 == 0 && RW <= 32, "request copy: one word per lane");
                        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&reqs[r]);
                        if (lane < RW)
                            reinterpret_cast<unsigned long long*>(&sm.rq[jj])[lane] = serving ? __ldcg(src + lane)
                                                                                               : src[lane];
                        __syncwarp();
                    }
                    if (!exhausted && lane == 0) {
                        const ReqDev& Rq = sm.rq[jj];
                        const int start = __ldcg(Rq.starts + qi);
                        const int pv = Rq.prev ? __ldcg(Rq.prev + qi) : -1;
                        const int t0 = Rq.step0 ? __ldcg(Rq.step0 + qi) : 0;
                        int lim = Rq.lengths ? __ldcg(Rq.lengths + qi) : Rq.max_len;
                        lim = min(lim, Rq.max_len);
                        sm.q[jj] = qi;
                        sm.req[jj] = r;
                        sm.k[jj] = 0;
                        if (start < 0 || start >= g.n || pv < -1 || pv >= g.n || t0 < 0) {
                            atomicAdd(&counters[C_BAD_INPUT], 1ull);
                            st = ST_FINISH;  // written out as an empty path
                        } else {
                            Rq.paths[qi * ((long long)Rq.max_len + 1)] = start;
                            sm.k[jj] = 1;
                            sm.cur[jj] = start;
                            sm.prev[jj] = pv;
                            sm.t[jj] = t0;
                            sm.lim[jj] = lim;
                            if (pv >= 0) {
                                const long long pb = __ldg(g.row_ptr + pv);
                                sm.pbeg[jj] = pb;
                                sm.pdeg[jj] = (int)(__ldg(g.row_ptr + pv + 1) - pb);
                            } else {
                                sm.pbeg[jj] = 0;
                                sm.pdeg[jj] = 0;
                            }
                            st = ST_READY;
                        }
                        sm.state[jj] = st;
                    }
                    __syncwarp();
                    st = __shfl_sync(FULL, lane == 0 ? *(volatile int*)&sm.state[jj] : 0, 0);
                }
                if (st == ST_FINISH) {
                    // retire: path_len and -1 padding
                    const ReqDev& Rq = sm.rq[jj];
                    const long long width = (long long)Rq.max_len + 1;
                    const int k = sm.k[jj];
                    int32_t* row = Rq.paths + sm.q[jj] * width;
                    for (long long e = k + lane; e < width; e += 32) row[e] = -1;
                    if (lane == 0) {
                        Rq.path_len[sm.q[jj]] = k;
                        cnt.v[C_WALKS] += 1;
                        sm.state[jj] = ST_EMPTY;
                        if (serving) {
                            // the request's last walk tells the host (all its
                            // writes are visible first)
                            __threadfence();
                            const int rs = sm.req[jj];
                            if (atomicAdd(&sv.done[rs], 1ull) + 1 == (unsigned long long)Rq.n_q) {
                                __threadfence_system();
                                sv.complete[rs] = global_timer_ns() | 1ull;
                            }
                        }
                    }
                    __syncwarp();
                    --i;  // revisit this slot: it can be refilled now
                    continue;
                }
                if (st == ST_HUB) waiting = true;
                if (st == ST_READY) {
                    s = jj;
                    rr = (jj - s0 + 1) % sw;
                    break;
                }
            }
            if (s < 0 && !waiting && serving) {
                // served form with nothing to do: poll for new requests,
                // backing off up to 32 us; return once the host asks to stop,
                // or (bounded wait) after 2 s without any work
                int quit = 0;
                if (lane == 0) {
                    const unsigned long long now = global_timer_ns();
                    quit = *sv.stop;
                    if (idle_since == 0) idle_since = now;
                    else if (now - idle_since > kWaitLimitNs) quit = 1;
                }
                if (__shfl_sync(FULL, quit, 0)) break;
                __nanosleep(nap);
                nap = min(nap * 2u, 32768u);
                continue;
            }
            if (s < 0) {
                if (!waiting) break;  // all slots empty and no more queries
                // only hub-parked walks left: help (above) or wait for them, bounded
                if (idle_since == 0) {
                    idle_since = global_timer_ns();
                } else if (__shfl_sync(FULL, (int)(global_timer_ns() - idle_since > kWaitLimitNs), 0)) {
                    if (lane == 0) {
                        atomicAdd(&counters[C_TIMEOUT], 1ull);
                        sm.abort_flag = 1;
                    }
                    break;
                }
                if (__shfl_sync(FULL, lane == 0 ? *(volatile int*)&sm.abort_flag : 0, 0)) break;
                // back off while nothing turns up: an idle warp's polling
                // takes issue slots from the warps that are scanning
                __nanosleep(nap);
                nap = min(nap * 2u, 1024u);
                continue;
            }

            // ---- one step of slot s ----
            R = &sm.rq[s];
            if (sm.t[s] >= sm.lim[s]) {
                if (lane == 0) sm.state[s] = ST_FINISH;
                __syncwarp();
                continue;
            }
            const int v = sm.cur[s];
            const long long beg = __ldg(g.row_ptr + v);
            const int d = (int)(__ldg(g.row_ptr + v + 1) - beg);
            if (d == 0) {  // dead end
                if (lane == 0) sm.state[s] = ST_FINISH;
                __syncwarp();
                continue;
            }
            c = make_ctx(sm, *R, s, beg, d);
            t = (uint32_t)sm.t[s];
            qid = (uint64_t)(R->q_id0 + sm.q[s]);
            seed = R->seed;
            const long long end = beg + d;
            qa = (beg >> 2) & ~3ll;  // chunk grid aligned to 16 entries
            qb = (end + 3) >> 2;

            // exact mode keeps one sum per 128-entry chunk: a row spanning
            // more chunks than that goes to the CTA sampler whatever d_t says
            const bool too_long = MODE == MODE_EXACT && qb - qa > (long long)CHQ * NCHUNK_MAX;
            if (d > d_t || too_long) {
                // publish as a CTA hub task, if a task entry is free
                int hh = -1;
                if (lane == 0) {
                    for (int i = 0; i < NHUB; ++i) {
                        const unsigned vv = *(volatile unsigned*)&sm.hub[i].ctl;
                        if ((vv >> 24) == H_FREE &&
                            atomicCAS(&sm.hub[i].ctl, vv, (unsigned)H_SETUP << 24) == vv) {
                            hh = i;
                            break;
                        }
                    }
                    if (hh >= 0) {
                        HubTask& H = sm.hub[hh];
                        const long long nq = qb - qa;
                        const long long sq = seg_quads(nq, seg_q);
                        H.slot = s;
                        H.seg_q = (int)sq;
                        H.nseg = (int)((nq + sq - 1) / sq);
                        H.done_seg = 0;
                        H.best = ~0ull;
                        H.c = c;
                        H.seed = seed;
                        H.qid = qid;
                        H.t = t;
                        sm.state[s] = ST_HUB;
                        __threadfence_block();
                        atomicExch(&H.ctl, (unsigned)H_ACTIVE << 24);
                    }
                }
                hh = __shfl_sync(FULL, hh, 0);
                if (hh >= 0) continue;  // the walk waits for the CTA sampler; go on with other work
                // no free task entry: the walk stays ready and is published
                // on a later visit, after this warp has helped the open tasks
                // (so a hub row is always sampled segment by segment with the
                // task's random streams, whoever finds the entry free)
                __nanosleep(nap);
                nap = min(nap * 2u, 1024u);
                continue;
            }
            stream = 0;
            if (MODE == MODE_EXACT) sums = chunk_sums;
        }
        idle_since = 0;
        nap = 128;

        // ------------------------------------ stream the row range (one site)
        // A hub segment or an exact-mode row is one range.  A fast-mode row
        // sampled by this warp alone is cut into the hub path's segments,
        // segment j drawing from random stream j, and the step keeps the
        // smallest (race time, index) over them, as a hub task's merge does.
        WarpRes res;
        unsigned long long lane_sum = 0;
        unsigned long long best = ~0ull;
        const long long end = c.beg + c.d;
        const long long sq = (MODE == MODE_FAST && !seg) ? seg_quads(qb - qa, seg_q) : qb - qa;
        bool scanned = true;
        for (long long sa = qa; sa < qb; sa += sq) {
            res.init();
            const long long sb = min(qb, sa + sq);
            bool ok;
            if constexpr (MODE == MODE_FAST)
                ok = scan_range_fast(g, c, sa, sb, lane, win, P, res, stream, seed, qid, t);
            else
                ok = scan_range<MODE>(g, c, sa, sb, end, lane, win, P, res, lane_sum, sums, stream, seed, qid, t);
            if (!ok) {
                scanned = false;
                break;
            }
            if (res.sel >= 0) best = min(best, race_key(res));
            ++stream;
        }
        if (!scanned) {
            if (lane == 0) atomicAdd(&counters[C_TIMEOUT], 1ull);
            break;
        }

        // ------------------------------------------------ use the result
        if (seg) {
            hub_merge<MODE, NT>(g, sm, sm.hub[h], j, res, lane_sum, lane, win, cnt);
            continue;
        }
        int sel = -1;
        uint32_t oz = 0xFFFFFFFFu;
        if (MODE == MODE_FAST) {
            sel = best == ~0ull ? -1 : (int)(best & 0xFFFFFFFFull);
            if (sel >= 0 && R->algo == FW_PPR) oz = step_block(seed, qid, t).z;
        } else {
            const unsigned long long W = warp_sum_u64(lane_sum);
            __syncwarp();
            if (W != 0) {
                const uint4 o = step_block(seed, qid, t);
                oz = o.z;
                const unsigned long long x = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
                unsigned long long r = __umul64hi(x, W);
                const int nch = (int)((qb - qa + CHQ - 1) / CHQ);
                const int ci = find_crossing(chunk_sums, nch, r, lane);
                if (ci >= 0) {  // always, as r < W; the guard keeps every read inside the row
                    const long long q0 = qa + (long long)CHQ * ci;
                    sel = exact_find(g, c, q0, min(qb, q0 + CHQ), end, r, lane, win);
                }
            }
        }
        if (lane == 0) {
            if (sel < 0) {
                sm.state[s] = ST_FINISH;  // nothing selectable: the walk stops here
            } else {
                cnt.step(c.d, c.algo, false);
                commit(g, sm, *R, s, c, __ldg(g.col + c.beg + sel), oz);
            }
        }
        __syncwarp();
    }
    if (lane == 0)
        for (int i = 0; i < C_NUM; ++i)
            if (cnt.v[i]) atomicAdd(&counters[i], cnt.v[i]);
}

template <int MODE, int NT>
cudaError_t launch_one(const GraphDev& g, const ReqTable& reqs, int n_req, int64_t total,
                       unsigned long long* cursor, unsigned long long* counters, const Tuning& tu,
                       cudaStream_t stream) {
    auto kern = walk_kernel<MODE, NT, false>;
    const size_t dyn = (size_t)(NT / 32) * WarpSmem<MODE>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (tu.ctas_per_sm > 0) per_sm = min(per_sm, tu.ctas_per_sm);
    const int sw = max(1, min(SW_MAX, tu.slots / (NT / 32)));
    long long grid = (long long)sms * per_sm;
    const long long need = (total + (long long)sw * (NT / 32) - 1) / ((long long)sw * (NT / 32));
    if (need < grid) grid = need > 0 ? need : 1;
    int d_t = tu.d_warp;
    if (MODE == MODE_EXACT) d_t = min(d_t, NCHUNK_MAX * 128 - 8);  // at most NCHUNK_MAX chunks
    ServeDev none;
    memset(&none, 0, sizeof none);
    kern<<<(unsigned)grid, NT, dyn, stream>>>(g, reqs, n_req, (long long)total, cursor, counters, sw, d_t,
                                              kSegQuads, none);
    return cudaGetLastError();
}

template <int MODE, int NT>
cudaError_t launch_serve_one(const GraphDev& g, const ServeDev& sv, Scratch* scratch, const Tuning& tu,
                             cudaStream_t stream) {
    auto kern = walk_kernel<MODE, NT, true>;
    const size_t dyn = (size_t)(NT / 32) * WarpSmem<MODE>::BYTES;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (tu.ctas_per_sm > 0) per_sm = min(per_sm, tu.ctas_per_sm);
    // The resident engine leaves room for other kernels: one CTA slot on
    // every SM (eight SMs when only one CTA fits).  Filling every SM would
    // hold back other streams' kernels for as long as the server runs, and
    // through the hardware queues streams share, the server's own copies
    // queued behind them.
    const long long grid = (long long)sms * per_sm - (per_sm > 1 ? sms : min(8, sms - 1));
    const int sw = max(1, min(SW_MAX, tu.slots / (NT / 32)));
    int d_t = tu.d_warp;
    if (MODE == MODE_EXACT) d_t = min(d_t, NCHUNK_MAX * 128 - 8);
    ReqTable tab;
    memset(&tab, 0, sizeof tab);
    kern<<<(unsigned)grid, NT, dyn, stream>>>(g, tab, 0, 0ll, &scratch->cursor, scratch->counters, sw, d_t,
                                              kSegQuads, sv);
    return cudaGetLastError();
}

}  // namespace

Tuning default_tuning() { return Tuning{512, 64, 65536, 0}; }

Tuning sanitize_tuning(Tuning t) {
    const Tuning d = default_tuning();
    if (t.block_threads != 128 && t.block_threads != 256 && t.block_threads != 512) t.block_threads = d.block_threads;
    if (t.slots <= 0) t.slots = 4 * (t.block_threads / 32);  // four walks per warp
    if (t.slots > (t.block_threads / 32) * SW_MAX) t.slots = (t.block_threads / 32) * SW_MAX;
    if (t.d_warp <= 0) t.d_warp = d.d_warp;
    if (t.d_warp < 128) t.d_warp = 128;
    if (t.d_warp > (1 << 30)) t.d_warp = 1 << 30;
    if (t.ctas_per_sm < 0) t.ctas_per_sm = 0;
    return t;
}

cudaError_t launch_serve(const GraphDev& g, int mode, const ServeDev& sv, Scratch* scratch, const Tuning& tune,
                         cudaStream_t stream) {
    const Tuning tu = sanitize_tuning(tune);
    const bool exact = mode == FW_EXACT;
    switch (tu.block_threads) {
        case 128:
            return exact ? launch_serve_one<MODE_EXACT, 128>(g, sv, scratch, tu, stream)
                         : launch_serve_one<MODE_FAST, 128>(g, sv, scratch, tu, stream);
        case 512:
            return exact ? launch_serve_one<MODE_EXACT, 512>(g, sv, scratch, tu, stream)
                         : launch_serve_one<MODE_FAST, 512>(g, sv, scratch, tu, stream);
        default:
            return exact ? launch_serve_one<MODE_EXACT, 256>(g, sv, scratch, tu, stream)
                         : launch_serve_one<MODE_FAST, 256>(g, sv, scratch, tu, stream);
    }
}

cudaError_t launch_walk(const GraphDev& g, int mode, const ReqTable& reqs, int n_req, int64_t total,
                        unsigned long long* cursor, unsigned long long* counters, const Tuning& tune,
                        cudaStream_t stream) {
    const Tuning tu = sanitize_tuning(tune);
    if (total <= 0) return cudaSuccess;
    const bool exact = mode == FW_EXACT;
    switch (tu.block_threads) {
        case 128:
            return exact ? launch_one<MODE_EXACT, 128>(g, reqs, n_req, total, cursor, counters, tu, stream)
                         : launch_one<MODE_FAST, 128>(g, reqs, n_req, total, cursor, counters, tu, stream);
        case 512:
            return exact ? launch_one<MODE_EXACT, 512>(g, reqs, n_req, total, cursor, counters, tu, stream)
                         : launch_one<MODE_FAST, 512>(g, reqs, n_req, total, cursor, counters, tu, stream);
        default:
            return exact ? launch_one<MODE_EXACT, 256>(g, reqs, n_req, total, cursor, counters, tu, stream)
                         : launch_one<MODE_FAST, 256>(g, reqs, n_req, total, cursor, counters, tu, stream);
    }
}

}  // namespace fw
