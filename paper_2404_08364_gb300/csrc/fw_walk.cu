// Persistent, degree-aware walk engine (FlowWalker Sections 4-5, re-designed
// for sm_103a).
//
// One CTA is an independent worker with a local task pool of `slots` walks in
// shared memory (Section 5.1's P_L).  Each iteration it
//   1. claims new queries for its empty slots from one global atomic cursor
//      (Section 5.2's global task pool P_G: the request arrays themselves,
//      nothing extra in global memory),
//   2. reads the row offsets of every active walk's current vertex and routes
//      the step by degree: d <= d_warp to a warp sampler, larger rows to the
//      CTA sampler (Section 5.1's two stages, d_t),
//   3. runs the warp samplers concurrently, one step per small task,
//   4. runs the CTA sampler on each large task in turn,
//   5. commits each move to the caller's path row and retires finished walks.
// A walk stays on its CTA for life; it moves between the warp and CTA
// samplers from step to step as the degree of its current vertex changes.
//
// Samplers (Section 4's selection phase, no O(d) buffer in global memory):
//   exact mode: W = sum of integer weights, r = floor(x * W / 2^64) from the
//     step's 64-bit Philox draw, pick = smallest i with inclusive prefix > r
//     (inverse transform sampling done in two passes over the row, the first
//     keeping per-segment sums in shared memory so the second re-reads one
//     segment only);
//   fast mode: a single pass of weighted reservoir sampling in its
//     exponential-race form, each lane running Efraimidis-Spirakis reservoir
//     sampling with exponential jumps over its share of the row (random draws
//     only when the reservoir changes, O(log d) per lane) and the lanes'
//     reservoirs merged by an arg-min over their race times.
#include <math.h>

#include "fw_internal.cuh"

namespace fw {
namespace {

constexpr int S_MAX = 128;   // slots per CTA, upper bound
constexpr int SUBMAX = 32;   // exact CTA sampler: segment sums kept per warp
constexpr int ST_EMPTY = 0, ST_ACTIVE = 1, ST_FINISH = 2;
constexpr int MODE_EXACT = 0, MODE_FAST = 1;

template <int NT>
struct __align__(16) Smem {
    long long q[S_MAX];      // local query index inside its request
    long long beg[S_MAX];    // row of cur
    long long pbeg[S_MAX];   // row of prev (node2vec)
    int req[S_MAX];
    int cur[S_MAX], prev[S_MAX], t[S_MAX], lim[S_MAX], k[S_MAX];
    int deg[S_MAX], pdeg[S_MAX];
    int state[S_MAX];
    int small_list[S_MAX], large_list[S_MAX], fin_list[S_MAX];
    int warp_empty[S_MAX / 32];
    int n_small, n_large, n_fin, n_active;
    unsigned long long claim_base;
    int claim_n, exhausted;
    // CTA sampler scratch
    unsigned long long red_sum[NT / 32];
    unsigned long long sub_sum[NT / 32][SUBMAX];
    float red_tau[NT / 32];
    int red_idx[NT / 32];
    int b_warp, b_sub, b_sel;
    unsigned long long b_r;
    unsigned int b_oz;
    unsigned long long cnt[C_NUM];
};

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan_u64(unsigned long long v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += n;
    }
    return v;
}

// arg-min over (tau, idx), ties to the smaller index; idx < 0 means "none".
__device__ __forceinline__ void warp_argmin(float& tau, int& idx) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float t2 = __shfl_xor_sync(0xffffffffu, tau, o);
        int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
        bool take = (i2 >= 0) && (idx < 0 || t2 < tau || (t2 == tau && i2 < idx));
        if (take) {
            tau = t2;
            idx = i2;
        }
    }
}

__device__ __forceinline__ float unit_open(uint32_t w) {
    // (0, 1): 24 random bits, centred in their cell
    return ((float)(w >> 8) + 0.5f) * (1.0f / 16777216.0f);
}

// Is u in the sorted row col[pb .. pb+pd)?  Plain binary search (v1).
__device__ __forceinline__ bool in_row(const int32_t* __restrict__ col, long long pb, int pd, int u) {
    int lo = 0, hi = pd;
    while (lo < hi) {
        int mid = (lo + hi) >> 1;
        int v = __ldg(col + pb + mid);
        if (v < u) lo = mid + 1;
        else hi = mid;
    }
    return lo < pd && __ldg(col + pb + lo) == u;
}

// Per-step view of one walk, held in registers by the lanes of its sampler.
struct StepCtx {
    long long beg;
    long long pbeg;
    int d;
    int pdeg;
    int prev;
    int algo;
    int want;   // MetaPath label for this move
    uint32_t fi[3];
    float ff[3];
};

__device__ __forceinline__ int n2v_class(const GraphDev& g, const StepCtx& c, int u) {
    if (u == c.prev) return 0;
    return in_row(g.col, c.pbeg, c.pdeg, u) ? 1 : 2;
}

__device__ __forceinline__ uint32_t weight_exact(const GraphDev& g, const StepCtx& c, int i) {
    const long long e = c.beg + i;
    uint32_t w = __ldg(g.w_u32 + e);
    if (c.algo == FW_METAPATH) {
        if (__ldg(g.etype + e) != c.want) w = 0;
    } else if (c.algo == FW_NODE2VEC && c.prev >= 0) {
        w *= c.fi[n2v_class(g, c, __ldg(g.col + e))];
    }
    return w;
}

__device__ __forceinline__ float weight_fast(const GraphDev& g, const StepCtx& c, int i) {
    const long long e = c.beg + i;
    float w = __ldg(g.w_f32 + e);
    if (c.algo == FW_METAPATH) {
        if (__ldg(g.etype + e) != c.want) w = 0.0f;
    } else if (c.algo == FW_NODE2VEC && c.prev >= 0) {
        w *= c.ff[n2v_class(g, c, __ldg(g.col + e))];
    }
    return w;
}

// One lane's weighted reservoir (exponential race with exponential jumps).
// tau = the lane's current minimum race time E_i / w_i (E_i ~ Exp(1)), sel its
// element; X = remaining weight before the next element beats tau.  An
// element with weight w beats the current minimum with probability
// 1 - exp(-w * tau), so the weight skipped before the next record is
// Exp(1) / tau; the record's own time is the race time conditioned on being
// below tau.
struct Reservoir {
    float tau;
    float X;
    int sel;
    uint32_t ctr;
    uint32_t spare0, spare1;
    bool has_spare;

    __device__ __forceinline__ void init() {
        tau = __int_as_float(0x7f800000);  // +inf
        X = 0.0f;
        sel = -1;
        ctr = 0;
        has_spare = false;
    }

    __device__ __forceinline__ void offer(int i, float w, uint64_t seed, uint64_t qid, uint32_t t,
                                          uint32_t lane) {
        if (!(w > 0.0f)) return;
        X -= w;
        if (X > 0.0f) return;
        uint32_t a, b;
        if (has_spare) {
            a = spare0;
            b = spare1;
            has_spare = false;
        } else {
            uint4 o = lane_block(seed, qid, t, lane, ctr++);
            a = o.x;
            b = o.y;
            spare0 = o.z;
            spare1 = o.w;
            has_spare = true;
        }
        const float u1 = unit_open(a), u2 = unit_open(b);
        float e;
        if (isinf(tau)) e = -logf(u1);
        else e = -log1pf(u1 * expm1f(-w * tau));
        tau = e / w;
        sel = i;
        X = -logf(u2) / tau;
    }
};

template <int NT>
__device__ __forceinline__ void count_step(Smem<NT>& sm, int d, int algo, bool warp_tier) {
    atomicAdd(&sm.cnt[C_STEPS], 1ull);
    atomicAdd(&sm.cnt[C_ROWS], (unsigned long long)d);
    atomicAdd(&sm.cnt[warp_tier ? C_WARP_STEPS : C_BLOCK_STEPS], 1ull);
    if (algo == FW_NODE2VEC) atomicAdd(&sm.cnt[C_PROBES], (unsigned long long)d);
    atomicAdd(&sm.cnt[C_ALGO_BYTES],
              (unsigned long long)(8ll * d + (algo == FW_METAPATH ? d : 0) + 16 + 4));
}

// Commit a move (one thread): append `next` to the path, advance the state,
// apply the PPR stop test and the length limit.
template <int NT>
__device__ __forceinline__ void commit(Smem<NT>& sm, const ReqDev& R, int s, int next, uint32_t oz) {
    const long long width = (long long)R.max_len + 1;
    const int k = sm.k[s];
    R.paths[sm.q[s] * width + k] = next;
    sm.k[s] = k + 1;
    sm.prev[s] = sm.cur[s];
    sm.pbeg[s] = sm.beg[s];
    sm.pdeg[s] = sm.deg[s];
    sm.cur[s] = next;
    const int t = sm.t[s] + 1;
    sm.t[s] = t;
    const bool stop = (R.algo == FW_PPR && oz < R.t_stop) || t >= sm.lim[s];
    if (stop) sm.state[s] = ST_FINISH;
}

template <int NT>
__device__ __forceinline__ StepCtx make_ctx(const Smem<NT>& sm, const ReqDev& R, int s) {
    StepCtx c;
    c.beg = sm.beg[s];
    c.d = sm.deg[s];
    c.pbeg = sm.pbeg[s];
    c.pdeg = sm.pdeg[s];
    c.prev = sm.prev[s];
    c.algo = R.algo;
    c.want = (R.algo == FW_METAPATH) ? (int)R.schema[sm.t[s] % R.schema_len] : -1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        c.fi[j] = R.fac_i[j];
        c.ff[j] = R.fac_f[j];
    }
    return c;
}

// ----------------------------------------------------------- warp samplers

template <int MODE, int NT>
__device__ void warp_step(const GraphDev& g, const ReqDev* __restrict__ reqs, Smem<NT>& sm, int s,
                          uint32_t* __restrict__ wbuf, int lane) {
    const ReqDev& R = reqs[sm.req[s]];
    const StepCtx c = make_ctx(sm, R, s);
    const uint32_t t = (uint32_t)sm.t[s];
    const uint64_t qid = (uint64_t)(R.q_id0 + sm.q[s]);
    int sel = -1;
    uint32_t oz = 0xFFFFFFFFu;
    if (MODE == MODE_EXACT) {
        unsigned long long sum = 0;
        for (int i = lane; i < c.d; i += 32) {
            const uint32_t w = weight_exact(g, c, i);
            wbuf[i] = w;
            sum += w;
        }
        const unsigned long long W = warp_sum_u64(sum);
        __syncwarp();
        if (W != 0) {
            const uint4 o = step_block(R.seed, qid, t);
            oz = o.z;
            const unsigned long long x = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
            const unsigned long long r = __umul64hi(x, W);
            unsigned long long run = 0;
            for (int base = 0; base < c.d; base += 32) {
                const int i = base + lane;
                const unsigned long long v = (i < c.d) ? wbuf[i] : 0ull;
                const unsigned long long incl = warp_incl_scan_u64(v, lane);
                const unsigned m = __ballot_sync(0xffffffffu, run + incl > r);
                if (m) {
                    sel = base + __ffs(m) - 1;
                    break;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
    } else {
        Reservoir res;
        res.init();
        for (int i = lane; i < c.d; i += 32) res.offer(i, weight_fast(g, c, i), R.seed, qid, t, lane);
        float tau = res.tau;
        int idx = res.sel;
        warp_argmin(tau, idx);
        sel = idx;
        if (sel >= 0 && R.algo == FW_PPR) oz = step_block(R.seed, qid, t).z;
    }
    if (lane == 0) {
        if (sel < 0) {
            sm.state[s] = ST_FINISH;  // nothing selectable: the walk stops here
        } else {
            count_step(sm, c.d, c.algo, true);
            commit(sm, R, s, __ldg(g.col + c.beg + sel), oz);
        }
    }
    __syncwarp();
}

// ------------------------------------------------------------ CTA sampler

template <int MODE, int NT>
__device__ void block_step(const GraphDev& g, const ReqDev* __restrict__ reqs, Smem<NT>& sm, int s) {
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const ReqDev& R = reqs[sm.req[s]];
    const StepCtx c = make_ctx(sm, R, s);
    const uint32_t t = (uint32_t)sm.t[s];
    const uint64_t qid = (uint64_t)(R.q_id0 + sm.q[s]);
    // warp w owns the contiguous segment [w0, w1) of the row
    const int seg = ((c.d + NW - 1) / NW + 31) & ~31;
    const int w0 = min(c.d, warp * seg), w1 = min(c.d, w0 + seg);

    if (MODE == MODE_EXACT) {
        int sub = (seg + SUBMAX - 1) / SUBMAX;
        sub = max(256, (sub + 31) & ~31);
        unsigned long long total = 0;
        int j = 0;
        for (int a = w0; a < w1; a += sub, ++j) {
            const int b = min(w1, a + sub);
            unsigned long long sum = 0;
            for (int i = a + lane; i < b; i += 32) sum += weight_exact(g, c, i);
            sum = warp_sum_u64(sum);
            if (lane == 0) sm.sub_sum[warp][j] = sum;
            total += sum;
        }
        if (lane == 0) sm.red_sum[warp] = total;
        __syncthreads();
        if (tid == 0) {
            unsigned long long W = 0;
            for (int w = 0; w < NW; ++w) W += sm.red_sum[w];
            sm.b_warp = -1;
            sm.b_sel = -1;
            if (W != 0) {
                const uint4 o = step_block(R.seed, qid, t);
                sm.b_oz = o.z;
                const unsigned long long x = (unsigned long long)o.x | ((unsigned long long)o.y << 32);
                unsigned long long r = __umul64hi(x, W);
                // r < W, so both searches stop inside the arrays; the bounds
                // only guard against a logic error
                int w = 0;
                while (w < NW - 1 && r >= sm.red_sum[w]) r -= sm.red_sum[w++];
                const int ws0 = min(c.d, w * seg);
                const int nsub = (min(c.d, ws0 + seg) - ws0 + sub - 1) / sub;
                int jj = 0;
                while (jj < nsub - 1 && r >= sm.sub_sum[w][jj]) r -= sm.sub_sum[w][jj++];
                sm.b_warp = w;
                sm.b_sub = ws0 + jj * sub;  // first element of the segment
                sm.b_r = r;
            }
        }
        __syncthreads();
        if (warp == sm.b_warp) {
            const int a = sm.b_sub;
            const int b = min(min(c.d, warp * seg + seg), a + sub);
            const unsigned long long r = sm.b_r;
            unsigned long long run = 0;
            for (int base = a; base < b; base += 32) {
                const int i = base + lane;
                const unsigned long long v = (i < b) ? weight_exact(g, c, i) : 0ull;
                const unsigned long long incl = warp_incl_scan_u64(v, lane);
                const unsigned m = __ballot_sync(0xffffffffu, run + incl > r);
                if (m) {
                    if (lane == 0) sm.b_sel = base + __ffs(m) - 1;
                    break;
                }
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
        }
        __syncthreads();
    } else {
        Reservoir res;
        res.init();
        for (int i = w0 + lane; i < w1; i += 32) res.offer(i, weight_fast(g, c, i), R.seed, qid, t, tid);
        float tau = res.tau;
        int idx = res.sel;
        warp_argmin(tau, idx);
        if (lane == 0) {
            sm.red_tau[warp] = tau;
            sm.red_idx[warp] = idx;
        }
        __syncthreads();
        if (warp == 0) {
            float tt = lane < NW ? sm.red_tau[lane] : __int_as_float(0x7f800000);
            int ii = lane < NW ? sm.red_idx[lane] : -1;
            warp_argmin(tt, ii);
            if (lane == 0) {
                sm.b_sel = ii;
                sm.b_oz = (ii >= 0 && R.algo == FW_PPR) ? step_block(R.seed, qid, t).z : 0xFFFFFFFFu;
            }
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int sel = sm.b_sel;
        if (sel < 0) {
            sm.state[s] = ST_FINISH;
        } else {
            count_step(sm, c.d, c.algo, false);
            commit(sm, R, s, __ldg(g.col + c.beg + sel), sm.b_oz);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ int find_req(const ReqDev* __restrict__ reqs, int n_req, long long gq) {
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&reqs[mid].q_begin) <= gq) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ------------------------------------------------------------- the engine

template <int MODE, int NT>
__global__ void __launch_bounds__(NT) walk_kernel(GraphDev g, const __grid_constant__ ReqTable tab,
                                                  int n_req, long long total, Scratch* scratch,
                                                  int slots, int d_warp) {
    constexpr int NW = NT / 32;
    const ReqDev* __restrict__ reqs = tab.ext ? tab.ext : tab.r;
    __shared__ Smem<NT> sm;
    extern __shared__ __align__(16) uint32_t dyn[];  // exact mode: NW x d_warp weights
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    for (int s = tid; s < S_MAX; s += NT) sm.state[s] = ST_EMPTY;
    if (tid < C_NUM) sm.cnt[tid] = 0;
    if (tid == 0) sm.exhausted = 0;
    __syncthreads();

    for (;;) {
        // ---- 1. claim queries for empty slots (one atomic per CTA) ----
        {
            const bool empty = tid < slots && sm.state[tid] == ST_EMPTY;
            const unsigned m = __ballot_sync(0xffffffffu, empty);
            if (lane == 0 && warp < S_MAX / 32) sm.warp_empty[warp] = __popc(m);
            __syncthreads();
            if (tid == 0) {
                int n_empty = 0;
                for (int w = 0; w < (slots + 31) / 32; ++w) {
                    const int e = sm.warp_empty[w];
                    sm.warp_empty[w] = n_empty;  // exclusive prefix
                    n_empty += e;
                }
                sm.claim_n = 0;
                if (!sm.exhausted && n_empty > 0) {
                    const unsigned long long base = atomicAdd(&scratch->cursor, (unsigned long long)n_empty);
                    sm.claim_base = base;
                    if (base >= (unsigned long long)total) {
                        sm.exhausted = 1;
                    } else {
                        const unsigned long long left = (unsigned long long)total - base;
                        sm.claim_n = (int)(left < (unsigned long long)n_empty ? left : n_empty);
                        if (left <= (unsigned long long)n_empty) sm.exhausted = 1;
                    }
                }
                sm.n_small = sm.n_large = sm.n_fin = sm.n_active = 0;
            }
            __syncthreads();
            // ---- 2. initialise the claimed slots ----
            if (empty) {
                const int rank = sm.warp_empty[warp] + __popc(m & ((1u << lane) - 1u));
                if (rank < sm.claim_n) {
                    const long long gq = (long long)sm.claim_base + rank;
                    const int r = find_req(reqs, n_req, gq);
                    const ReqDev& R = reqs[r];
                    const long long i = gq - R.q_begin;
                    const int start = __ldg(R.starts + i);
                    const int pv = R.prev ? __ldg(R.prev + i) : -1;
                    const int t0 = R.step0 ? __ldg(R.step0 + i) : 0;
                    int lim = R.lengths ? __ldg(R.lengths + i) : R.max_len;
                    lim = min(lim, R.max_len);
                    sm.q[tid] = i;
                    sm.req[tid] = r;
                    sm.k[tid] = 0;
                    if (start < 0 || start >= g.n || pv < -1 || pv >= g.n || t0 < 0) {
                        atomicAdd(&scratch->counters[C_BAD_INPUT], 1ull);
                        sm.state[tid] = ST_FINISH;  // written out as an empty path
                    } else {
                        R.paths[i * ((long long)R.max_len + 1)] = start;
                        sm.k[tid] = 1;
                        sm.cur[tid] = start;
                        sm.prev[tid] = pv;
                        sm.t[tid] = t0;
                        sm.lim[tid] = lim;
                        if (pv >= 0) {
                            const long long pb = __ldg(g.row_ptr + pv);
                            sm.pbeg[tid] = pb;
                            sm.pdeg[tid] = (int)(__ldg(g.row_ptr + pv + 1) - pb);
                        } else {
                            sm.pbeg[tid] = 0;
                            sm.pdeg[tid] = 0;
                        }
                        sm.state[tid] = ST_ACTIVE;
                    }
                }
            }
        }
        // ---- 3. route every active walk by the degree of its vertex ----
        if (tid < slots) {
            int st = sm.state[tid];
            if (st == ST_ACTIVE) {
                if (sm.t[tid] >= sm.lim[tid]) {
                    st = ST_FINISH;
                } else {
                    const int v = sm.cur[tid];
                    const long long b = __ldg(g.row_ptr + v);
                    const long long d = __ldg(g.row_ptr + v + 1) - b;
                    sm.beg[tid] = b;
                    sm.deg[tid] = (int)d;
                    if (d == 0) st = ST_FINISH;  // dead end
                    else if (d <= d_warp) sm.small_list[atomicAdd(&sm.n_small, 1)] = tid;
                    else sm.large_list[atomicAdd(&sm.n_large, 1)] = tid;
                }
                sm.state[tid] = st;
            }
            if (st == ST_FINISH) sm.fin_list[atomicAdd(&sm.n_fin, 1)] = tid;
        }
        __syncthreads();
        if (sm.n_small + sm.n_large + sm.n_fin == 0 && sm.exhausted) break;

        // ---- 4. retire finished walks: path_len and -1 padding ----
        for (int f = warp; f < sm.n_fin; f += NW) {
            const int s = sm.fin_list[f];
            const ReqDev& R = reqs[sm.req[s]];
            const long long width = (long long)R.max_len + 1;
            const int k = sm.k[s];
            int32_t* row = R.paths + sm.q[s] * width;
            for (long long j = k + lane; j < width; j += 32) row[j] = -1;
            if (lane == 0) {
                R.path_len[sm.q[s]] = k;
                sm.state[s] = ST_EMPTY;
                atomicAdd(&sm.cnt[C_WALKS], 1ull);
            }
        }
        // ---- 5. warp samplers: one step for every small task ----
        for (int i = warp; i < sm.n_small; i += NW)
            warp_step<MODE, NT>(g, reqs, sm, sm.small_list[i], dyn + warp * d_warp, lane);
        __syncthreads();
        // ---- 6. CTA sampler: one step for each large task in turn ----
        const int nl = sm.n_large;
        for (int i = 0; i < nl; ++i) block_step<MODE, NT>(g, reqs, sm, sm.large_list[i]);
        __syncthreads();
    }
    if (tid < C_NUM && sm.cnt[tid]) atomicAdd(&scratch->counters[tid], sm.cnt[tid]);
}

template <int MODE, int NT>
cudaError_t launch_one(const GraphDev& g, const ReqTable& reqs, int n_req, int64_t total, Scratch* scratch,
                       const Tuning& tu, cudaStream_t stream) {
    auto kern = walk_kernel<MODE, NT>;
    const size_t dyn = MODE == MODE_EXACT ? (size_t)(NT / 32) * tu.d_warp * sizeof(uint32_t) : 0;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, dyn);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    if (tu.ctas_per_sm > 0) per_sm = min(per_sm, tu.ctas_per_sm);
    long long grid = (long long)sms * per_sm;
    const long long need = (total + tu.slots - 1) / tu.slots;
    if (need < grid) grid = need > 0 ? need : 1;
    kern<<<(unsigned)grid, NT, dyn, stream>>>(g, reqs, n_req, (long long)total, scratch, tu.slots,
                                                tu.d_warp);
    return cudaGetLastError();
}

}  // namespace

Tuning default_tuning() { return Tuning{256, 64, 1024, 0}; }

Tuning sanitize_tuning(Tuning t) {
    const Tuning d = default_tuning();
    if (t.block_threads != 128 && t.block_threads != 256 && t.block_threads != 512) t.block_threads = d.block_threads;
    if (t.slots <= 0) t.slots = d.slots;
    if (t.slots > S_MAX) t.slots = S_MAX;
    if (t.slots > t.block_threads) t.slots = t.block_threads;
    if (t.d_warp <= 0) t.d_warp = d.d_warp;
    if (t.d_warp > 4096) t.d_warp = 4096;
    t.d_warp = (t.d_warp + 31) & ~31;
    if (t.ctas_per_sm < 0) t.ctas_per_sm = 0;
    return t;
}

cudaError_t launch_walk(const GraphDev& g, int mode, const ReqTable& reqs, int n_req, int64_t total,
                        Scratch* scratch, const Tuning& tune, cudaStream_t stream) {
    const Tuning tu = sanitize_tuning(tune);
    if (total <= 0) return cudaSuccess;
    const bool exact = mode == FW_EXACT;
    switch (tu.block_threads) {
        case 128:
            return exact ? launch_one<MODE_EXACT, 128>(g, reqs, n_req, total, scratch, tu, stream)
                         : launch_one<MODE_FAST, 128>(g, reqs, n_req, total, scratch, tu, stream);
        case 512:
            return exact ? launch_one<MODE_EXACT, 512>(g, reqs, n_req, total, scratch, tu, stream)
                         : launch_one<MODE_FAST, 512>(g, reqs, n_req, total, scratch, tu, stream);
        default:
            return exact ? launch_one<MODE_EXACT, 256>(g, reqs, n_req, total, scratch, tu, stream)
                         : launch_one<MODE_FAST, 256>(g, reqs, n_req, total, scratch, tu, stream);
    }
}

}  // namespace fw
