// Parallel weighted samplers side by side (Section 4): the paper's direct
// parallel reservoir sampling (DPRS, Alg. 3) and zig-zag parallel reservoir
// sampling (ZPRS, Alg. 4), and the exponential-jump reservoir the walk engine
// uses (its fast mode), each run by a group of k threads (a warp, k = 32, or a
// CTA, k = 256) drawing one index from one weight array.
//
// Many independent draws run at once (one per sampler group, `reps` in all)
// over the same weights, so the timing measures the samplers' collective and
// random-number costs (Section 4's beta and gamma) rather than DRAM: every
// array here fits in L2.  Each draw r uses random counters of its own, so the
// returned indices are independent draws from w_i / sum(w).
#include <stdarg.h>
#include <stdio.h>

#include "fw_internal.cuh"

using namespace fw;

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int SAMP_EXPJ = 0, SAMP_DPRS = 1, SAMP_ZPRS = 2;

int fail_s(int status, const char* fmt, ...) {
    char buf[300];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(status, buf);
}

// uniform in [0, 1) from 24 random bits
__device__ __forceinline__ float unit24(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f); }
// uniform in (0, 1): 23 bits centred in their cell
__device__ __forceinline__ float unit_open23(uint32_t x) { return ((float)(x >> 9) + 0.5f) * (1.0f / 8388608.0f); }

// Per-element uniforms for thread j of draw r: one Philox block gives the
// uniforms of the thread's iterations 4c .. 4c + 3.
__device__ __forceinline__ uint4 elem_block(uint64_t seed, uint64_t r, uint32_t j, uint32_t c) {
    return philox4x32_10(make_uint4((uint32_t)r, (uint32_t)(r >> 32), j, c), make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}
__device__ __forceinline__ uint32_t pick_word(const uint4& b, int i) {
    return (i & 3) == 0 ? b.x : (i & 3) == 1 ? b.y : (i & 3) == 2 ? b.z : b.w;
}

// Group collectives for K = 32 (shuffles) or K = 256 (shuffles + shared).
template <int K>
struct Group {
    float* fbuf;   // K / 32 floats
    int* ibuf;     // K / 32 ints
    int tid;

    __device__ __forceinline__ void sync() {
        if (K == 32) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ float incl_scan(float v) {
        const int lane = tid & 31;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float n = __shfl_up_sync(FULL, v, o);
            if (lane >= o) v += n;
        }
        if (K == 32) return v;
        const int wp = tid >> 5;
        if (lane == 31) fbuf[wp] = v;
        __syncthreads();
        float before = 0.0f;
        for (int i = 0; i < wp; ++i) before += fbuf[i];
        __syncthreads();
        return v + before;
    }
    __device__ __forceinline__ float total(float incl) {
        if (K == 32) return __shfl_sync(FULL, incl, 31);
        __shared__ float t;
        if (tid == K - 1) t = incl;
        __syncthreads();
        const float r = t;
        __syncthreads();
        return r;
    }
    __device__ __forceinline__ int max_int(int v) {
        v = __reduce_max_sync(FULL, v);
        if (K == 32) return v;
        if ((tid & 31) == 0) ibuf[tid >> 5] = v;
        __syncthreads();
        int m = ibuf[0];
        for (int i = 1; i < K / 32; ++i) m = max(m, ibuf[i]);
        __syncthreads();
        return m;
    }
};

// DPRS (Alg. 3): per iteration, k consecutive weights, their inclusive
// prefix sum plus the weight of the earlier iterations (w_B), one uniform per
// element against w / (W_P + w_B), and the largest selected index so far.
template <int K>
__device__ int draw_dprs(Group<K>& G, const float* __restrict__ w, int64_t n, uint64_t seed, uint64_t r) {
    const int j = G.tid;
    float wB = 0.0f;
    int C = -1, selected = -1;
    uint4 blk = make_uint4(0, 0, 0, 0);
    const int64_t iters = (n + K - 1) / K;
    for (int64_t i = 0; i < iters; ++i) {
        const int64_t e = j + i * K;
        const float wl = e < n ? __ldg(w + e) : 0.0f;
        const float incl = G.incl_scan(wl);
        if ((i & 3) == 0) blk = elem_block(seed, r, (uint32_t)j, (uint32_t)(i >> 2));
        const float u = unit24(pick_word(blk, (int)(i & 3)));
        if (wl > 0.0f && u < wl / (incl + wB)) C = (int)e;
        selected = G.max_int(C);  // the algorithm reduces every iteration
        wB += G.total(incl);
    }
    return selected;
}

// ZPRS (Alg. 4): thread j sums its strided subsequence S_j, an exclusive
// prefix sum over the threads starts each running total, a second pass tests
// each element against w / (running total), and the selection of the highest
// thread that selected anything wins.
template <int K>
__device__ int draw_zprs(Group<K>& G, const float* __restrict__ w, int64_t n, uint64_t seed, uint64_t r) {
    const int j = G.tid;
    float s = 0.0f;
    for (int64_t e = j; e < n; e += K) s += __ldg(w + e);
    float P = G.incl_scan(s) - s;  // exclusive
    int C = -1;
    uint4 blk = make_uint4(0, 0, 0, 0);
    int64_t i = 0;
    for (int64_t e = j; e < n; e += K, ++i) {
        const float we = __ldg(w + e);
        P += we;
        if ((i & 3) == 0) blk = elem_block(seed, r, (uint32_t)j, (uint32_t)(i >> 2));
        const float u = unit24(pick_word(blk, (int)(i & 3)));
        if (we > 0.0f && u < we / P) C = (int)e;
    }
    const int top = G.max_int(C >= 0 ? j : -1);
    // broadcast the winner's C (K <= 256: through the group's int buffer)
    if (K == 32) return top < 0 ? -1 : __shfl_sync(FULL, C, top);
    if (j == top) G.ibuf[0] = C;
    __syncthreads();
    const int sel = top < 0 ? -1 : G.ibuf[0];
    __syncthreads();
    return sel;
}

// The engine's sampler: a warp's exponential race with exponential jumps
// over 128-entry chunks (prefix sum per chunk, a record only when the skip
// budget runs out), X kept as an FP32 two-sum; at CTA width each warp takes a
// contiguous segment with its own random stream and the smallest race time
// wins (ties: smaller index).
struct Race {
    float tau, Xh, Xl;
    int sel;
    uint32_t ctr;
};

__device__ __noinline__ Race race_record(Race R, int idx, float wv, uint64_t seed, uint64_t r, uint32_t stream) {
    const uint4 o = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)(r >> 32), 0x80000000u | stream, R.ctr++),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float u1 = unit_open23(o.x), u2 = unit_open23(o.y);
    float e;
    if (isinf(R.tau)) e = -logf(u1);
    else e = -log1pf(u1 * expm1f(-wv * R.tau));
    R.tau = e / wv;
    R.sel = idx;
    R.Xh = -logf(u2) / R.tau;
    R.Xl = 0.0f;
    return R;
}

__device__ Race race_segment(const float* __restrict__ w, int64_t a, int64_t b, int lane, uint64_t seed, uint64_t r,
                             uint32_t stream) {
    Race R;
    R.tau = __int_as_float(0x7f800000);
    R.Xh = 0.0f;
    R.Xl = 0.0f;
    R.sel = -1;
    R.ctr = 0;
    for (int64_t base = a; base < b; base += 128) {
        float wv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t e = base + lane * 4 + q;
            wv[q] = e < b ? __ldg(w + e) : 0.0f;
        }
        const float own = (wv[0] + wv[1]) + (wv[2] + wv[3]);
        float incl = own;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const float nb = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += nb;
        }
        const float tot = __shfl_sync(FULL, incl, 31);
        if (R.Xh - tot + R.Xl > 0.0f) {
            const float sh = R.Xh - tot;
            R.Xl += (R.Xh - sh) - tot;
            R.Xh = sh;
            continue;
        }
        float cum[4];
        cum[0] = (incl - own) + wv[0];
#pragma unroll
        for (int q = 1; q < 4; ++q) cum[q] = cum[q - 1] + wv[q];
        float target = R.Xh + R.Xl;
        int last = -1;
        for (;;) {
            int jj = -1;
#pragma unroll
            for (int q = 3; q >= 0; --q)
                if (lane * 4 + q > last && wv[q] > 0.0f && cum[q] >= target) jj = q;
            const unsigned m = __ballot_sync(FULL, jj >= 0);
            if (!m) {
                R.Xh = target - tot;
                R.Xl = 0.0f;
                break;
            }
            const int L = __ffs(m) - 1;
            float wj = 0.0f, cj = 0.0f;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (q == jj) {
                    wj = wv[q];
                    cj = cum[q];
                }
            const float wr = __shfl_sync(FULL, wj, L);
            const float cr = __shfl_sync(FULL, cj, L);
            const int jl = __shfl_sync(FULL, jj, L);
            last = L * 4 + jl;
            R = race_record(R, (int)(base + last), wr, seed, r, stream);
            target = cr + R.Xh;
        }
    }
    return R;
}

template <int K>
__device__ int draw_expj(Group<K>& G, const float* __restrict__ w, int64_t n, uint64_t seed, uint64_t r) {
    const int lane = G.tid & 31;
    if (K == 32) return race_segment(w, 0, n, lane, seed, r, 0).sel;
    // CTA width: K / 32 contiguous segments (multiples of 128 entries)
    const int wp = G.tid >> 5;
    const int64_t seg = ((n + K / 32 - 1) / (K / 32) + 127) / 128 * 128;
    const int64_t a = min(n, (int64_t)wp * seg), b = min(n, a + seg);
    const Race R = race_segment(w, a, b, lane, seed, r, (uint32_t)wp);
    __shared__ unsigned long long best;
    if (G.tid == 0) best = ~0ull;
    __syncthreads();
    if (lane == 0 && R.sel >= 0) atomicMin(&best, ((unsigned long long)__float_as_uint(R.tau) << 32) | (unsigned)R.sel);
    __syncthreads();
    const unsigned long long bv = best;
    __syncthreads();
    return bv == ~0ull ? -1 : (int)(bv & 0xFFFFFFFFull);
}

template <int METHOD, int K>
__global__ void __launch_bounds__(256) sampler_kernel(const float* __restrict__ w, int64_t n, int64_t reps,
                                                      uint64_t seed, int32_t* __restrict__ out) {
    __shared__ float fbuf[8];
    __shared__ int ibuf[8];
    Group<K> G;
    G.fbuf = fbuf;
    G.ibuf = ibuf;
    G.tid = (int)(threadIdx.x % K);
    const int groups = (int)(blockDim.x / K);
    const int gi = (int)(threadIdx.x / K);
    for (int64_t r = (int64_t)blockIdx.x * groups + gi; r < reps; r += (int64_t)gridDim.x * groups) {
        int sel;
        if (METHOD == SAMP_DPRS) sel = draw_dprs<K>(G, w, n, seed, (uint64_t)r);
        else if (METHOD == SAMP_ZPRS) sel = draw_zprs<K>(G, w, n, seed, (uint64_t)r);
        else sel = draw_expj<K>(G, w, n, seed, (uint64_t)r);
        if (G.tid == 0) out[r] = sel;
    }
}

template <int METHOD, int K>
cudaError_t launch_sampler(const float* w, int64_t n, int64_t reps, uint64_t seed, int32_t* out, cudaStream_t st) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sampler_kernel<METHOD, K>, 256, 0);
    if (e != cudaSuccess) return e;
    const int64_t groups = 256 / K;
    int64_t grid = (int64_t)sms * (per_sm > 0 ? per_sm : 1);
    const int64_t need = (reps + groups - 1) / groups;
    if (need < grid) grid = need;
    sampler_kernel<METHOD, K><<<(unsigned)grid, 256, 0, st>>>(w, n, reps, seed, out);
    return cudaGetLastError();
}

}  // namespace

extern "C" int fw_sampler_run(int32_t method, int32_t width, const float* d_w, int64_t n, int64_t reps,
                              uint64_t seed, int32_t* d_out, void* stream, float* ms) {
    if (!d_w || !d_out) return fail_s(FW_EINVAL, "fw_sampler_run: NULL weights or output");
    if (n < 1 || n > 0x7fffffffll || reps < 1) return fail_s(FW_EINVAL, "fw_sampler_run: n must be in [1, 2^31), reps >= 1");
    if (width != 32 && width != 256) return fail_s(FW_EINVAL, "fw_sampler_run: width must be 32 or 256");
    if (method < SAMP_EXPJ || method > SAMP_ZPRS) return fail_s(FW_EINVAL, "fw_sampler_run: unknown method");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    cudaError_t e;
    if (width == 32) {
        e = method == SAMP_DPRS   ? launch_sampler<SAMP_DPRS, 32>(d_w, n, reps, seed, d_out, st)
            : method == SAMP_ZPRS ? launch_sampler<SAMP_ZPRS, 32>(d_w, n, reps, seed, d_out, st)
                                  : launch_sampler<SAMP_EXPJ, 32>(d_w, n, reps, seed, d_out, st);
    } else {
        e = method == SAMP_DPRS   ? launch_sampler<SAMP_DPRS, 256>(d_w, n, reps, seed, d_out, st)
            : method == SAMP_ZPRS ? launch_sampler<SAMP_ZPRS, 256>(d_w, n, reps, seed, d_out, st)
                                  : launch_sampler<SAMP_EXPJ, 256>(d_w, n, reps, seed, d_out, st);
    }
    if (ms) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        *ms = t;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
    if (e != cudaSuccess) return fail_s(FW_ECUDA, "fw_sampler_run: %s", cudaGetErrorString(e));
    return FW_OK;
}
