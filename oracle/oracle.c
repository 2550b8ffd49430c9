/*
 * CPU oracle for the dynamic-graph random walk step (FlowWalker, arXiv 2404.08364).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline leg of the benchmark may load this library.  It shares no
 * code, header, table or constant generator with the CUDA path.
 *
 * Plain, slow, single-threaded C.  Each function names the passage it follows:
 *
 *   walk loop ............ Alg. 1 (initialisation phase, then selection phase,
 *                          repeated until Stop(Q)); Section 2.1.
 *   weighted step ........ Section 2.1: p(u) proportional to w(v, u).
 *   MetaPath ............. Eq. 1, weighted variant (multiply by w(v, u)).
 *   node2vec ............. Eq. 2, weighted variant; dist(v', u) = 1 is
 *                          decided by binary search in the sorted N(v')
 *                          (Appendix C.3 attributes the random accesses of
 *                          node2vec to this search).
 *   PPR .................. stop probability 0.2 after each move (Section 6.1,
 *                          "Datasets and Workloads"); a do-while as in Alg. 1.
 *   "no vertex selected" . Section 4.1: returning S[0] means nothing matched
 *                          (e.g. no MetaPath label fits); the walk stops.
 *   output layout ........ Section 5.2: results stored contiguously per query,
 *                          |P_G| x (L_max + 1) entries with the start vertex
 *                          first (Eq. 3's L_max + 1).
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - length L counts moves; a path stores L + 1 vertices, padded with -1;
 *   - node2vec factors: 1/a for u == v', 1 for u in N(v'), 1/b otherwise,
 *     tested in that order; a walk with no previous vertex takes a
 *     first-order weighted step (factor 1 for every neighbour);
 *   - MetaPath move t (0-based) needs label schema[t mod schema_len];
 *   - exact mode: integer weights and integer node2vec factors, one
 *     Philox-4x32-10 block per (seed, query, step); r = floor(x * W / 2^64)
 *     with x the low 64 bits of the block; the pick is the smallest i whose
 *     inclusive prefix sum exceeds r (inverse transform sampling without a
 *     stored prefix table);
 *   - PPR stops after a move when word 2 of the same block is below
 *     floor(p_stop * 2^32).
 *
 * Random numbers: Philox-4x32-10 from its published definition (Salmon,
 * Moraes, Dror, Shaw, "Parallel Random Numbers: As Easy as 1, 2, 3", SC'11).
 * Counter (t, q_lo, q_hi, 0), key (seed_lo, seed_hi).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_WEIGHTED 0
#define ORC_NODE2VEC 1
#define ORC_METAPATH 2
#define ORC_PPR 3

#define ORC_OK 0
#define ORC_EINVAL -1

/* ---------------------------------------------------------------- Philox */

/* One Philox-4x32 round: two 32x32->64 multiplications by the round
 * multipliers, the high halves xored with the other two words and the key,
 * then the words permuted (SC'11, Section 3 "Philox"). */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* Philox-4x32-10: ten rounds, the key advanced by the Weyl constants
 * (golden ratio, sqrt(3) - 1) between rounds. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    memcpy(out, c, sizeof c);
}

static void step_block(uint64_t seed, int64_t q, int32_t t, uint32_t out[4]) {
    uint32_t ctr[4] = {(uint32_t)t, (uint32_t)((uint64_t)q & 0xFFFFFFFFu),
                       (uint32_t)((uint64_t)q >> 32), 0u};
    uint32_t key[2] = {(uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

/* ---------------------------------------------------------- parameters */

typedef struct {
    /* exact-mode node2vec factors: S/a, S, S/b for one integer scale S */
    uint32_t n2v_ret_i, n2v_in_i, n2v_out_i;
    /* fast-mode node2vec factors as the float values 1/a, 1, 1/b */
    float n2v_ret, n2v_in, n2v_out;
    int32_t schema_len;
    int8_t schema[16];
    double ppr_stop;
} orc_params;

/* Is u in the sorted row N(v')?  Plain binary search. */
static int in_sorted_row(const int32_t* row, int64_t len, int32_t u) {
    int64_t lo = 0, hi = len;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (row[mid] < u) lo = mid + 1;
        else hi = mid;
    }
    return lo < len && row[lo] == u;
}

/* Node2vec class of neighbour u of the current vertex given prev = v':
 * 0 -> dist 0 (u == v'), 1 -> dist 1 (u in N(v')), 2 -> dist 2. */
static int n2v_class(const int64_t* row_ptr, const int32_t* col, int32_t prev, int32_t u) {
    if (u == prev) return 0;
    if (in_sorted_row(col + row_ptr[prev], row_ptr[prev + 1] - row_ptr[prev], u)) return 1;
    return 2;
}

/* Initialisation phase of Alg. 1 in exact mode: integer weight of every
 * neighbour of cur.  Fills wp[0..d) and returns d. */
static int64_t exact_weights(const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                             const int8_t* etype, int algo, const orc_params* p,
                             int32_t cur, int32_t prev, int32_t t, uint64_t* wp) {
    int64_t beg = row_ptr[cur], d = row_ptr[cur + 1] - beg;
    for (int64_t i = 0; i < d; ++i) {
        uint64_t wi = w[beg + i];
        if (algo == ORC_METAPATH) {
            int8_t want = p->schema[t % p->schema_len];
            if (etype[beg + i] != want) wi = 0;
        } else if (algo == ORC_NODE2VEC && prev >= 0) {
            int cls = n2v_class(row_ptr, col, prev, col[beg + i]);
            uint64_t f = cls == 0 ? p->n2v_ret_i : (cls == 1 ? p->n2v_in_i : p->n2v_out_i);
            wi *= f;
        }
        wp[i] = wi;
    }
    return d;
}

/* Selection phase, exact mode: smallest i with inclusive prefix sum > r. */
int64_t orc_pick(const uint64_t* wp, int64_t d, uint64_t r) {
    uint64_t prefix = 0;
    for (int64_t i = 0; i < d; ++i) {
        prefix += wp[i];
        if (prefix > r) return i;
    }
    return -1;
}

/* r = floor(x * W / 2^64), the 64-bit draw x mapped onto [0, W). */
uint64_t orc_scale_draw(uint64_t x, uint64_t W) {
    unsigned __int128 prod = (unsigned __int128)x * W;
    return (uint64_t)(prod >> 64);
}

uint32_t orc_ppr_threshold(double p_stop) {
    double t = p_stop * 4294967296.0;
    if (t <= 0.0) return 0u;
    if (t >= 4294967295.0) return 0xFFFFFFFFu;
    return (uint32_t)t; /* floor for positive values */
}

/* ------------------------------------------------------------- walking */

/*
 * Exact-mode walk of queries [0, n_q) (Alg. 1).  Query i uses global query id
 * q0 + i in the random-number counter.  lengths == NULL means every query
 * walks max_len moves; prev_in / step0 == NULL mean a fresh walk (no previous
 * vertex, step 0).  paths is n_q x (max_len + 1), padded with -1.
 */
int orc_walk_exact(int64_t n, const int64_t* row_ptr, const int32_t* col, const uint32_t* w,
                   const int8_t* etype, int algo, const orc_params* p,
                   const int32_t* starts, int64_t n_q, int64_t q0,
                   const int32_t* lengths, int32_t max_len, uint64_t seed,
                   const int32_t* prev_in, const int32_t* step0,
                   int32_t* paths, int32_t* path_len) {
    if (algo < 0 || algo > 3 || max_len < 0) return ORC_EINVAL;
    if (algo == ORC_METAPATH && (etype == NULL || p->schema_len <= 0 || p->schema_len > 16))
        return ORC_EINVAL;
    int64_t dmax = 0;
    for (int64_t v = 0; v < n; ++v) {
        int64_t d = row_ptr[v + 1] - row_ptr[v];
        if (d > dmax) dmax = d;
    }
    uint64_t* wp = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(dmax > 0 ? dmax : 1));
    if (!wp) return ORC_EINVAL;
    uint32_t t_stop = orc_ppr_threshold(algo == ORC_PPR ? p->ppr_stop : 0.0);
    int64_t width = (int64_t)max_len + 1;

    for (int64_t i = 0; i < n_q; ++i) {
        int32_t* path = paths + i * width;
        int32_t cur = starts[i];
        int32_t prev = prev_in ? prev_in[i] : -1;
        int32_t t = step0 ? step0[i] : 0;
        int32_t L = lengths ? lengths[i] : max_len;
        if (L > max_len) L = max_len;
        int64_t k = 0;
        path[k++] = cur;
        while (t < L) {
            int64_t d = exact_weights(row_ptr, col, w, etype, algo, p, cur, prev, t, wp);
            if (d == 0) break; /* dead end */
            uint64_t W = 0;
            for (int64_t j = 0; j < d; ++j) W += wp[j];
            if (W == 0) break; /* nothing selectable (Section 4.1, S[0]) */
            uint32_t o[4];
            step_block(seed, q0 + i, t, o);
            uint64_t x = (uint64_t)o[0] | ((uint64_t)o[1] << 32);
            uint64_t r = orc_scale_draw(x, W);
            int64_t sel = orc_pick(wp, d, r);
            int32_t next = col[row_ptr[cur] + sel];
            path[k++] = next;
            prev = cur;
            cur = next;
            ++t;
            if (algo == ORC_PPR && o[2] < t_stop) break;
        }
        path_len[i] = (int32_t)k;
        for (; k < width; ++k) path[k] = -1;
    }
    free(wp);
    return ORC_OK;
}

/*
 * Exact transition law from state (cur, prev, t): writes d weights and
 * returns d.  mode 0 = exact-mode integer weights (w_u32 and the integer
 * node2vec factors), stored in wexact; mode 1 = fast-mode weights (w_f32 and
 * the float factors) computed in double, stored in wfast.  The probability of
 * neighbour i is weight_i / sum(weights).
 */
int64_t orc_transition(const int64_t* row_ptr, const int32_t* col, const uint32_t* w_u32,
                       const float* w_f32, const int8_t* etype, int algo, const orc_params* p,
                       int mode, int32_t cur, int32_t prev, int32_t t,
                       uint64_t* wexact, double* wfast) {
    int64_t beg = row_ptr[cur], d = row_ptr[cur + 1] - beg;
    for (int64_t i = 0; i < d; ++i) {
        int32_t u = col[beg + i];
        int keep = 1;
        int cls = -1;
        if (algo == ORC_METAPATH) keep = etype[beg + i] == p->schema[t % p->schema_len];
        if (algo == ORC_NODE2VEC && prev >= 0) cls = n2v_class(row_ptr, col, prev, u);
        if (mode == 0) {
            uint64_t f = 1;
            if (cls >= 0) f = cls == 0 ? p->n2v_ret_i : (cls == 1 ? p->n2v_in_i : p->n2v_out_i);
            wexact[i] = keep ? (uint64_t)w_u32[beg + i] * f : 0;
        } else {
            double f = 1.0;
            if (cls >= 0) f = cls == 0 ? (double)p->n2v_ret : (cls == 1 ? (double)p->n2v_in : (double)p->n2v_out);
            wfast[i] = keep ? (double)w_f32[beg + i] * f : 0.0;
        }
    }
    return d;
}
