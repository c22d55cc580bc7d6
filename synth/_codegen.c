/*
 * Seeded construction of left-regular LDPC parity-check matrices (input data).
 *
 * This file builds INPUTS shared by the FP64 oracle and the CUDA library:
 * the parity-check matrix H is data handed to both sides, never a result
 * of the method.  It contains none of the reconciliation arithmetic.
 *
 * Construction (the code family the paper's experiment substitutes with
 * random regular codes, Sec. V; block subdivision of Sec. III-A):
 *   - n variable nodes, each of degree dv  -> dv*n sockets;
 *   - M check nodes; the first (dv*n - M*d_lo) checks have degree d_lo+1,
 *     the rest degree d_lo = floor(dv*n / M);
 *   - variable sockets are placed on check sockets by a seeded permutation
 *     (drawn by the caller and passed in), then double edges and edges on
 *     4-cycles are broken by socket swaps with uniformly drawn partner edges
 *     (splitmix64 stream, Steele/Lea/Flood 2014), at most `max_passes` passes;
 *   - repeated (check, variable) pairs still left (dense codes) are then
 *     swapped away on their own, so H is always a set of distinct pairs.
 * Swapping the variable ends of two edges keeps every node degree.
 *
 * The socket permutation can also be drawn here (synth_philox_permutation):
 * Philox-4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11: ten rounds of two 64x64
 * -> 128-bit products with the Weyl key schedule) keyed by (seed, 0) with a
 * counter that starts at 1, its 64-bit outputs taken in order and split into
 * two 32-bit draws low half first; a Fisher-Yates shuffle of 0..E-1 from the
 * last position down, position i swapped with a draw in [0, i] taken by masked
 * rejection (the smallest all-ones mask covering i; 32-bit draws while
 * i < 2^32).  These are the stream conventions of numpy's Philox bit generator
 * and Generator.permutation, so the C and numpy constructions give the same
 * matrix for the same seed (checked in the tests).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static uint64_t splitmix64(uint64_t *s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* ------------------------------------------------------ Philox-4x64-10 */
typedef struct {
    uint64_t key[2], ctr[4], buf[4];
    int pos;               /* next unread output of buf (4 = empty) */
    int has32;             /* a high 32-bit half is waiting */
    uint32_t half;
} synth_philox;

static void philox_block(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B97F4A7C15ULL; k1 += 0xBB67AE8584CAA73BULL; }
        const unsigned __int128 p0 = (unsigned __int128)0xD2E7470EE14C6C93ULL * c0;
        const unsigned __int128 p1 = (unsigned __int128)0xCA5A826395121157ULL * c2;
        const uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        const uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void philox_init(synth_philox *g, uint64_t seed) {
    memset(g, 0, sizeof(*g));
    g->key[0] = seed;
    g->pos = 4;
}

static uint64_t philox_next64(synth_philox *g) {
    if (g->pos == 4) {
        /* 256-bit counter incremented before each block */
        for (int i = 0; i < 4; ++i)
            if (++g->ctr[i] != 0) break;
        philox_block(g->ctr, g->key, g->buf);
        g->pos = 0;
    }
    return g->buf[g->pos++];
}

static uint32_t philox_next32(synth_philox *g) {
    if (g->has32) { g->has32 = 0; return g->half; }
    const uint64_t v = philox_next64(g);
    g->has32 = 1;
    g->half = (uint32_t)(v >> 32);
    return (uint32_t)v;
}

/* uniform integer in [0, hi] by masked rejection */
static uint64_t philox_interval(synth_philox *g, uint64_t hi) {
    if (hi == 0) return 0;
    uint64_t mask = hi;
    for (int sh = 1; sh < 64; sh <<= 1) mask |= mask >> sh;
    uint64_t v;
    if (hi <= 0xFFFFFFFFULL) {
        do { v = philox_next32(g) & mask; } while (v > hi);
    } else {
        do { v = philox_next64(g) & mask; } while (v > hi);
    }
    return v;
}

/* perm[0..E) = a uniformly random permutation of 0..E-1 drawn from `seed` */
void synth_philox_permutation(uint64_t seed, int64_t E, int32_t *perm) {
    synth_philox g;
    philox_init(&g, seed);
    for (int64_t i = 0; i < E; ++i) perm[i] = (int32_t)i;
    for (int64_t i = E - 1; i > 0; --i) {
        const int64_t j = (int64_t)philox_interval(&g, (uint64_t)i);
        const int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/* uniform integer in [0, bound) by rejection (no modulo bias) */
static uint64_t draw_below(uint64_t *s, uint64_t bound) {
    uint64_t lim = UINT64_MAX - (UINT64_MAX % bound);
    uint64_t r;
    do { r = splitmix64(s); } while (r >= lim);
    return r % bound;
}

/*
 * Mark every edge that is (a) a repeated variable inside one check or
 * (b) the edge (c_a, v) of a 4-cycle v - c_a - u - c_b - v found from v.
 * Returns the number of marked edges; bad[] gets 0/1 per edge.
 * Also returns in *n_cycles the number of (v, c_a, u) detections, which
 * counts each 4-cycle a bounded number of times (0 iff girth >= 6 and no
 * double edge).
 */
static int64_t find_bad(int32_t n, int32_t M, const int32_t *rp, const int32_t *ci,
                        int32_t *vptr, int32_t *vedge, int32_t *vfill,
                        int64_t *stamp, int32_t *stamp_chk, uint8_t *bad, int64_t *n_cycles) {
    int64_t E = rp[M];
    /* variable -> edges (CSC) */
    memset(vptr, 0, sizeof(int32_t) * (size_t)(n + 1));
    for (int64_t e = 0; e < E; ++e) vptr[ci[e] + 1]++;
    for (int32_t v = 0; v < n; ++v) vptr[v + 1] += vptr[v];
    memcpy(vfill, vptr, sizeof(int32_t) * (size_t)n);
    int32_t *chk_of_edge = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    for (int32_t c = 0; c < M; ++c)
        for (int32_t e = rp[c]; e < rp[c + 1]; ++e) {
            chk_of_edge[e] = c;
            vedge[vfill[ci[e]]++] = e;
        }
    memset(bad, 0, (size_t)E);
    int64_t nbad = 0, ncyc = 0;
    /* double edges: a variable appearing twice in one check */
    for (int32_t v = 0; v < n; ++v) stamp[v] = -1;
    for (int32_t c = 0; c < M; ++c)
        for (int32_t e = rp[c]; e < rp[c + 1]; ++e) {
            int32_t v = ci[e];
            if (stamp[v] == c) { if (!bad[e]) { bad[e] = 1; nbad++; } ncyc++; }
            stamp[v] = c;
        }
    /* 4-cycles: for each v, walk its checks; a neighbour u reached through two
       different checks closes a 4-cycle */
    for (int32_t u = 0; u < n; ++u) { stamp[u] = -1; stamp_chk[u] = -1; }
    for (int32_t v = 0; v < n; ++v) {
        for (int32_t k = vptr[v]; k < vptr[v + 1]; ++k) {
            int32_t ev = vedge[k];
            int32_t c = chk_of_edge[ev];
            for (int32_t e = rp[c]; e < rp[c + 1]; ++e) {
                int32_t u = ci[e];
                if (u == v) continue;
                if (stamp[u] == v && stamp_chk[u] != c) {
                    if (!bad[ev]) { bad[ev] = 1; nbad++; }
                    ncyc++;
                }
                stamp[u] = v;
                stamp_chk[u] = c;
            }
        }
    }
    free(chk_of_edge);
    *n_cycles = ncyc;
    return nbad;
}

/*
 * ci[E] on entry: variable index of each check socket (already permuted).
 * rp[M+1]: check row pointers (degrees fixed by the caller).
 * Returns the residual count of 4-cycle/double-edge detections after the
 * last pass (0 = girth >= 6), or -1 on allocation failure.
 */
int64_t synth_break_short_cycles(int32_t n, int32_t M, const int32_t *rp, int32_t *ci,
                                 uint64_t seed, int32_t max_passes) {
    int64_t E = rp[M];
    int32_t *vptr = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
    int32_t *vedge = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    int32_t *vfill = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int32_t *stamp_chk = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    uint8_t *bad = (uint8_t *)malloc((size_t)E);
    if (!vptr || !vedge || !vfill || !stamp || !stamp_chk || !bad) {
        free(vptr); free(vedge); free(vfill); free(stamp); free(stamp_chk); free(bad);
        return -1;
    }
    uint64_t s = seed ^ 0xD1B54A32D192ED03ULL;
    int64_t ncyc = 0;
    for (int32_t pass = 0; pass <= max_passes; ++pass) {
        int64_t nbad = find_bad(n, M, rp, ci, vptr, vedge, vfill, stamp, stamp_chk, bad, &ncyc);
        if (nbad == 0 || pass == max_passes) break;
        for (int64_t e = 0; e < E; ++e) {
            if (!bad[e]) continue;
            int64_t p = (int64_t)draw_below(&s, (uint64_t)E);
            int32_t t = ci[e]; ci[e] = ci[p]; ci[p] = t;
        }
    }
    /* dense codes keep 4-cycles that no swap removes, and the last 4-cycle swaps
       can leave repeated variables in a check: a parity-check matrix is a set of
       (check, variable) pairs, so swap those edges alone until none is left */
    for (int32_t pass = 0; pass < 100 * (max_passes + 1); ++pass) {
        int64_t nrep = 0;
        memset(bad, 0, (size_t)E);
        for (int32_t v = 0; v < n; ++v) stamp[v] = -1;
        for (int32_t c = 0; c < M; ++c)
            for (int32_t e = rp[c]; e < rp[c + 1]; ++e) {
                if (stamp[ci[e]] == c) { bad[e] = 1; nrep++; }
                stamp[ci[e]] = c;
            }
        if (nrep == 0) break;
        for (int64_t e = 0; e < E; ++e) {
            if (!bad[e]) continue;
            int64_t p = (int64_t)draw_below(&s, (uint64_t)E);
            int32_t t = ci[e]; ci[e] = ci[p]; ci[p] = t;
        }
        find_bad(n, M, rp, ci, vptr, vedge, vfill, stamp, stamp_chk, bad, &ncyc);
    }
    free(vptr); free(vedge); free(vfill); free(stamp); free(stamp_chk); free(bad);
    return ncyc;
}

/*
 * The whole construction: degrees, the Philox socket permutation, then the
 * cycle-breaking passes above.  rp [M + 1] and ci [dv n] are written.
 * Returns the residual detection count (0 = girth >= 6), or -1 on bad sizes
 * or allocation failure.
 */
int64_t synth_make_regular_code(uint64_t seed, int32_t n, int32_t M, int32_t dv, int32_t max_passes,
                                int32_t *rp, int32_t *ci) {
    const int64_t E = (int64_t)dv * n;
    if (n <= 0 || dv <= 0 || M <= 0 || M > E || E > INT32_MAX) return -1;
    const int64_t d_lo = E / M, n_hi = E - (int64_t)M * d_lo;
    rp[0] = 0;
    for (int32_t c = 0; c < M; ++c) rp[c + 1] = rp[c] + (int32_t)(d_lo + (c < n_hi ? 1 : 0));
    int32_t *perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    if (!perm) return -1;
    synth_philox_permutation(seed, E, perm);
    /* socket s belongs to variable s / dv */
    for (int64_t e = 0; e < E; ++e) ci[e] = perm[e] / dv;
    free(perm);
    return synth_break_short_cycles(n, M, rp, ci, seed, max_passes);
}
