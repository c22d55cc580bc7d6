// Bob's quantiser / bit slicing and Alice's slice LLRs (Sec. III-B steps 1-5).
#include <math.h>

#include "common.cuh"
#include "qkdrec_selftest.h"
#include "profile.cuh"

namespace qkd {

constexpr int kMaxM = 8;
constexpr int kMaxK = 1 << kMaxM;

// ------------------------------------------------------------------ quantiser
struct QuantParams {
    float tf[kMaxK];        // tf[i] = smallest float >= t_{i+1} (FP64 threshold), i < K-1
    uint8_t lab[kMaxK];     // label of interval k
    int32_t m, K;
};

// Interval k = number of thresholds t <= y.  Because y is a float,
// y >= t (FP64) is the same test as y >= tf (t rounded up to a float).
// NaN compares "not below" every threshold, so it lands in the last bin.
__global__ void quantise_kernel(const float *__restrict__ y, int64_t count, QuantParams p,
                                uint8_t *__restrict__ idx_out, uint8_t *__restrict__ bits_out,
                                unsigned long long *prof) {
    // per-lane table lookups diverge: stage the tables in shared memory
    __shared__ float tf[kMaxK];
    __shared__ uint8_t lab_s[kMaxK];
    for (int t = threadIdx.x; t < p.K; t += blockDim.x) {
        tf[t] = p.tf[t];
        lab_s[t] = p.lab[t];
    }
    __syncthreads();
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        ++units;
        float v = y[i];
        int k = 0;
        for (int s = p.K >> 1; s >= 1; s >>= 1)
            if (!(v < tf[k + s - 1])) k += s;
        if (idx_out) idx_out[i] = (uint8_t)k;
        if (bits_out) {
            int lab = lab_s[k];
            for (int j = 0; j < p.m; ++j) bits_out[(int64_t)j * count + i] = (uint8_t)((lab >> j) & 1);
        }
    }
    // y read, index and bit planes written
    prof_add(prof, units, units * (4 + (idx_out ? 1 : 0) + (bits_out ? p.m : 0)));
}

// ------------------------------------------------------------------ slice LLR
struct __align__(8) LlrParams {
    double td[kMaxK + 1];    // the same thresholds in FP64
    float tf[kMaxK + 1];     // t_0 .. t_K as floats (t_0 = -inf, t_K = +inf)
    uint8_t k_of_label[kMaxK];
    // the candidates of each lower-bit pattern `low` in increasing interval
    // order, cand[low nc + i] (nc = K >> j), and bit j of each interval's label
    uint8_t cand[kMaxK];
    uint8_t bitj[kMaxK];
    float inv_sigma;
    double inv_sigma_d;
    float ln_h;              // ln of the interval width in units of sigma_n
    float h;                 // the width itself
    float ln_half_n;         // ln (nc / 2): candidates per set
    float lo_f;              // quantiser origin t_0' = lo (thresholds lo + k delta)
    float inv_delta;         // 1 / delta: x in interval units
    float inv_h;             // sigma_n / delta
    float reach2;            // 2 (kSkipLinNats + ln sqrt(2 pi) - ln 2 - ln h): see llr_one
    int32_t m, K, j;
    int32_t all;             // 1: every candidate evaluated (llr_all), 0: a window of them (llr_one)
};

// Per-block tables derived from LlrParams in shared memory: each candidate as
// interval | bit_j << 8, and each interval's two bounds side by side.
struct LlrTables {
    uint16_t cb[kMaxK];
    float2 tf2[kMaxK];
};

__device__ __forceinline__ void llr_fill_tables(const LlrParams &p, LlrTables &t) {
    for (int i = threadIdx.x; i < p.K; i += blockDim.x) {
        const int k = p.cand[i];
        t.cb[i] = (uint16_t)(k | (p.bitj[k] << 8));
        t.tf2[i] = make_float2(p.tf[i], p.tf[i + 1]);
    }
}

// The derived tables of p from k_of_label, m, K, j, the quantiser step delta
// and inv_sigma (host side; the per-frame kernel fills the same fields itself).
constexpr float kSkipNats = 25.0f;   // terms below e^-25 of the set's nearest term are dropped
constexpr float kSkipLinNats = 16.0f;  // same, in the linear-domain sums (<= 2^m e^-16 relative)
constexpr float kLinDist = 9.0f;     // nearest terms within 9 sigma: P >= ~1e-19, sums in linear FP32
constexpr float kFarNats = 50.0f;    // both sets below e^-50: the set sums are redone in FP64
constexpr float kLn05 = -0.69314718055994531f;

__host__ __device__ inline void llr_scalars(LlrParams &p, double lo, double delta) {
    const double h = delta * p.inv_sigma_d;
    p.ln_h = (float)log(h);
    p.h = (float)h;
    p.ln_half_n = (float)log(0.5 * (double)(p.K >> p.j));
    p.lo_f = (float)lo;
    p.inv_delta = (float)(1.0 / delta);
    p.inv_h = (float)(1.0 / h);
    p.reach2 = (float)(2.0 * (kSkipLinNats + 0.91893853320467274 - 0.69314718055994531 - log(h)));
    // Evaluate every candidate when a typical window (nearest terms about h
    // away) would hold all but a few of them: finding the window costs about
    // as much as eight more terms (measured).
    const int nc = p.K >> p.j;
    const double span = 2.0 * sqrt(4.0 * h * h + (double)p.reach2) / h + 2.0;   // intervals
    const double in_window = fmin((double)nc, span * nc / p.K);
    p.all = nc <= in_window + 8.0 ? 1 : 0;
}

static void llr_tables(LlrParams &p, double lo, double delta) {
    const int nc = p.K >> p.j, lowmask = (1 << p.j) - 1;
    int fill[kMaxK] = {0};
    uint8_t lab_of_k[kMaxK];
    for (int l = 0; l < p.K; ++l) lab_of_k[p.k_of_label[l]] = (uint8_t)l;
    for (int k = 0; k < p.K; ++k) {
        const int low = lab_of_k[k] & lowmask;
        p.cand[low * nc + fill[low]++] = (uint8_t)k;
        p.bitj[k] = (uint8_t)((lab_of_k[k] >> p.j) & 1);
    }
    llr_scalars(p, lo, delta);
}


// log Q(z), z >= 0, through the scaled complement erfcx (no underflow at any z):
// Q(z) = erfc(z/sqrt 2)/2 = erfcx(z/sqrt 2) exp(-z^2/2)/2.
__device__ __forceinline__ float log_q32(float z) {
    if (isinf(z)) return -INFINITY;
    return logf(0.5f * erfcxf(z * 0.70710678118654752f)) - 0.5f * z * z;
}
__device__ __forceinline__ double log_q64(double z) {
    if (isinf(z)) return -INFINITY;
    return log(0.5 * erfcx(z * 0.70710678118654752440)) - 0.5 * z * z;
}

// log P(k | x) for standardised interval bounds a < b:
//   interval containing x : log(1 - Q(-a) - Q(b));
//   interval beside x     : near edge dn, far edge df on the same side,
//                           log(Q(dn) - Q(df)) = log Q(dn) + log(-expm1(log Q(df) - log Q(dn))).
__device__ __forceinline__ float logp32(float a, float b) {
    if (a < 0.0f && b > 0.0f) {
        const float r2 = 0.70710678118654752f;
        return log1pf(-0.5f * (erfcf(-a * r2) + erfcf(b * r2)));
    }
    const float dn = a >= 0.0f ? a : -b, df = a >= 0.0f ? b : -a;
    const float ln = log_q32(dn);
    return ln + logf(-expm1f(log_q32(df) - ln));
}
__device__ __forceinline__ double logp64(double a, double b) {
    if (a < 0.0 && b > 0.0) {
        const double r2 = 0.70710678118654752440;
        return log1p(-0.5 * (erfc(-a * r2) + erfc(b * r2)));
    }
    const double dn = a >= 0.0 ? a : -b, df = a >= 0.0 ? b : -a;
    const double ln = log_q64(dn);
    return ln + log(-expm1(log_q64(df) - ln));
}

// P(k | x) in linear FP32 for standardised bounds a < b, from the complementary
// error function on the side away from x (no cancellation except inside the
// containing interval, where P is at least the interval's width-scaled mass).
__device__ __forceinline__ float p_lin32(float a, float b) {
    const float r2 = 0.70710678118654752f;
    if (a >= 0.0f) return 0.5f * (erfcf(a * r2) - erfcf(b * r2));
    if (b <= 0.0f) return 0.5f * (erfcf(-b * r2) - erfcf(-a * r2));
    return 1.0f - 0.5f * (erfcf(-a * r2) + erfcf(b * r2));
}

// standardised distance from x to interval k (0 if x lies inside)
__device__ __forceinline__ float interval_dist(const LlrParams &p, int k, float x) {
    float a = (p.tf[k] - x) * p.inv_sigma;
    float b = (p.tf[k + 1] - x) * p.inv_sigma;
    return a >= 0.0f ? a : (b <= 0.0f ? -b : 0.0f);
}

__device__ __forceinline__ float lp_interval32(const LlrParams &p, int k, float x) {
    return logp32((p.tf[k] - x) * p.inv_sigma, (p.tf[k + 1] - x) * p.inv_sigma);
}
__device__ __forceinline__ double lp_interval64(const LlrParams &p, int k, double x) {
    return logp64((p.td[k] - x) * p.inv_sigma_d, (p.td[k + 1] - x) * p.inv_sigma_d);
}

// P(k | x) from the tails at its two bounds a < b (the same values p_lin32 forms):
// beside x above, T(a) - T(b); below, T(b) - T(a); containing x, 1 - T(a) - T(b).
__device__ __forceinline__ float p_from_tails(float a, float b, float Ta, float Tb) {
    return a >= 0.0f ? Ta - Tb : (b <= 0.0f ? Tb - Ta : 1.0f - Ta - Tb);
}

// Gaussian upper tail Q(z) = P(N(0,1) > z), z >= 0, of two values at once
// (packed FP32x2), from a fit of the Mills ratio M(z) = Q(z) sqrt(2 pi) e^{z^2/2}:
// Q(z) = e^{-z^2/2} r p(z r), r = 1/(z + 4), p the degree-8 polynomial that
// fit_tail.py fits to (z + 4) M(z) / sqrt(2 pi) on [0, 14] (5.7e-8 relative in
// exact arithmetic).  The exponent -z^2/2 log2 e is carried with the rounding
// errors of the square and of the product (FMA residuals), so the result stays
// within about 1.2e-6 relative on [0, 13]; from 14 on the tail is below the
// smallest normal float and the flushed exponential gives 0.
__device__ __forceinline__ float2 q_tail_fit2(float2 z) {
    const float kHi = -7.213475108e-01f, kLo = -9.629815168e-09f;
    z = make_float2(fminf(z.x, 14.0f), fminf(z.y, 14.0f));
    const float2 r = make_float2(rcp_approx(z.x + 4.0f), rcp_approx(z.y + 4.0f));
    const float2 sv = __fmul2_rn(z, r);
    float2 poly = __ffma2_rn(f2(1.028932724e-01f), sv, f2(-2.119122891e-01f));
    poly = __ffma2_rn(poly, sv, f2(-2.131454570e-01f));
    poly = __ffma2_rn(poly, sv, f2(7.901322532e-01f));
    poly = __ffma2_rn(poly, sv, f2(2.679492624e-01f));
    poly = __ffma2_rn(poly, sv, f2(-3.187017428e+00f));
    poly = __ffma2_rn(poly, sv, f2(5.233348686e+00f));
    poly = __ffma2_rn(poly, sv, f2(-4.383058265e+00f));
    poly = __ffma2_rn(poly, sv, f2(1.999999886e+00f));
    const float2 zz = __fmul2_rn(z, z);
    const float2 ez = __ffma2_rn(z, z, make_float2(-zz.x, -zz.y));
    const float2 e = __fmul2_rn(zz, f2(kHi));
    const float2 corr =
        __ffma2_rn(zz, f2(kLo), __ffma2_rn(ez, f2(kHi), __ffma2_rn(zz, f2(kHi), make_float2(-e.x, -e.y))));
    const float2 e0 = make_float2(ex2_approx(e.x), ex2_approx(e.y));
    return __fmul2_rn(__ffma2_rn(e0, __fmul2_rn(corr, f2(0.6931471805599453f)), e0), __fmul2_rn(poly, r));
}

// The log-domain sums for the rare samples whose nearest candidates are not
// both ordinary linear-domain terms (x far from every candidate of a set, as
// when the lower bits are wrong): FP32 relative to each set's nearest term, in
// FP64 when both sets lie beyond e^-50.  ub0, ub1 bound the sets' totals.
__device__ __noinline__ float llr_log_domain(const LlrParams &p, float x, int low, float ub0, float ub1, int kmin0,
                                             int kmin1) {
    const int nc = p.K >> p.j;
    const float lpn0 = lp_interval32(p, kmin0, x), lpn1 = lp_interval32(p, kmin1, x);
    const uint8_t *cand = p.cand + low * nc;
    float llr;
    if (ub1 < lpn0 - kLlrClip) {
        llr = kLlrClip;
    } else if (ub0 < lpn1 - kLlrClip) {
        llr = -kLlrClip;
    } else if (fmaxf(lpn0, lpn1) >= -kFarNats) {
        // FP32: sums relative to each set's nearest term
        float r0 = 1.0f, r1 = 1.0f;
        for (int i = 0; i < nc; ++i) {
            const int k = cand[i];
            const int b = p.bitj[k];
            if (k == (b ? kmin1 : kmin0)) continue;
            const float d = interval_dist(p, k, x);
            const float bound = d > 0.0f ? kLn05 - 0.5f * d * d : 0.0f;
            const float ref = b ? lpn1 : lpn0;
            if (bound < ref - kSkipNats) continue;
            const float t = expf(lp_interval32(p, k, x) - ref);
            if (b) r1 += t;
            else r0 += t;
        }
        llr = (lpn0 + logf(r0)) - (lpn1 + logf(r1));
    } else {
        // far Gaussian tails of both sets (x beyond e^-50 of every candidate):
        // the log-probabilities are large, so the difference is formed in FP64
        const double xd = (double)x;
        const double q0 = lp_interval64(p, kmin0, xd), q1 = lp_interval64(p, kmin1, xd);
        double r0 = 1.0, r1 = 1.0;
        for (int i = 0; i < nc; ++i) {
            const int k = cand[i];
            const int b = p.bitj[k];
            if (k == (b ? kmin1 : kmin0)) continue;
            const float d = interval_dist(p, k, x);
            const float bound = kLn05 - 0.5f * d * d;
            if (bound < (b ? lpn1 : lpn0) - kSkipNats) continue;
            const double t = exp(lp_interval64(p, k, xd) - (b ? q1 : q0));
            if (b) r1 += t;
            else r0 += t;
        }
        llr = (float)((q0 + log(r0)) - (q1 + log(r1)));
    }
    return fminf(fmaxf(llr, -kLlrClip), kLlrClip);
}


// Longest run of consecutive candidates (in interval order) with the same bit
// j: 2 under the Gray labelling (the candidates of a lower-bit pattern follow
// the pattern 0 1 1 0 0 1 1 ...), 1 under the binary one.  So the nearest
// candidate of each set lies within kSetRun + 1 positions of x's place.
constexpr int kSetRun = 2;

// First position in a candidate list (ascending intervals) whose interval is
// >= key; nc is a power of two.
__device__ __forceinline__ int cand_lower_bound(const uint16_t *cl, int nc, int key) {
    int pos = 0;
    for (int s = nc >> 1; s >= 1; s >>= 1)
        if ((cl[pos + s - 1] & 0xff) < key) pos += s;
    return pos + ((cl[pos] & 0xff) < key ? 1 : 0);
}

// LLR of one sample with every candidate of its lower bits evaluated in the
// linear domain (few candidates per sample).  Each term is accurate to about
// 1e-6 relative while its tails are normal floats (z below about 12.9) and
// loses precision or flushes to 0 beyond, an absolute error below the
// smallest normal float per term.  Once the larger sum is at least kLinFloor,
// a smaller sum within the clip (e^-30) of it keeps those errors below 3e-3
// relative for up to 2^11 candidates, under the 1e-4 |L| allowed at |L| near
// 30, and one further below only moves a clipped result.  With correct lower
// bits the set holding Bob's interval is within a few sigma of x (its sum near
// 1e-3 or more); otherwise the log-domain sums take over.
constexpr float kLinFloor = 1e-19f;
__device__ __forceinline__ float llr_all(const LlrParams &p, const LlrTables &tb, float x, int low) {
    const int nc = p.K >> p.j;
    const uint16_t *cl = tb.cb + low * nc;
    float s0 = 0.0f, s1 = 0.0f;
    for (int i = 0; i < nc; ++i) {
        const int e = cl[i], k = e & 0xff;
        const float2 tt = tb.tf2[k];
        const float a_ = (tt.x - x) * p.inv_sigma, b_ = (tt.y - x) * p.inv_sigma;
        const float2 T = q_tail_fit2(make_float2(fabsf(a_), fabsf(b_)));
        const float pk = p_from_tails(a_, b_, T.x, T.y);
        if (e >> 8) s1 += pk;
        else s0 += pk;
    }
    // ln(s0 / s1) from one MUFU logarithm; a set flushed to 0 gives +-inf, clipped
    if (fmaxf(s0, s1) >= kLinFloor)
        return fminf(fmaxf(lg2_approx(s0 * rcp_approx(s1)) * 0.6931471805599453f, -kLlrClip), kLlrClip);
    // far from every candidate: each set's nearest candidate, then the log domain
    float dmin0 = INFINITY, dmin1 = INFINITY;
    int kmin0 = 0, kmin1 = 0;
    for (int i = 0; i < nc; ++i) {
        const int e = cl[i], k = e & 0xff;
        const float d = interval_dist(p, k, x);
        if (e >> 8) {
            if (d < dmin1) { dmin1 = d; kmin1 = k; }
        } else if (d < dmin0) {
            dmin0 = d;
            kmin0 = k;
        }
    }
    const float ub0 = p.ln_half_n + (dmin0 > 0.0f ? kLn05 - 0.5f * dmin0 * dmin0 : 0.0f);
    const float ub1 = p.ln_half_n + (dmin1 > 0.0f ? kLn05 - 0.5f * dmin1 * dmin1 : 0.0f);
    return llr_log_domain(p, x, low, ub0, ub1, kmin0, kmin1);
}

// LLR of one sample (x, reconciled lower bits `low`) with the tables of p.
// The lanes of a warp run the common (linear-domain) case in step: each finds
// its window of candidates, the warp loops to the longest window.
__device__ __forceinline__ float llr_one(const LlrParams &p, const LlrTables &tb, float x, int low) {
    const int nc = p.K >> p.j;  // candidates consistent with the lower bits
    const uint16_t *cl = tb.cb + low * nc;
    // x's interval on the float thresholds (the number of t_1 .. t_{K-1} <= x):
    // from its position in interval units, corrected by one step either way
    const float top = (float)(p.K - 1);
    const float u = (x - p.lo_f) * p.inv_delta;
    int kx = (int)fminf(fmaxf(floorf(u), 0.0f), top);
    if (x < p.tf[kx]) --kx;
    else if (!(x < p.tf[kx + 1])) kx = min(kx + 1, p.K - 1);
    // x's place among the candidates; distances fall toward it from both
    // sides, so each set's nearest candidate lies in [px - kSetRun - 1, px + kSetRun]
    const int px = cand_lower_bound(cl, nc, kx);
    constexpr int kScan = 2 * kSetRun + 2;
    const int scan = min(nc, kScan);
    const int first = max(0, min(px - kSetRun - 1, nc - scan));
    float dmin0 = INFINITY, dmin1 = INFINITY;
    int kmin0 = 0, kmin1 = 0;
#pragma unroll
    for (int t = 0; t < kScan; ++t) {
        if (t >= scan) break;
        const int e = cl[first + t], k = e & 0xff;
        const float2 tt = tb.tf2[k];
        const float a_ = (tt.x - x) * p.inv_sigma, b_ = (tt.y - x) * p.inv_sigma;
        const float d = a_ >= 0.0f ? a_ : (b_ <= 0.0f ? -b_ : 0.0f);
        if (e >> 8) {
            if (d < dmin1) { dmin1 = d; kmin1 = k; }
        } else if (d < dmin0) {
            dmin0 = d;
            kmin0 = k;
        }
    }
    // bounds on each set's total: above, |K_b| x the largest term's bound
    // (Q(d) <= e^{-d^2/2} / 2 beside x, 1 inside); below, the nearest term alone,
    // which holds a strip of width h at most d + h from x: P >= h phi(d + h)
    const float h = p.h;
    const float ub0 = p.ln_half_n + (dmin0 > 0.0f ? kLn05 - 0.5f * dmin0 * dmin0 : 0.0f);
    const float ub1 = p.ln_half_n + (dmin1 > 0.0f ? kLn05 - 0.5f * dmin1 * dmin1 : 0.0f);
    const float lb0 = p.ln_h - 0.5f * (dmin0 + h) * (dmin0 + h) - 0.91893853f;
    const float lb1 = p.ln_h - 0.5f * (dmin1 + h) * (dmin1 + h) - 0.91893853f;
    // a set whose whole mass is provably more than the clip below the other's
    // cannot move the clipped result
    const bool sat_hi = ub1 < lb0 - kLlrClip;
    const bool sat_lo = !sat_hi && ub0 < lb1 - kLlrClip;
    const float dmx = fmaxf(dmin0, dmin1);
    const bool lin = !sat_hi && !sat_lo && dmx <= kLinDist;
    // Linear domain: both nearest terms are ordinary floats.  A term at distance
    // d is bounded by e^{-d^2/2}/2, below e^-16 of its set's lower bound once
    // d^2 > (d_set + h)^2 + reach2; the window holds every interval within that
    // reach of x for the farther set (so within it for both).
    int i0 = 0, cnt = 0;
    if (lin) {
        const float w = sqrtf((dmx + h) * (dmx + h) + p.reach2) * p.inv_h;   // in intervals
        const int klo = (int)fminf(fmaxf(floorf(u - w), 0.0f), top);
        const int khi = (int)fminf(fmaxf(floorf(u + w), 0.0f), top);
        i0 = cand_lower_bound(cl, nc, klo);
        cnt = cand_lower_bound(cl, nc, khi + 1) - i0;
    }
    const int steps = __reduce_max_sync(__activemask(), cnt);
    float s0 = 0.0f, s1 = 0.0f;
    for (int t = 0; t < steps; ++t) {
        const int e = cl[min(i0 + t, nc - 1)], k = e & 0xff;
        const float2 tt = tb.tf2[k];
        const float a_ = (tt.x - x) * p.inv_sigma, b_ = (tt.y - x) * p.inv_sigma;
        const float2 T = q_tail_fit2(make_float2(fabsf(a_), fabsf(b_)));
        float pk = p_from_tails(a_, b_, T.x, T.y);
        pk = t < cnt ? pk : 0.0f;
        if (e >> 8) s1 += pk;
        else s0 += pk;
    }
    if (sat_hi) return kLlrClip;
    if (sat_lo) return -kLlrClip;
    // ln(s0 / s1) from one MUFU logarithm (both sums hold their nearest term,
    // at least h phi(9 + h) > 0)
    if (lin) return fminf(fmaxf(lg2_approx(s0 * rcp_approx(s1)) * 0.6931471805599453f, -kLlrClip), kLlrClip);
    return llr_log_domain(p, x, low, ub0, ub1, kmin0, kmin1);
}

__global__ void slice_llr_kernel(const float *__restrict__ xs, int64_t count,
                                 const uint8_t *__restrict__ lower, const LlrParams p_in,
                                 float *__restrict__ out, unsigned long long *prof) {
    // per-lane table lookups diverge: stage the tables in shared memory
    __shared__ LlrParams sp;
    __shared__ LlrTables st;
    {
        const int n4 = (int)(sizeof(LlrParams) / 4);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&p_in);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
        for (int t = threadIdx.x; t < n4; t += blockDim.x) dst[t] = src[t];
    }
    llr_fill_tables(p_in, st);
    __syncthreads();
    const LlrParams &p = sp;
    int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        ++units;
        int low = 0;
        for (int b = 0; b < p.j; ++b) low |= (int)(lower[(int64_t)b * count + i] & 1) << b;
        out[i] = p.all ? llr_all(p, st, xs[i], low) : llr_one(p, st, xs[i], low);
    }
    // x and the lower bits read, the LLR written
    prof_add(prof, units, units * (8 + p.j));
}

// ------------------------------------------------- soft lower slices
// log P(b | L) for an LLR L = ln P(0)/P(1): z = L for b = 0, -L for b = 1;
// -log(1 + e^-z) = min(z, 0) - log1p(e^-|z|)  (z = +-inf allowed).
__device__ __forceinline__ float log_sigmoid(float z) { return fminf(z, 0.0f) - log1pf(expf(-fabsf(z))); }
__device__ __forceinline__ double log_sigmoid64(double z) { return fmin(z, 0.0) - log1p(exp(-fabs(z))); }

constexpr float kSoftSkipNats = 40.0f;   // terms below e^-40 of the largest bound are dropped
constexpr float kSoftLinNats = 10.0f;    // largest bound above e^-10: plain FP32 sums of P(k|x) w_k
constexpr float kSkipLinSoftNats = 20.0f;  // in those sums, terms bounded below e^-20 of the largest bound drop

// LLR of slice j with every interval weighted by the lower slices' bit
// probabilities: L = ln sum_{b_j(k)=0} P(k|x) w_k - ln sum_{b_j(k)=1} P(k|x) w_k,
// w_k = prod_{l<j} P(b_l(k) | L_l).  Log domain: a first pass bounds every term
// (log P(k|x) <= ln 1/2 - d^2/2 beside x, 0 inside), the second evaluates the
// terms within e^-40 of the largest bound (e^-20 in the plain sums; the bound is
// within a few nats of the exact term, so the dropped mass stays below 1e-5): as
// plain FP32 sums of P(k|x) w_k when that bound is above e^-10 (every such term lies within 10 sigma of x, so
// P(k|x) is an ordinary float), in the FP32 log domain below, in FP64 when the
// bound is below e^-50.
__device__ float llr_soft_one(const LlrParams &p, const uint8_t *lab_of_k, float x, const float *la,
                              const float *lb) {
    // pass 1: the largest bound of each set (b_j = 0, 1)
    float mub[2] = {-INFINITY, -INFINITY};
    for (int k = 0; k < p.K; ++k) {
        float prior = 0.0f;
        for (int l = 0; l < p.j; ++l) prior += ((lab_of_k[k] >> l) & 1) ? lb[l] : la[l];
        const float d = interval_dist(p, k, x);
        const int b = (lab_of_k[k] >> p.j) & 1;
        mub[b] = fmaxf(mub[b], (d > 0.0f ? kLn05 - 0.5f * d * d : 0.0f) + prior);
    }
    const float maxub = fmaxf(mub[0], mub[1]);
    // a set whose bound is more than the clip (plus the bound's slack) below the
    // other's cannot move the clipped result
    if (mub[1] < maxub - kSoftSkipNats) return kLlrClip;
    if (mub[0] < maxub - kSoftSkipNats) return -kLlrClip;
    const bool lin = maxub >= -kSoftLinNats;
    const bool wide = maxub < -kFarNats;
    const float cut0 = mub[0] - (lin ? kSkipLinSoftNats : kSoftSkipNats);
    const float cut1 = mub[1] - (lin ? kSkipLinSoftNats : kSoftSkipNats);
    // pass 2: the terms within reach of their own set's largest bound
    float t[2] = {0.0f, 0.0f}, m[2] = {-INFINITY, -INFINITY};
    double M[2] = {-INFINITY, -INFINITY}, S[2] = {0.0, 0.0};
    for (int k = 0; k < p.K; ++k) {
        float prior = 0.0f;
        for (int l = 0; l < p.j; ++l) prior += ((lab_of_k[k] >> l) & 1) ? lb[l] : la[l];
        const float d = interval_dist(p, k, x);
        const int b = (lab_of_k[k] >> p.j) & 1;
        if ((d > 0.0f ? kLn05 - 0.5f * d * d : 0.0f) + prior < (b ? cut1 : cut0)) continue;
        if (lin) {
            // every kept term lies within ~10 sigma of x: P(k|x) is an ordinary float
            t[b] += p_lin32((p.tf[k] - x) * p.inv_sigma, (p.tf[k + 1] - x) * p.inv_sigma) * expf(prior);
        } else if (!wide) {
            const float lw = lp_interval32(p, k, x) + prior;
            if (lw > m[b]) { t[b] = t[b] * expf(m[b] - lw) + 1.0f; m[b] = lw; }
            else t[b] += expf(lw - m[b]);
        } else {
            double prior64 = 0.0;
            for (int l = 0; l < p.j; ++l) prior64 += (double)(((lab_of_k[k] >> l) & 1) ? lb[l] : la[l]);
            const double lw = lp_interval64(p, k, (double)x) + prior64;
            if (lw > M[b]) { S[b] = S[b] * exp(M[b] - lw) + 1.0; M[b] = lw; }
            else S[b] += exp(lw - M[b]);
        }
    }
    float llr;
    if (lin) {
        llr = !(t[0] > 0.0f) ? -kLlrClip : (!(t[1] > 0.0f) ? kLlrClip : logf(t[0]) - logf(t[1]));
    } else if (!wide) {
        llr = !(t[0] > 0.0f) ? -kLlrClip : (!(t[1] > 0.0f) ? kLlrClip : (m[0] + logf(t[0])) - (m[1] + logf(t[1])));
    } else {
        llr = !(S[0] > 0.0) ? -kLlrClip
                            : (!(S[1] > 0.0) ? kLlrClip : (float)((M[0] + log(S[0])) - (M[1] + log(S[1]))));
    }
    return fminf(fmaxf(llr, -kLlrClip), kLlrClip);
}

__global__ void slice_llr_soft_kernel(const float *__restrict__ xs, int64_t count, const float *__restrict__ post,
                                      const LlrParams p_in, float *__restrict__ out, unsigned long long *prof) {
    __shared__ LlrParams sp;
    __shared__ uint8_t lab_of_k[kMaxK];
    {
        const int n4 = (int)(sizeof(LlrParams) / 4);
        const uint32_t *src = reinterpret_cast<const uint32_t *>(&p_in);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sp);
        for (int t = threadIdx.x; t < n4; t += blockDim.x) dst[t] = src[t];
        for (int t = threadIdx.x; t < p_in.K; t += blockDim.x) lab_of_k[p_in.k_of_label[t]] = (uint8_t)t;
    }
    __syncthreads();
    const LlrParams &p = sp;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    unsigned long long units = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        ++units;
        float la[kMaxM], lb[kMaxM];   // log P(bit 0 | L_l), log P(bit 1 | L_l)
        for (int l = 0; l < p.j; ++l) {
            const float L = post[(int64_t)l * count + i];
            la[l] = log_sigmoid(L);
            lb[l] = log_sigmoid(-L);
        }
        out[i] = llr_soft_one(p, lab_of_k, xs[i], la, lb);
    }
    // x and the lower LLRs read, the LLR written
    prof_add(prof, units, units * (8 + 4 * p.j));
}

// Known bits as certain LLRs: 0 -> +inf, 1 -> -inf.
__global__ void bits_to_llr_kernel(const uint8_t *__restrict__ bits, int64_t count, float *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride)
        out[i] = (bits[i] & 1) ? -INFINITY : INFINITY;
}

// ------------------------------------------- frames with their own parameters
// One block per frame: the block builds the frame's tables (thresholds from its
// quantiser range, its noise level) in shared memory, then walks its samples.
__global__ void quantise_frames_kernel(const float *__restrict__ y, const int64_t *__restrict__ off,
                                       const double *__restrict__ par, int64_t count, int32_t m, int32_t gray,
                                       uint8_t *__restrict__ idx_out, uint8_t *__restrict__ bits_out,
                                       unsigned long long *prof) {
    __shared__ float tf[kMaxK];
    __shared__ uint8_t lab_s[kMaxK];
    const int K = 1 << m;
    unsigned long long units = 0;
    const int64_t f = blockIdx.x;
    const double lo = par[2 * f], hi = par[2 * f + 1], delta = (hi - lo) / K;
    for (int t = threadIdx.x; t < K; t += blockDim.x) {
        // rounded like the host tables (no fused multiply-add): smallest float >= t_k
        if (t >= 1) tf[t - 1] = __double2float_ru(__dadd_rn(lo, __dmul_rn(delta, (double)t)));
        lab_s[t] = (uint8_t)(gray ? (t ^ (t >> 1)) : t);
    }
    __syncthreads();
    const int64_t ib = max(off[f], (int64_t)0), ie = min(off[f + 1], count);
    for (int64_t i = ib + threadIdx.x; i < ie; i += blockDim.x) {
        ++units;
        const float v = y[i];
        int k = 0;
        for (int s = K >> 1; s >= 1; s >>= 1)
            if (!(v < tf[k + s - 1])) k += s;
        if (idx_out) idx_out[i] = (uint8_t)k;
        if (bits_out) {
            const int lab = lab_s[k];
            for (int j = 0; j < m; ++j) bits_out[(int64_t)j * count + i] = (uint8_t)((lab >> j) & 1);
        }
    }
    prof_add(prof, units, units * (4 + (idx_out ? 1 : 0) + (bits_out ? m : 0)));
}

__global__ void slice_llr_frames_kernel(const float *__restrict__ xs, const int64_t *__restrict__ off,
                                        const double *__restrict__ par, int64_t count, int32_t m, int32_t j,
                                        int32_t gray, const uint8_t *__restrict__ lower, float *__restrict__ out,
                                        unsigned long long *prof) {
    __shared__ LlrParams sp;
    const int64_t f = blockIdx.x;
    const int K = 1 << m;
    const double lo = par[3 * f], hi = par[3 * f + 1], sn = par[3 * f + 2], delta = (hi - lo) / K;
    for (int t = threadIdx.x; t <= K; t += blockDim.x) {
        const double td = t == 0 ? -INFINITY : (t == K ? INFINITY : __dadd_rn(lo, __dmul_rn(delta, (double)t)));
        sp.td[t] = td;
        sp.tf[t] = (float)td;
        if (t < K) sp.k_of_label[gray ? (t ^ (t >> 1)) : t] = (uint8_t)t;
    }
    if (threadIdx.x == 0) {
        sp.inv_sigma = (float)(1.0 / sn);
        sp.inv_sigma_d = 1.0 / sn;
        sp.m = m;
        sp.K = K;
        sp.j = j;
        llr_scalars(sp, lo, delta);
    }
    if (threadIdx.x < K) {
        // candidate lists in interval order: interval k's rank among the
        // intervals sharing its lower label bits
        const int k = threadIdx.x, lowmask = (1 << j) - 1, nc = K >> j;
        const int lab = gray ? (k ^ (k >> 1)) : k, low = lab & lowmask;
        int rank = 0;
        for (int k2 = 0; k2 < k; ++k2) rank += ((gray ? (k2 ^ (k2 >> 1)) : k2) & lowmask) == low;
        sp.cand[low * nc + rank] = (uint8_t)k;
        sp.bitj[k] = (uint8_t)((lab >> j) & 1);
    }
    __syncthreads();
    __shared__ LlrTables st;
    llr_fill_tables(sp, st);
    __syncthreads();
    unsigned long long units = 0;
    const int64_t ib = max(off[f], (int64_t)0), ie = min(off[f + 1], count);
    for (int64_t i = ib + threadIdx.x; i < ie; i += blockDim.x) {
        ++units;
        int low = 0;
        for (int b = 0; b < j; ++b) low |= (int)(lower[(int64_t)b * count + i] & 1) << b;
        out[i] = sp.all ? llr_all(sp, st, xs[i], low) : llr_one(sp, st, xs[i], low);
    }
    prof_add(prof, units, units * (8 + j));
}

__global__ void gauss_tail_selftest_kernel(const float2 *__restrict__ z, int64_t pairs, float2 *__restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs; i += stride) {
        const float2 v = z[i];
        out[i] = q_tail_fit2(make_float2(fabsf(v.x), fabsf(v.y)));
    }
}

static int label_of(int k, qkdrec_label lab) { return lab == QKDREC_LABEL_BINARY ? k : (k ^ (k >> 1)); }

static float round_up_to_float(double t) {
    float f = (float)t;
    if ((double)f < t) f = nextafterf(f, INFINITY);
    return f;
}

static int grid_for(int64_t count, int block) {
    int64_t want = ceil_div(count, block);
    int64_t cap = (int64_t)sm_count() * 16;
    return (int)(want < cap ? (want > 0 ? want : 1) : cap);
}

}  // namespace qkd

using namespace qkd;

extern "C" {

qkdrec_status qkdrec_quantise_slices(const float *y, int64_t count, int32_t m, double lo, double hi,
                                     qkdrec_label label, uint8_t *idx_out, uint8_t *bits_out,
                                     void *stream) {
    clear_error();
    if (count < 0) QKD_FAIL(QKDREC_ERR_ARG, "count < 0");
    if (m < 1 || m > kMaxM) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, %d]", m, kMaxM);
    if (!(lo < hi)) QKD_FAIL(QKDREC_ERR_ARG, "need lo < hi");
    if (label != QKDREC_LABEL_GRAY && label != QKDREC_LABEL_BINARY) QKD_FAIL(QKDREC_ERR_ARG, "bad label");
    if (count == 0) return QKDREC_OK;
    if (!y) QKD_FAIL(QKDREC_ERR_ARG, "y is NULL");
    QuantParams p;
    p.m = m;
    p.K = 1 << m;
    const double delta = (hi - lo) / p.K;
    for (int k = 1; k < p.K; ++k) p.tf[k - 1] = round_up_to_float(lo + delta * k);
    for (int k = 0; k < p.K; ++k) p.lab[k] = (uint8_t)label_of(k, label);
    const int block = 256;
    prof::Scope ps(prof::kQuantise, as_stream(stream));
    quantise_kernel<<<grid_for(count, block), block, 0, as_stream(stream)>>>(y, count, p, idx_out, bits_out,
                                                                             prof::counters(prof::kQuantise));
    QKD_LAUNCHED("quantise_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_slice_llr(const float *x, int64_t count, int32_t m, int32_t j, double lo,
                               double hi, double sigma_n, qkdrec_label label,
                               const uint8_t *lower_bits, float *llr_out, void *stream) {
    clear_error();
    if (count < 0) QKD_FAIL(QKDREC_ERR_ARG, "count < 0");
    if (m < 1 || m > kMaxM) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, %d]", m, kMaxM);
    if (j < 0 || j >= m) QKD_FAIL(QKDREC_ERR_ARG, "slice j=%d outside [0, %d)", j, m);
    if (!(lo < hi) || !(sigma_n > 0)) QKD_FAIL(QKDREC_ERR_ARG, "need lo < hi and sigma_n > 0");
    if (label != QKDREC_LABEL_GRAY && label != QKDREC_LABEL_BINARY) QKD_FAIL(QKDREC_ERR_ARG, "bad label");
    if (count == 0) return QKDREC_OK;
    if (!x || !llr_out) QKD_FAIL(QKDREC_ERR_ARG, "x/llr_out NULL");
    if (j > 0 && !lower_bits) QKD_FAIL(QKDREC_ERR_ARG, "lower_bits NULL for j=%d", j);
    LlrParams p;
    p.m = m;
    p.K = 1 << m;
    p.j = j;
    const double delta = (hi - lo) / p.K;
    p.td[0] = -INFINITY;
    p.td[p.K] = INFINITY;
    for (int k = 1; k < p.K; ++k) p.td[k] = lo + delta * k;
    for (int k = 0; k <= p.K; ++k) p.tf[k] = (float)p.td[k];
    for (int k = 0; k < p.K; ++k) p.k_of_label[label_of(k, label)] = (uint8_t)k;
    p.inv_sigma = (float)(1.0 / sigma_n);
    p.inv_sigma_d = 1.0 / sigma_n;
    llr_tables(p, lo, delta);
    const int block = 128;
    prof::Scope ps(prof::kSliceLlr, as_stream(stream));
    slice_llr_kernel<<<grid_for(count, block), block, 0, as_stream(stream)>>>(x, count, lower_bits, p, llr_out,
                                                                              prof::counters(prof::kSliceLlr));
    QKD_LAUNCHED("slice_llr_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_slice_llr_soft(const float *x, int64_t count, int32_t m, int32_t j, double lo, double hi,
                                    double sigma_n, qkdrec_label label, const float *lower_post, float *llr_out,
                                    void *stream) {
    clear_error();
    if (count < 0) QKD_FAIL(QKDREC_ERR_ARG, "count < 0");
    if (m < 1 || m > kMaxM) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, %d]", m, kMaxM);
    if (j < 0 || j >= m) QKD_FAIL(QKDREC_ERR_ARG, "slice j=%d outside [0, %d)", j, m);
    if (!(lo < hi) || !(sigma_n > 0)) QKD_FAIL(QKDREC_ERR_ARG, "need lo < hi and sigma_n > 0");
    if (label != QKDREC_LABEL_GRAY && label != QKDREC_LABEL_BINARY) QKD_FAIL(QKDREC_ERR_ARG, "bad label");
    if (count == 0) return QKDREC_OK;
    if (!x || !llr_out) QKD_FAIL(QKDREC_ERR_ARG, "x/llr_out NULL");
    if (j > 0 && !lower_post) QKD_FAIL(QKDREC_ERR_ARG, "lower_post NULL for j=%d", j);
    LlrParams p;
    p.m = m;
    p.K = 1 << m;
    p.j = j;
    const double delta = (hi - lo) / p.K;
    p.td[0] = -INFINITY;
    p.td[p.K] = INFINITY;
    for (int k = 1; k < p.K; ++k) p.td[k] = lo + delta * k;
    for (int k = 0; k <= p.K; ++k) p.tf[k] = (float)p.td[k];
    for (int k = 0; k < p.K; ++k) p.k_of_label[label_of(k, label)] = (uint8_t)k;
    p.inv_sigma = (float)(1.0 / sigma_n);
    p.inv_sigma_d = 1.0 / sigma_n;
    const int block = 128;
    prof::Scope ps(prof::kSliceLlr, as_stream(stream));
    slice_llr_soft_kernel<<<grid_for(count, block), block, 0, as_stream(stream)>>>(
        x, count, lower_post, p, llr_out, prof::counters(prof::kSliceLlr));
    QKD_LAUNCHED("slice_llr_soft_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_selftest_gauss_tail(const float *z, int64_t count, float *out, void *stream) {
    clear_error();
    if (count < 0 || (count & 1)) QKD_FAIL(QKDREC_ERR_ARG, "count=%lld must be even and >= 0", (long long)count);
    if (count == 0) return QKDREC_OK;
    if (!z || !out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (((uintptr_t)z | (uintptr_t)out) & 7) QKD_FAIL(QKDREC_ERR_ARG, "z/out must be 8-byte aligned");
    const int64_t pairs = count / 2;
    gauss_tail_selftest_kernel<<<(unsigned)std::min<int64_t>(ceil_div(pairs, 256), 4096), 256, 0,
                                 as_stream(stream)>>>(reinterpret_cast<const float2 *>(z), pairs,
                                                      reinterpret_cast<float2 *>(out));
    QKD_LAUNCHED("gauss_tail_selftest_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_bits_to_llr(const uint8_t *bits, int64_t count, float *llr_out, void *stream) {
    clear_error();
    if (count < 0) QKD_FAIL(QKDREC_ERR_ARG, "count < 0");
    if (count == 0) return QKDREC_OK;
    if (!bits || !llr_out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    bits_to_llr_kernel<<<grid_for(count, 256), 256, 0, as_stream(stream)>>>(bits, count, llr_out);
    QKD_LAUNCHED("bits_to_llr_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_quantise_slices_frames(const float *y, int64_t count, const int64_t *frame_offsets,
                                            const double *frame_ranges, int32_t F, int32_t m, qkdrec_label label,
                                            uint8_t *idx_out, uint8_t *bits_out, void *stream) {
    clear_error();
    if (count < 0 || F < 0) QKD_FAIL(QKDREC_ERR_ARG, "count/F < 0");
    if (m < 1 || m > kMaxM) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, %d]", m, kMaxM);
    if (label != QKDREC_LABEL_GRAY && label != QKDREC_LABEL_BINARY) QKD_FAIL(QKDREC_ERR_ARG, "bad label");
    if (F == 0 || count == 0) return QKDREC_OK;
    if (!y || !frame_offsets || !frame_ranges) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (F > 2147483647) QKD_FAIL(QKDREC_ERR_ARG, "too many frames");
    prof::Scope ps(prof::kQuantise, as_stream(stream));
    quantise_frames_kernel<<<(unsigned)F, 256, 0, as_stream(stream)>>>(
        y, frame_offsets, frame_ranges, count, m, label == QKDREC_LABEL_GRAY, idx_out, bits_out,
        prof::counters(prof::kQuantise));
    QKD_LAUNCHED("quantise_frames_kernel");
    return QKDREC_OK;
}

qkdrec_status qkdrec_slice_llr_frames(const float *x, int64_t count, const int64_t *frame_offsets,
                                      const double *frame_params, int32_t F, int32_t m, int32_t j,
                                      qkdrec_label label, const uint8_t *lower_bits, float *llr_out,
                                      void *stream) {
    clear_error();
    if (count < 0 || F < 0) QKD_FAIL(QKDREC_ERR_ARG, "count/F < 0");
    if (m < 1 || m > kMaxM) QKD_FAIL(QKDREC_ERR_ARG, "m_slices=%d outside [1, %d]", m, kMaxM);
    if (j < 0 || j >= m) QKD_FAIL(QKDREC_ERR_ARG, "slice j=%d outside [0, %d)", j, m);
    if (label != QKDREC_LABEL_GRAY && label != QKDREC_LABEL_BINARY) QKD_FAIL(QKDREC_ERR_ARG, "bad label");
    if (F == 0 || count == 0) return QKDREC_OK;
    if (!x || !frame_offsets || !frame_params || !llr_out) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    if (j > 0 && !lower_bits) QKD_FAIL(QKDREC_ERR_ARG, "lower_bits NULL for j=%d", j);
    prof::Scope ps(prof::kSliceLlr, as_stream(stream));
    slice_llr_frames_kernel<<<(unsigned)F, 256, 0, as_stream(stream)>>>(
        x, frame_offsets, frame_params, count, m, j, label == QKDREC_LABEL_GRAY, lower_bits, llr_out,
        prof::counters(prof::kSliceLlr));
    QKD_LAUNCHED("slice_llr_frames_kernel");
    return QKDREC_OK;
}

}  // extern "C"
