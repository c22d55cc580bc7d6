/*
 * Forward error bounds of the low-precision decoder forms around the FP64
 * decoders of bp.c.
 *
 * TEST INFRASTRUCTURE ONLY (part of the oracle; nothing on the product path
 * links it).  The paper leaves the BP decoder's precision open (Sec. III-C);
 * the precision study runs the same rules with FP32 arithmetic and the edge
 * messages STORED in IEEE binary16 (FP16).  Such a decoder does not compute
 * the FP64 result; this file bounds how far from it it can land.
 *
 * Each decoder below repeats the FP64 recurrence of its counterpart in bp.c
 * (same order, same saturation constants) and carries, next to every message
 * m and posterior L, a radius r: an upper bound on |m~ - m| (|L~ - L|) over
 * every decoder that evaluates the same rules with
 *   - each FP32 operation rounded to nearest, |fl(x op y) - (x op y)| <= u32
 *     |fl(x op y)| with u32 = 2^-24 (the standard model, Higham, "Accuracy and
 *     Stability of Numerical Algorithms", Sec. 2.2; a sum of k terms is off by
 *     at most k u32 (1 + k u32) times the sum of the magnitudes, Sec. 3.1);
 *   - each stored message rounded to binary16, |fl16(x) - x| <= u16 |x| +
 *     2^-25 with u16 = 2^-11 (2^-25: half the spacing of the binary16
 *     subnormals); |x| > 65504 (overflow) makes the radius infinite;
 *   - the check function phi evaluated with relative error at most phi_rel
 *     (sum-product only; the caller states the accuracy it relies on).
 * Rules for the radius, from the exact value v and radius r of each input:
 *   q = L - m                      r_q = r_L + r_m + u32 (|q| + r_L + r_m)
 *   min over other edges of |q|    the minimum of |q~| lies in [min (|q| - r_q),
 *                                  min (|q| + r_q)] over those edges
 *   max(x - beta, 0)               r   = r_x + u32 (|x - beta| + r_x)
 *   phi on [a - r, a + r]          phi is decreasing, so the image lies in
 *                                  [phi(a + r), phi(a - r)] (clamped to the
 *                                  saturation range), widened by phi_rel; the
 *                                  sums of phi values carry these intervals
 *                                  (lower and upper ends) rather than radii
 *   sign of a product              exact unless some factor has |q| <= r_q; then
 *                                  the message can take either sign and
 *                                  r = 2 |m| + r_|m|
 * The midpoints are the FP64 results of bp.c's decoders for the same inputs
 * (fixed iteration count, no stopping test), so a decoder of that precision
 * must satisfy |L~ - L| <= r_L for every posterior.  A frame of F frames is
 * processed one at a time, as in bp.c.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define B_A_MIN 1e-30
#define B_A_MAX 30.0
#define U32 5.9604644775390625e-08            /* 2^-24 */
#define U16 4.8828125e-04                     /* 2^-11 */
#define SUB16 2.98023223876953125e-08         /* 2^-25 */
#define MAX16 65504.0

static double bclamp(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double bphi(double x) { return log1p(2.0 / expm1(x)); }

/* radius of a message after storage: binary16 (f16 = 1) or binary32 (f16 = 0) */
static double stored(double m, double r, int f16) {
    double a = fabs(m) + r;
    if (f16) {
        if (a > MAX16) return INFINITY;
        return r + U16 * a + SUB16;
    }
    return r + U32 * a;
}

/* sum of F frames' posteriors after exactly T iterations, with radii.
 * algo 0: sum-product flooding; 1: offset min-sum flooding; 2: offset min-sum
 * layered (layer_ptr / layer_checks as in bp.c).  f16: messages stored as
 * binary16 (1) or binary32 (0).  post / rad: [F][n]. */
int oracle_lowp_bound(int algo, int f16, int n, int M, const int32_t *rp, const int32_t *ci,
                      int n_layers, const int32_t *layer_ptr, const int32_t *layer_checks,
                      const double *llr, const uint8_t *synd, int F, int T, double beta,
                      double phi_rel, double *post, double *rad) {
    int32_t E = rp[M];
    int32_t dmax = 0;
    for (int c = 0; c < M; ++c) if (rp[c + 1] - rp[c] > dmax) dmax = rp[c + 1] - rp[c];
    int32_t *vdeg = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    double *m = (double *)malloc(sizeof(double) * (size_t)E);
    double *rm = (double *)malloc(sizeof(double) * (size_t)E);
    double *mn = (double *)malloc(sizeof(double) * (size_t)E);
    double *rmn = (double *)malloc(sizeof(double) * (size_t)E);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *rL = (double *)malloc(sizeof(double) * (size_t)n);
    double *sabs = (double *)malloc(sizeof(double) * (size_t)n);   /* sum of magnitudes of a variable sum */
    double *q = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *rq = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *fv = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *flo = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *fhi = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    if (!vdeg || !m || !rm || !mn || !rmn || !L || !rL || !sabs || !q || !rq || !fv || !flo || !fhi) {
        free(vdeg); free(m); free(rm); free(mn); free(rmn); free(L); free(rL); free(sabs);
        free(q); free(rq); free(fv); free(flo); free(fhi);
        return -1;
    }
    for (int32_t e = 0; e < E; ++e) vdeg[ci[e]]++;
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        for (int32_t e = 0; e < E; ++e) { m[e] = 0.0; rm[e] = 0.0; }
        for (int v = 0; v < n; ++v) { L[v] = lf[v]; rL[v] = 0.0; }
        for (int t = 0; t < T; ++t) {
            int nl = algo == 2 ? n_layers : 1;
            for (int l = 0; l < nl; ++l) {
                int32_t kb = algo == 2 ? layer_ptr[l] : 0, ke = algo == 2 ? layer_ptr[l + 1] : M;
                for (int32_t kk = kb; kk < ke; ++kk) {
                    int c = algo == 2 ? layer_checks[kk] : kk;
                    int32_t beg = rp[c], d = rp[c + 1] - rp[c];
                    for (int32_t k = 0; k < d; ++k) {
                        int32_t e = beg + k, v = ci[e];
                        q[k] = L[v] - m[e];
                        rq[k] = rL[v] + rm[e] + U32 * (fabs(q[k]) + rL[v] + rm[e]);
                        if (algo == 0) {
                            /* phi(|q~|) lies in [flo, fhi]: phi is decreasing */
                            double a = bclamp(fabs(q[k]), B_A_MIN, B_A_MAX);
                            fv[k] = bphi(a);
                            flo[k] = bphi(bclamp(a + rq[k], B_A_MIN, B_A_MAX)) * (1.0 - phi_rel);
                            fhi[k] = bphi(bclamp(a - rq[k], B_A_MIN, B_A_MAX)) * (1.0 + phi_rel);
                        }
                    }
                    for (int32_t i = 0; i < d; ++i) {
                        double sign = (sf[c] & 1) ? -1.0 : 1.0, mag, rmag;
                        int unsure = 0;
                        if (algo == 0) {
                            double s = 0.0, slo = 0.0, shi = 0.0;
                            for (int32_t k = 0; k < d; ++k) {
                                if (k == i) continue;
                                sign *= q[k] < 0.0 ? -1.0 : 1.0;
                                unsure |= fabs(q[k]) <= rq[k];
                                s += fv[k];
                                slo += flo[k];
                                shi += fhi[k];
                            }
                            /* the exclusion sum in FP32, formed either directly or as
                               (sum of all but the largest) + (largest - own term): at
                               most d + 2 roundings of partial sums no larger than
                               3 x the sum of the other terms (the own term is at most
                               the largest, which the exclusion sum contains) */
                            double rnd = 3.0 * (d + 2) * U32 * (1.0 + (d + 2) * U32) * shi;
                            slo -= rnd;
                            shi += rnd;
                            mag = bphi(bclamp(s, B_A_MIN, B_A_MAX));
                            double mlo = bphi(bclamp(shi, B_A_MIN, B_A_MAX)) * (1.0 - phi_rel);
                            double mhi = bphi(bclamp(slo, B_A_MIN, B_A_MAX)) * (1.0 + phi_rel);
                            rmag = fmax(mhi - mag, mag - mlo);
                        } else {
                            /* the minimum of |q~| lies between the minima of the
                               interval ends |q| -+ r_q of the other edges */
                            double mmin = INFINITY, lo = INFINITY, hi = INFINITY;
                            for (int32_t k = 0; k < d; ++k) {
                                if (k == i) continue;
                                sign *= q[k] < 0.0 ? -1.0 : 1.0;
                                unsure |= fabs(q[k]) <= rq[k];
                                if (fabs(q[k]) < mmin) mmin = fabs(q[k]);
                                lo = fmin(lo, fmax(fabs(q[k]) - rq[k], 0.0));
                                hi = fmin(hi, fabs(q[k]) + rq[k]);
                            }
                            double rmin = fmax(mmin - lo, hi - mmin);
                            double x = mmin - beta;
                            mag = x > 0.0 ? x : 0.0;
                            rmag = rmin + U32 * (fabs(x) + rmin);
                        }
                        double r = unsure ? 2.0 * mag + rmag : rmag;
                        mn[beg + i] = sign * mag;
                        rmn[beg + i] = stored(mag, r, f16);
                    }
                    if (algo == 2) {
                        /* layered: L = q + (stored message), in place */
                        for (int32_t k = 0; k < d; ++k) {
                            int32_t e = beg + k, v = ci[e];
                            m[e] = mn[e];
                            rm[e] = rmn[e];
                            L[v] = q[k] + m[e];
                            rL[v] = rq[k] + rm[e] + U32 * (fabs(L[v]) + rq[k] + rm[e]);
                        }
                    }
                }
            }
            if (algo != 2) {
                /* flooding variable update: L = llr + sum of the stored messages, in
                   ascending edge order, in FP32 */
                for (int v = 0; v < n; ++v) { L[v] = lf[v]; rL[v] = 0.0; sabs[v] = fabs(lf[v]); }
                for (int32_t e = 0; e < E; ++e) {
                    m[e] = mn[e];
                    rm[e] = rmn[e];
                    L[ci[e]] += m[e];
                    rL[ci[e]] += rm[e];
                    sabs[ci[e]] += fabs(m[e]) + rm[e];
                }
                for (int v = 0; v < n; ++v) rL[v] += vdeg[v] * U32 * (1.0 + vdeg[v] * U32) * sabs[v];
            }
        }
        for (int v = 0; v < n; ++v) {
            post[(size_t)f * n + v] = L[v];
            rad[(size_t)f * n + v] = rL[v];
        }
    }
    free(vdeg); free(m); free(rm); free(mn); free(rmn); free(L); free(rL); free(sabs);
    free(q); free(rq); free(fv); free(flo); free(fhi);
    return 0;
}
