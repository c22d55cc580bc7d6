/*
 * FP64 reference decoders for syndrome-based LDPC belief propagation.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, plain oracle that the CUDA
 * library is checked against; nothing in the product path may link or call it.
 * It shares no code, header or constant table with the CUDA library.
 *
 * The paper adopts "the well-known BP decoder" without fixing a variant
 * (Sec. III-C, text before Eq. rob2) and counts its work as 7G operations per
 * iteration (Eq. EP).  Each decoder below is written from the textbook
 * definition of the message-passing rules, in the order they are defined, one
 * frame at a time (frames are the N_d independent sub-blocks of Sec. III-A,
 * Fig. 2), with no blocking or fusion:
 *
 *   LLR convention   L = ln P(b=0)/P(b=1); hard decision b = 1 iff L < 0.
 *   Syndrome-signed check rule  (Bob sends s = H S_j, Sec. III-B step 2-3):
 *       a check with syndrome bit s_c flips the sign of its outgoing messages.
 *   Stopping   the syndrome of the hard decision is tested before the first
 *       iteration and after every iteration; with early stop the frame stops at
 *       the first success; `iters` = iterations executed, `conv` = syndrome met.
 *
 * Sum-product (flooding), with the saturation constants A_MIN/A_MAX:
 *   q_vc   = L_v - m_cv
 *   a_vc   = clamp(|q_vc|, A_MIN, A_MAX)
 *   m_cv'  = (-1)^{s_c} prod_{v'!=v} sgn(q_v'c) * phi( clamp(sum_{v'!=v} phi(a_v'c), A_MIN, A_MAX) )
 *   L_v'   = llr_v + sum_c m_cv'
 *   phi(x) = -ln tanh(x/2) = ln((e^x+1)/(e^x-1)), evaluated as log1p(2/expm1(x)).
 *   sgn(0) = +1.
 * Offset min-sum (flooding or layered), offset beta:
 *   m_cv'  = (-1)^{s_c} prod_{v'!=v} sgn(q_v'c) * max(min_{v'!=v} |q_v'c| - beta, 0)
 *   layered: checks are processed layer by layer (a layer is a set of checks that
 *   share no variable); for each check q = L_v - m_cv, new m_cv, L_v = q + m_cv.
 * Integer offset min-sum (6-bit messages, clip +-31, offset 1 LSB):
 *   llr_q = clamp(round_half_away(llr / step), -31, 31), posterior int16 saturating,
 *   v->c message clamp(q, -31, 31), c->v message sign * max(min - 1, 0).
 * Weighted offset min-sum (unrolled, flooding), per-iteration per-degree-class
 * weights alpha[t][d], beta[t][d]:
 *   m_cv'  = (-1)^{s_c} prod sgn * alpha * max(min_{v'!=v}|q| - beta, 0),
 *   with reverse-mode gradients of a BCE loss on the final posteriors.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define A_MIN 1e-30
#define A_MAX 30.0

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double sgn(double x) { return x < 0.0 ? -1.0 : 1.0; }
static double phi(double x) { return log1p(2.0 / expm1(x)); }

/* 1 if the hard decision of L satisfies every check of the syndrome */
static int syndrome_ok_d(int M, const int32_t *rp, const int32_t *ci, const double *L,
                         const uint8_t *s) {
    for (int c = 0; c < M; ++c) {
        int par = s[c] & 1;
        for (int32_t e = rp[c]; e < rp[c + 1]; ++e) par ^= (L[ci[e]] < 0.0);
        if (par) return 0;
    }
    return 1;
}

static int syndrome_ok_i(int M, const int32_t *rp, const int32_t *ci, const int32_t *L,
                         const uint8_t *s) {
    for (int c = 0; c < M; ++c) {
        int par = s[c] & 1;
        for (int32_t e = rp[c]; e < rp[c + 1]; ++e) par ^= (L[ci[e]] < 0);
        if (par) return 0;
    }
    return 1;
}

static void finish_frame_d(int n, const double *L, uint8_t *bits, double *post) {
    for (int v = 0; v < n; ++v) {
        bits[v] = (uint8_t)(L[v] < 0.0);
        if (post) post[v] = L[v];
    }
}

/* ---------------------------------------------------------------- SP flooding */
static void sp_check_update(int32_t beg, int32_t end, int sc, const int32_t *ci,
                            const double *L, const double *m_old, double *m_new) {
    int32_t d = end - beg;
    for (int32_t i = 0; i < d; ++i) {
        double sum = 0.0, sign = (sc & 1) ? -1.0 : 1.0;
        for (int32_t k = 0; k < d; ++k) {
            if (k == i) continue;
            double q = L[ci[beg + k]] - m_old[beg + k];
            sign *= sgn(q);
            sum += phi(clampd(fabs(q), A_MIN, A_MAX));
        }
        m_new[beg + i] = sign * phi(clampd(sum, A_MIN, A_MAX));
    }
}

int oracle_sp_flood(int n, int M, const int32_t *rp, const int32_t *ci,
                    const double *llr, const uint8_t *synd, int F, int max_iter,
                    int early_stop, uint8_t *bits, int32_t *iters, uint8_t *conv,
                    double *post) {
    int32_t E = rp[M];
    double *m_old = (double *)malloc(sizeof(double) * (size_t)E);
    double *m_new = (double *)malloc(sizeof(double) * (size_t)E);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    if (!m_old || !m_new || !L) { free(m_old); free(m_new); free(L); return -1; }
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        memset(m_old, 0, sizeof(double) * (size_t)E);
        for (int v = 0; v < n; ++v) L[v] = lf[v];
        int it = 0, ok = syndrome_ok_d(M, rp, ci, L, sf);
        while (it < max_iter && !(early_stop && ok)) {
            /* check phase: every check reads the previous iteration's messages */
            for (int c = 0; c < M; ++c) sp_check_update(rp[c], rp[c + 1], sf[c], ci, L, m_old, m_new);
            /* variable phase: posteriors from the channel plus all incoming messages */
            for (int v = 0; v < n; ++v) L[v] = lf[v];
            for (int32_t e = 0; e < E; ++e) L[ci[e]] += m_new[e];
            double *t = m_old; m_old = m_new; m_new = t;
            ++it;
            ok = syndrome_ok_d(M, rp, ci, L, sf);
        }
        iters[f] = it;
        conv[f] = (uint8_t)ok;
        finish_frame_d(n, L, bits + (size_t)f * n, post ? post + (size_t)f * n : NULL);
    }
    free(m_old); free(m_new); free(L);
    return 0;
}

/* ----------------------------------------------------------- OMS (floating) */
static void oms_check_update(int32_t beg, int32_t end, int sc, const double *q, double beta,
                             double *m_out) {
    int32_t d = end - beg;
    for (int32_t i = 0; i < d; ++i) {
        double mn = INFINITY, sign = (sc & 1) ? -1.0 : 1.0;
        for (int32_t k = 0; k < d; ++k) {
            if (k == i) continue;
            sign *= sgn(q[k]);
            if (fabs(q[k]) < mn) mn = fabs(q[k]);
        }
        double mag = mn - beta;
        m_out[beg + i] = sign * (mag > 0.0 ? mag : 0.0);
    }
}

int oracle_oms_flood(int n, int M, const int32_t *rp, const int32_t *ci,
                     const double *llr, const uint8_t *synd, int F, int max_iter,
                     double beta, int early_stop, uint8_t *bits, int32_t *iters,
                     uint8_t *conv, double *post) {
    int32_t E = rp[M];
    int32_t dmax = 0;
    for (int c = 0; c < M; ++c) if (rp[c + 1] - rp[c] > dmax) dmax = rp[c + 1] - rp[c];
    double *m_old = (double *)malloc(sizeof(double) * (size_t)E);
    double *m_new = (double *)malloc(sizeof(double) * (size_t)E);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    if (!m_old || !m_new || !L || !q) { free(m_old); free(m_new); free(L); free(q); return -1; }
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        memset(m_old, 0, sizeof(double) * (size_t)E);
        for (int v = 0; v < n; ++v) L[v] = lf[v];
        int it = 0, ok = syndrome_ok_d(M, rp, ci, L, sf);
        while (it < max_iter && !(early_stop && ok)) {
            for (int c = 0; c < M; ++c) {
                for (int32_t e = rp[c]; e < rp[c + 1]; ++e) q[e - rp[c]] = L[ci[e]] - m_old[e];
                oms_check_update(rp[c], rp[c + 1], sf[c], q, beta, m_new);
            }
            for (int v = 0; v < n; ++v) L[v] = lf[v];
            for (int32_t e = 0; e < E; ++e) L[ci[e]] += m_new[e];
            double *t = m_old; m_old = m_new; m_new = t;
            ++it;
            ok = syndrome_ok_d(M, rp, ci, L, sf);
        }
        iters[f] = it;
        conv[f] = (uint8_t)ok;
        finish_frame_d(n, L, bits + (size_t)f * n, post ? post + (size_t)f * n : NULL);
    }
    free(m_old); free(m_new); free(L); free(q);
    return 0;
}

/* layer_checks: the checks listed layer after layer; layer_ptr[n_layers+1]
   delimits them.  Inside a layer the checks share no variable. */
int oracle_oms_layered(int n, int M, const int32_t *rp, const int32_t *ci,
                       int n_layers, const int32_t *layer_ptr, const int32_t *layer_checks,
                       const double *llr, const uint8_t *synd, int F, int max_iter,
                       double beta, int early_stop, uint8_t *bits, int32_t *iters,
                       uint8_t *conv, double *post) {
    int32_t E = rp[M];
    int32_t dmax = 0;
    for (int c = 0; c < M; ++c) if (rp[c + 1] - rp[c] > dmax) dmax = rp[c + 1] - rp[c];
    double *m = (double *)malloc(sizeof(double) * (size_t)E);
    double *L = (double *)malloc(sizeof(double) * (size_t)n);
    double *q = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    if (!m || !L || !q) { free(m); free(L); free(q); return -1; }
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        memset(m, 0, sizeof(double) * (size_t)E);
        for (int v = 0; v < n; ++v) L[v] = lf[v];
        int it = 0, ok = syndrome_ok_d(M, rp, ci, L, sf);
        while (it < max_iter && !(early_stop && ok)) {
            for (int l = 0; l < n_layers; ++l) {
                for (int32_t k = layer_ptr[l]; k < layer_ptr[l + 1]; ++k) {
                    int c = layer_checks[k];
                    for (int32_t e = rp[c]; e < rp[c + 1]; ++e) q[e - rp[c]] = L[ci[e]] - m[e];
                    oms_check_update(rp[c], rp[c + 1], sf[c], q, beta, m);
                    for (int32_t e = rp[c]; e < rp[c + 1]; ++e) L[ci[e]] = q[e - rp[c]] + m[e];
                }
            }
            ++it;
            ok = syndrome_ok_d(M, rp, ci, L, sf);
        }
        iters[f] = it;
        conv[f] = (uint8_t)ok;
        finish_frame_d(n, L, bits + (size_t)f * n, post ? post + (size_t)f * n : NULL);
    }
    free(m); free(L); free(q);
    return 0;
}

/* ------------------------------------------------- integer OMS (6-bit, +-31) */
#define QMAX 31
#define PMAX 32767

static int32_t clampi(int32_t x, int32_t lo, int32_t hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* round half away from zero of llr/step, then clip to the 6-bit range */
static int32_t quantise_llr(double llr, double step) {
    double r = llr / step;
    double a = floor(fabs(r) + 0.5);
    double v = r < 0.0 ? -a : a;
    if (v > QMAX) v = QMAX;
    if (v < -QMAX) v = -QMAX;
    return (int32_t)v;
}

static void ioms_check_update(int32_t beg, int32_t end, int sc, const int32_t *q, int32_t *m_out) {
    int32_t d = end - beg;
    for (int32_t i = 0; i < d; ++i) {
        int32_t mn = 1 << 30, neg = sc & 1;
        for (int32_t k = 0; k < d; ++k) {
            if (k == i) continue;
            neg ^= (q[k] < 0);
            int32_t a = q[k] < 0 ? -q[k] : q[k];
            if (a < mn) mn = a;
        }
        int32_t mag = mn - 1 > 0 ? mn - 1 : 0;
        m_out[beg + i] = neg ? -mag : mag;
    }
}

static void finish_frame_i(int n, const int32_t *L, double step, uint8_t *bits, double *post) {
    for (int v = 0; v < n; ++v) {
        bits[v] = (uint8_t)(L[v] < 0);
        if (post) post[v] = (double)L[v] * step;
    }
}

int oracle_ioms(int layered, int n, int M, const int32_t *rp, const int32_t *ci,
                int n_layers, const int32_t *layer_ptr, const int32_t *layer_checks,
                const double *llr, const uint8_t *synd, int F, int max_iter, double step,
                int early_stop, uint8_t *bits, int32_t *iters, uint8_t *conv, double *post) {
    int32_t E = rp[M];
    int32_t dmax = 0;
    for (int c = 0; c < M; ++c) if (rp[c + 1] - rp[c] > dmax) dmax = rp[c + 1] - rp[c];
    int32_t *m_old = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    int32_t *m_new = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    int32_t *L = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *lq = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)(dmax + 1));
    int32_t *qf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(dmax + 1));
    if (!m_old || !m_new || !L || !lq || !q || !qf) {
        free(m_old); free(m_new); free(L); free(lq); free(q); free(qf);
        return -1;
    }
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        memset(m_old, 0, sizeof(int32_t) * (size_t)E);
        for (int v = 0; v < n; ++v) { lq[v] = quantise_llr(lf[v], step); L[v] = lq[v]; }
        int it = 0, ok = syndrome_ok_i(M, rp, ci, L, sf);
        while (it < max_iter && !(early_stop && ok)) {
            if (!layered) {
                for (int c = 0; c < M; ++c) {
                    for (int32_t e = rp[c]; e < rp[c + 1]; ++e)
                        q[e - rp[c]] = clampi(L[ci[e]] - m_old[e], -QMAX, QMAX);
                    ioms_check_update(rp[c], rp[c + 1], sf[c], q, m_new);
                }
                for (int v = 0; v < n; ++v) L[v] = lq[v];
                for (int32_t e = 0; e < E; ++e) L[ci[e]] = clampi(L[ci[e]] + m_new[e], -PMAX, PMAX);
                int32_t *t = m_old; m_old = m_new; m_new = t;
            } else {
                for (int l = 0; l < n_layers; ++l) {
                    for (int32_t k = layer_ptr[l]; k < layer_ptr[l + 1]; ++k) {
                        int c = layer_checks[k];
                        for (int32_t e = rp[c]; e < rp[c + 1]; ++e) {
                            qf[e - rp[c]] = clampi(L[ci[e]] - m_old[e], -PMAX, PMAX);
                            q[e - rp[c]] = clampi(qf[e - rp[c]], -QMAX, QMAX);
                        }
                        ioms_check_update(rp[c], rp[c + 1], sf[c], q, m_old);
                        for (int32_t e = rp[c]; e < rp[c + 1]; ++e)
                            L[ci[e]] = clampi(qf[e - rp[c]] + m_old[e], -PMAX, PMAX);
                    }
                }
            }
            ++it;
            ok = syndrome_ok_i(M, rp, ci, L, sf);
        }
        iters[f] = it;
        conv[f] = (uint8_t)ok;
        finish_frame_i(n, L, step, bits + (size_t)f * n, post ? post + (size_t)f * n : NULL);
    }
    free(m_old); free(m_new); free(L); free(lq); free(q); free(qf);
    return 0;
}

/* --------------------------- unrolled weighted offset min-sum and its gradient
 *
 * T flooding iterations, no stopping test.  Iteration t (1-based) uses the
 * weights alpha[t-1][cls], beta[t-1][cls] of the check's degree class
 * (cls = 0 for checks of the smallest degree in the code, 1 otherwise):
 *   q_e     = L^{t-1}_{v(e)} - m^{t-1}_e                    (m^0 = 0, L^0 = llr)
 *   mn_e    = min over the check's other edges of |q|
 *   m^t_e   = (-1)^{s_c} prod_{other edges} sgn(q) * alpha * max(mn_e - beta, 0)
 *   L^t_v   = llr_v + sum_{e at v} m^t_e
 * Loss = mean over frames and variables of the binary cross-entropy of
 * P(b = 1) = sigma(-L^T_v) against the target bits:
 *   b softplus(L) + (1 - b) softplus(-L).
 * Reverse mode with the conventions: the gradient of a minimum goes to its
 * argmin (ties: the lowest edge index), max(x, 0)' = 0 at x <= 0, sgn(0) = +1;
 * the signs are piecewise constant and carry no gradient.  All iterations are
 * stored (no checkpointing).  galpha/gbeta [T][2] are overwritten.
 */
static double softplus(double x) { return x > 0.0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigmoid(double x) { return x >= 0.0 ? 1.0 / (1.0 + exp(-x)) : exp(x) / (1.0 + exp(x)); }

/* lowest-index argmin of |q| over a check's edges, optionally excluding one edge */
static int32_t argmin_abs(const double *q, int32_t d, int32_t skip) {
    int32_t best = -1;
    for (int32_t k = 0; k < d; ++k) {
        if (k == skip) continue;
        if (best < 0 || fabs(q[k]) < fabs(q[best])) best = k;
    }
    return best;
}

int oracle_woms(int n, int M, const int32_t *rp, const int32_t *ci, const double *llr,
                const uint8_t *synd, const uint8_t *target, int F, int T, const double *alpha,
                const double *beta, double *loss, double *galpha, double *gbeta, double *post) {
    int32_t E = rp[M];
    int32_t dmin = 1 << 30, dmax = 0;
    for (int c = 0; c < M; ++c) {
        int32_t d = rp[c + 1] - rp[c];
        if (d < dmin) dmin = d;
        if (d > dmax) dmax = d;
    }
    double *m = (double *)calloc((size_t)(T + 1) * E, sizeof(double));   /* m[t][e] */
    double *L = (double *)malloc(sizeof(double) * (size_t)(T + 1) * n);  /* L[t][v] */
    double *q = (double *)malloc(sizeof(double) * (size_t)(dmax + 1));
    double *gL = (double *)malloc(sizeof(double) * (size_t)n);
    double *gLn = (double *)malloc(sizeof(double) * (size_t)n);
    double *gm = (double *)malloc(sizeof(double) * (size_t)E);
    double *gq = (double *)malloc(sizeof(double) * (size_t)E);
    if (!m || !L || !q || !gL || !gLn || !gm || !gq) {
        free(m); free(L); free(q); free(gL); free(gLn); free(gm); free(gq);
        return -1;
    }
    for (int i = 0; i < 2 * T; ++i) { galpha[i] = 0.0; gbeta[i] = 0.0; }
    double total = 0.0;
    const double scale = 1.0 / ((double)F * (double)n);
    for (int f = 0; f < F; ++f) {
        const double *lf = llr + (size_t)f * n;
        const uint8_t *sf = synd + (size_t)f * M;
        const uint8_t *bf = target + (size_t)f * n;
        memset(m, 0, sizeof(double) * (size_t)E);
        for (int v = 0; v < n; ++v) L[v] = lf[v];
        /* forward, every iteration kept */
        for (int t = 1; t <= T; ++t) {
            const double *mo = m + (size_t)(t - 1) * E;
            double *mt = m + (size_t)t * E;
            const double *Lo = L + (size_t)(t - 1) * n;
            double *Lt = L + (size_t)t * n;
            for (int c = 0; c < M; ++c) {
                int32_t beg = rp[c], d = rp[c + 1] - rp[c];
                int cls = d == dmin ? 0 : 1;
                double a = alpha[2 * (t - 1) + cls], b = beta[2 * (t - 1) + cls];
                for (int32_t k = 0; k < d; ++k) q[k] = Lo[ci[beg + k]] - mo[beg + k];
                for (int32_t k = 0; k < d; ++k) {
                    double sign = (sf[c] & 1) ? -1.0 : 1.0;
                    for (int32_t j = 0; j < d; ++j)
                        if (j != k) sign *= sgn(q[j]);
                    double mn = fabs(q[argmin_abs(q, d, k)]);
                    double r = mn - b;
                    mt[beg + k] = sign * a * (r > 0.0 ? r : 0.0);
                }
            }
            for (int v = 0; v < n; ++v) Lt[v] = lf[v];
            for (int32_t e = 0; e < E; ++e) Lt[ci[e]] += mt[e];
        }
        const double *LT = L + (size_t)T * n;
        for (int v = 0; v < n; ++v) {
            total += bf[v] ? softplus(LT[v]) : softplus(-LT[v]);
            if (post) post[(size_t)f * n + v] = LT[v];
            gL[v] = scale * (bf[v] ? sigmoid(LT[v]) : -sigmoid(-LT[v]));
        }
        /* reverse */
        memset(gm, 0, sizeof(double) * (size_t)E);     /* d loss / d m^t through q^{t+1} */
        for (int t = T; t >= 1; --t) {
            const double *mo = m + (size_t)(t - 1) * E;
            const double *Lo = L + (size_t)(t - 1) * n;
            memset(gq, 0, sizeof(double) * (size_t)E);
            for (int c = 0; c < M; ++c) {
                int32_t beg = rp[c], d = rp[c + 1] - rp[c];
                int cls = d == dmin ? 0 : 1;
                double a = alpha[2 * (t - 1) + cls], b = beta[2 * (t - 1) + cls];
                for (int32_t k = 0; k < d; ++k) q[k] = Lo[ci[beg + k]] - mo[beg + k];
                for (int32_t k = 0; k < d; ++k) {
                    int32_t e = beg + k;
                    double g = gm[e] + gL[ci[e]];            /* d loss / d m^t_e */
                    double sign = (sf[c] & 1) ? -1.0 : 1.0;
                    for (int32_t j = 0; j < d; ++j)
                        if (j != k) sign *= sgn(q[j]);
                    int32_t src = argmin_abs(q, d, k);
                    double r = fabs(q[src]) - b;
                    double relu = r > 0.0 ? r : 0.0;
                    galpha[2 * (t - 1) + cls] += g * sign * relu;
                    if (r > 0.0) {
                        double gr = g * sign * a;
                        gbeta[2 * (t - 1) + cls] -= gr;
                        gq[beg + src] += gr * sgn(q[src]);
                    }
                }
            }
            /* q^t = L^{t-1} - m^{t-1};  L^{t-1} = llr + sum m^{t-1} */
            for (int v = 0; v < n; ++v) gLn[v] = 0.0;
            for (int32_t e = 0; e < E; ++e) {
                gLn[ci[e]] += gq[e];
                gm[e] = -gq[e];
            }
            for (int v = 0; v < n; ++v) gL[v] = gLn[v];
        }
    }
    *loss = total * scale;
    free(m); free(L); free(q); free(gL); free(gLn); free(gm); free(gq);
    return 0;
}
