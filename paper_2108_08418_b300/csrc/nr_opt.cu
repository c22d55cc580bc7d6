// Optimum sub-block length N_R of the block-wise parallel reconciliation
// (Sec. III-B, III-C, IV and the appendix): host arithmetic around the
// decoder, which supplies its two measured inputs, the time per arithmetic
// operation c_h and the decoding iterations D_j.
//
// K'(N_R) = (N C_Finite(N_R) - B_1) / (B_2 N_R) bits per second with
//   C_Finite(N_R) = C(gamma) - (sqrt(N_R A) Q^-1(eps_EC) + 1/2 log2 N_R) / N_R,
//   B_1 = N S_BE + sqrt(N) Delta_AEP + 2 log2(1 / (2 eps_PA)),
//   B_2 = sum_j 7 (G_j / N_R) D_j c_h,
// maximised over nr_min <= N_R <= N (the stationary point where dK'/dN_R = 0,
// or an end of the range).  Readings of the garbled or silent parts (base-2
// logarithms; the AWGN dispersion; the squares the appendix drops; the
// heterodyne detector term) are stated at include/qkdrec.h.
#include <math.h>

#include "common.cuh"

namespace qkd {

// Q(z) = P(N(0,1) > z) and its inverse by Newton steps from the tail asymptote
static double q_tail(double z) { return 0.5 * erfc(z * 0.70710678118654752440); }
static double q_inverse(double p) {
    if (p > 0.5) return -q_inverse(1.0 - p);
    const double l = -2.0 * log(p);
    double z = p < 0.25 ? sqrt(fmax(l - log(l) - log(2.0 * M_PI), 0.0)) : 0.0;
    for (int it = 0; it < 100; ++it) {
        const double dens = exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
        const double step = (q_tail(z) - p) / dens;
        z += step;
        if (fabs(step) <= 1e-15 * fmax(1.0, fabs(z))) break;
    }
    return z;
}

// (x + 1) log2(x + 1) - x log2 x
static double thermal_entropy(double x) { return x <= 0.0 ? 0.0 : (x + 1.0) * log2(x + 1.0) - x * log2(x); }

static void symplectic(double a, double b, double *l1, double *l2) {
    const double r = sqrt(fmax(a * a - 4.0 * b, 0.0));
    *l1 = sqrt((a + r) / 2.0);
    *l2 = sqrt(fmax((a - r) / 2.0, 0.0));
}

// Holevo information between Bob's heterodyne outcome and Eve (reverse
// reconciliation, Gaussian collective attack): entropy of Eve's state before
// minus after Bob's measurement, from the symplectic eigenvalues of the shared
// state's covariance matrix before and after the detection.
static double holevo_be(double va, double T, double xi_ch, double eta, double xi_d) {
    const double V = va + 1.0, chi_ch = (1.0 - T) / T + xi_ch;
    const double P1 = V * V * (1.0 - 2.0 * T) + 2.0 * T + T * T * (V + chi_ch) * (V + chi_ch);
    const double P2 = T * T * (V * chi_ch + 1.0) * (V * chi_ch + 1.0);
    const double ch = (2.0 - eta + 2.0 * xi_d) / eta, ct = chi_ch + ch / T;
    const double den = T * T * (V + ct) * (V + ct);
    const double Q1 = (P1 * ch * ch + P2 + 1.0 + 2.0 * ch * (T * (V + chi_ch) + V * sqrt(P2)) +
                       2.0 * T * (va * va + 2.0 * va)) / den;
    const double q2 = (V + ch * sqrt(P2)) / (T * (V + ct));
    double a1, a2, b1, b2;
    symplectic(P1, P2, &a1, &a2);
    symplectic(Q1, q2 * q2, &b1, &b2);
    return thermal_entropy((a1 - 1.0) / 2.0) + thermal_entropy((a2 - 1.0) / 2.0) -
           thermal_entropy((b1 - 1.0) / 2.0) - thermal_entropy((b2 - 1.0) / 2.0);
}

struct NrConst {
    double N, snr, iab, A, q, daep, sbe, tl, xu, b1, b2;
};

static qkdrec_status nr_const(const qkdrec_nr_params *p, NrConst &c) {
    if (!p) QKD_FAIL(QKDREC_ERR_ARG, "params NULL");
    const int m = p->m_slices;
    if (!(p->n_signals >= 2) || m < 1 || m > 16 || !p->edges_per_sample || !p->iterations)
        QKD_FAIL(QKDREC_ERR_ARG, "need N >= 2, 1 <= m <= 16 and the per-slice arrays");
    const double e[4] = {p->eps_ec, p->eps_s, p->eps_pa, p->eps_pe};
    for (double v : e)
        if (!(v > 0.0 && v < 0.5)) QKD_FAIL(QKDREC_ERR_ARG, "failure probabilities must lie in (0, 1/2)");
    if (!(p->va > 0) || !(p->transmissivity > 0 && p->transmissivity <= 1) || !(p->xi_ch >= 0) ||
        !(p->xi_d >= 0) || !(p->eta_d > 0 && p->eta_d <= 1) || !(p->c_h > 0))
        QKD_FAIL(QKDREC_ERR_ARG, "channel or hardware parameter out of range");
    c.N = p->n_signals;
    const double T = p->transmissivity, xi = p->xi_ch + p->xi_d;
    c.snr = 0.5 * p->va * T / (1.0 + 0.5 * xi);                 // Eq. SNR
    c.iab = 0.5 * log2(1.0 + c.snr);                             // C(gamma)
    c.A = p->dispersion_form == 1
              ? 0.5 * c.snr * (c.snr + 2.0) / ((c.snr + 1.0) * (c.snr + 1.0)) * log2(p->eps_ec) * log2(p->eps_ec)
              : c.snr * (c.snr + 2.0) / (2.0 * (c.snr + 1.0) * (c.snr + 1.0)) * M_LOG2E * M_LOG2E;
    c.q = q_inverse(p->eps_ec);
    const double eps = p->eps_ec + 2.0 * p->eps_s + p->eps_pa + p->eps_pe;   // Eq. AEP
    c.daep = (m + 1.0) * (m + 1.0) + 4.0 * (m + 1.0) * sqrt(log2(2.0 / (p->eps_s * p->eps_s))) +
             2.0 * log2(2.0 / (eps * eps * p->eps_s)) + 4.0 * p->eps_s * m / (eps * sqrt(c.N));
    // parameter estimation on N_e signals: worst-case T and xi_ch (appendix)
    const double ne = p->n_estimation > 0 ? p->n_estimation : c.N / 2.0;
    const double th = sqrt(p->eta_d * T), s2 = T * p->eta_d * p->xi_ch + 1.0 + p->xi_d;
    const double tau = q_inverse(p->eps_pe / 2.0);
    c.tl = (th - tau * sqrt(s2 / (ne * p->va))) * (th - tau * sqrt(s2 / (ne * p->va)));
    c.xu = (s2 + tau * s2 * sqrt(2.0) / sqrt(ne) - 1.0 - p->xi_d) / (th * th);
    if (!(c.tl > 0)) QKD_FAIL(QKDREC_ERR_ARG, "parameter estimation leaves no transmissivity (T^L <= 0)");
    c.sbe = holevo_be(p->va, c.tl, c.xu, p->eta_d, p->xi_d);
    c.b1 = c.N * c.sbe + sqrt(c.N) * c.daep + 2.0 * log2(1.0 / (2.0 * p->eps_pa));
    c.b2 = 0.0;
    for (int j = 0; j < m; ++j) {
        if (!(p->edges_per_sample[j] >= 0) || !(p->iterations[j] >= 0))
            QKD_FAIL(QKDREC_ERR_ARG, "slice %d: negative edges or iterations", j);
        c.b2 += 7.0 * p->edges_per_sample[j] * p->iterations[j] * p->c_h;   // Eqs. EP, DeltaT
    }
    if (!(c.b2 > 0)) QKD_FAIL(QKDREC_ERR_ARG, "no decoding work (B_2 = 0)");
    return QKDREC_OK;
}

static double c_finite(const NrConst &c, double x) { return c.iab - (sqrt(x * c.A) * c.q + 0.5 * log2(x)) / x; }
static double key_rate(const NrConst &c, double x) { return (c.N * c_finite(c, x) - c.b1) / (c.b2 * x); }
// dK'/dN_R = N / (B_2 N_R^2) x this bracket (Eq. diff_eq2 with base-2 logarithms)
static double dk_bracket(const NrConst &c, double x) {
    return 1.5 * sqrt(c.A) * c.q / sqrt(x) + (log2(x) - 0.5 / M_LN2) / x - c.iab + c.b1 / c.N;
}
// d^2 K'/dN_R^2 = (h'' x^2 - 2 h' x + 2 h) / (B_2 x^3), h = N C_Finite - B_1
static double d2_key_rate(const NrConst &c, double x) {
    const double h = c.N * c_finite(c, x) - c.b1;
    const double h1 = c.N * (0.5 * sqrt(c.A) * c.q * pow(x, -1.5) - (1.0 / M_LN2 - log2(x)) / (2.0 * x * x));
    const double h2 = c.N * (-0.75 * sqrt(c.A) * c.q * pow(x, -2.5) - (2.0 * log2(x) - 3.0 / M_LN2) / (2.0 * x * x * x));
    return (h2 * x * x - 2.0 * h1 * x + 2.0 * h) / (c.b2 * x * x * x);
}

}  // namespace qkd

using namespace qkd;

extern "C" {

qkdrec_status qkdrec_nr_key_rate(const qkdrec_nr_params *p, double nr, double *key_rate_out) {
    clear_error();
    if (!key_rate_out) QKD_FAIL(QKDREC_ERR_ARG, "key_rate NULL");
    NrConst c;
    qkdrec_status s = nr_const(p, c);
    if (s != QKDREC_OK) return s;
    if (!(nr >= 1.0)) QKD_FAIL(QKDREC_ERR_ARG, "N_R=%g below 1", nr);
    *key_rate_out = key_rate(c, nr);
    return QKDREC_OK;
}

qkdrec_status qkdrec_nr_optimise(const qkdrec_nr_params *p, qkdrec_nr_result *out) {
    clear_error();
    if (!out) QKD_FAIL(QKDREC_ERR_ARG, "out NULL");
    NrConst c;
    qkdrec_status s = nr_const(p, c);
    if (s != QKDREC_OK) return s;
    const double lo = p->nr_min > 0 ? p->nr_min : 1e5, hi = c.N;
    if (!(lo < hi)) QKD_FAIL(QKDREC_ERR_ARG, "N_R range [%g, %g] is empty", lo, hi);
    out->snr = c.snr;
    out->i_ab = c.iab;
    out->dispersion = c.A;
    out->qinv_ec = c.q;
    out->delta_aep = c.daep;
    out->s_be = c.sbe;
    out->t_low = c.tl;
    out->xi_up = c.xu;
    out->b1 = c.b1;
    out->b2 = c.b2;
    out->nr_stationary = 0.0;
    // the stationary point: bisection on ln N_R where dK'/dN_R changes sign
    // from rising to falling
    if (dk_bracket(c, lo) > 0.0 && dk_bracket(c, hi) < 0.0) {
        double a = log(lo), b = log(hi);
        for (int it = 0; it < 400 && b - a > 1e-15 * fabs(b); ++it) {
            const double mid = 0.5 * (a + b);
            if (dk_bracket(c, exp(mid)) > 0.0) a = mid;
            else b = mid;
        }
        out->nr_stationary = exp(0.5 * (a + b));
    }
    double best = lo;
    if (key_rate(c, hi) > key_rate(c, best)) best = hi;
    if (out->nr_stationary > 0 && key_rate(c, out->nr_stationary) >= key_rate(c, best)) best = out->nr_stationary;
    out->nr_opt = best;
    out->key_rate_opt = key_rate(c, best);
    out->d2_key_rate = d2_key_rate(c, best);
    out->at_boundary = best != out->nr_stationary;
    return QKDREC_OK;
}

}  // extern "C"
