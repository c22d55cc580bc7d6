// Code objects (parity-check matrices H_j), error strings and host helpers.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace qkd {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

static void free_code(CodeDev &d) {
    cudaFree(d.rp);
    cudaFree(d.ci);
    cudaFree(d.vptr);
    cudaFree(d.vedge);
    cudaFree(d.layer_ptr);
    cudaFree(d.layer_chk);
    cudaFree(d.qc_shift);
    free(d.h_layer_of);
    d = CodeDev();
}

template <class T>
static qkdrec_status upload(T **dst, const T *src, size_t count) {
    size_t bytes = sizeof(T) * (count ? count : 1);
    cudaError_t e = cudaMalloc((void **)dst, bytes);
    if (e != cudaSuccess) QKD_FAIL(QKDREC_ERR_NOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    if (count) QKD_CUDA(cudaMemcpy(*dst, src, sizeof(T) * count, cudaMemcpyHostToDevice));
    return QKDREC_OK;
}

}  // namespace qkd

using namespace qkd;

// seeded left-regular construction (synth/_codegen.c, compiled into the library)
extern "C" int64_t synth_make_regular_code(uint64_t seed, int32_t n, int32_t M, int32_t dv, int32_t max_passes,
                                           int32_t *rp, int32_t *ci);

extern "C" {

const char *qkdrec_last_error(void) { return g_err; }

const char *qkdrec_version(void) { return "qkdrec 0.1 (sm_103a)"; }

qkdrec_status qkdrec_code_create(int32_t n, int32_t m_checks, const int32_t *row_ptr,
                                 const int32_t *col_idx, uint64_t seed, qkdrec_code_t *out) {
    clear_error();
    if (!out) QKD_FAIL(QKDREC_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n <= 0 || m_checks <= 0) QKD_FAIL(QKDREC_ERR_ARG, "n=%d m_checks=%d must be positive", n, m_checks);
    if (!row_ptr || !col_idx) QKD_FAIL(QKDREC_ERR_ARG, "row_ptr/col_idx NULL");
    const int32_t M = m_checks;
    if (row_ptr[0] != 0) QKD_FAIL(QKDREC_ERR_CSR, "row_ptr[0] = %d, expected 0", row_ptr[0]);
    int32_t dc_max = 0, dc_min = INT32_MAX;
    for (int32_t c = 0; c < M; ++c) {
        int32_t d = row_ptr[c + 1] - row_ptr[c];
        if (d < 2) QKD_FAIL(QKDREC_ERR_CSR, "check %d has degree %d (< 2)", c, d);
        dc_max = std::max(dc_max, d);
        dc_min = std::min(dc_min, d);
    }
    const int64_t E = row_ptr[M];
    std::vector<int32_t> vdeg(n, 0), stamp(n, -1);
    for (int32_t c = 0; c < M; ++c)
        for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) {
            int32_t v = col_idx[e];
            if (v < 0 || v >= n) QKD_FAIL(QKDREC_ERR_CSR, "col_idx[%d] = %d outside [0, %d)", e, v, n);
            if (stamp[v] == c) QKD_FAIL(QKDREC_ERR_CSR, "variable %d appears twice in check %d", v, c);
            stamp[v] = c;
            vdeg[v]++;
        }
    int32_t dv_max = 0;
    for (int32_t v = 0; v < n; ++v) dv_max = std::max(dv_max, vdeg[v]);

    // variable -> edges (ascending edge index)
    std::vector<int32_t> vptr(n + 1, 0), vedge(E > 0 ? E : 1), fill(n);
    for (int32_t v = 0; v < n; ++v) vptr[v + 1] = vptr[v] + vdeg[v];
    for (int32_t v = 0; v < n; ++v) fill[v] = vptr[v];
    for (int64_t e = 0; e < E; ++e) vedge[fill[col_idx[e]]++] = (int32_t)e;

    // greedy first-fit layers, checks in index order
    std::vector<int32_t> layer_of(M);
    std::vector<std::vector<int32_t>> used(n);
    std::vector<int32_t> taken;
    int32_t n_layers = 0;
    for (int32_t c = 0; c < M; ++c) {
        taken.clear();
        for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e)
            for (int32_t l : used[col_idx[e]]) taken.push_back(l);
        std::sort(taken.begin(), taken.end());
        int32_t lay = 0;
        for (int32_t l : taken) {
            if (l == lay) ++lay;
            else if (l > lay) break;
        }
        layer_of[c] = lay;
        n_layers = std::max(n_layers, lay + 1);
        for (int32_t e = row_ptr[c]; e < row_ptr[c + 1]; ++e) used[col_idx[e]].push_back(lay);
    }
    std::vector<int32_t> lptr(n_layers + 1, 0), lchk(M);
    for (int32_t c = 0; c < M; ++c) lptr[layer_of[c] + 1]++;
    for (int32_t l = 0; l < n_layers; ++l) lptr[l + 1] += lptr[l];
    {
        std::vector<int32_t> f2(lptr.begin(), lptr.end() - 1);
        for (int32_t c = 0; c < M; ++c) lchk[f2[layer_of[c]]++] = c;
    }

    qkdrec_code_t h = new (std::nothrow) qkdrec_code_s();
    if (!h) QKD_FAIL(QKDREC_ERR_NOMEM, "host allocation");
    CodeDev &d = h->d;
    d.n = n;
    d.M = M;
    d.E = E;
    d.dc_max = dc_max;
    d.dc_min = dc_min;
    d.dv_max = dv_max;
    d.n_layers = n_layers;
    d.seed = seed;
    cudaGetDevice(&d.device);
    d.h_layer_of = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
    if (!d.h_layer_of) {
        delete h;
        QKD_FAIL(QKDREC_ERR_NOMEM, "host allocation");
    }
    memcpy(d.h_layer_of, layer_of.data(), sizeof(int32_t) * (size_t)M);
    d.h_layer_ptr = lptr;
    qkdrec_status st;
    if ((st = upload(&d.rp, row_ptr, (size_t)M + 1)) != QKDREC_OK ||
        (st = upload(&d.ci, col_idx, (size_t)E)) != QKDREC_OK ||
        (st = upload(&d.vptr, vptr.data(), (size_t)n + 1)) != QKDREC_OK ||
        (st = upload(&d.vedge, vedge.data(), (size_t)E)) != QKDREC_OK ||
        (st = upload(&d.layer_ptr, lptr.data(), (size_t)n_layers + 1)) != QKDREC_OK ||
        (st = upload(&d.layer_chk, lchk.data(), (size_t)M)) != QKDREC_OK) {
        free_code(d);
        delete h;
        return st;
    }
    *out = h;
    return QKDREC_OK;
}

void qkdrec_code_destroy(qkdrec_code_t code) {
    if (!code) return;
    free_code(code->d);
    delete code;
}

qkdrec_status qkdrec_code_info(qkdrec_code_t code, int32_t *n, int32_t *m_checks, int64_t *edges,
                               int32_t *n_layers, int32_t *dc_max) {
    clear_error();
    if (!code) QKD_FAIL(QKDREC_ERR_ARG, "code is NULL");
    if (n) *n = code->d.n;
    if (m_checks) *m_checks = code->d.M;
    if (edges) *edges = code->d.E;
    if (n_layers) *n_layers = code->d.n_layers;
    if (dc_max) *dc_max = code->d.dc_max;
    return QKDREC_OK;
}

qkdrec_status qkdrec_code_set_qc(qkdrec_code_t code, int32_t Z, int32_t mb, int32_t nb, const int32_t *shifts,
                                 int32_t tma_staging) {
    clear_error();
    if (!code || !shifts) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    CodeDev &d = code->d;
    if (Z < 1 || mb < 1 || nb < 2) QKD_FAIL(QKDREC_ERR_ARG, "need Z >= 1, mb >= 1, nb >= 2");
    if ((int64_t)nb * Z != d.n || (int64_t)mb * Z != d.M || (int64_t)mb * Z * nb != d.E)
        QKD_FAIL(QKDREC_ERR_ARG, "n = %d, M = %d, E = %lld do not match a %d x %d base matrix of %d x %d circulants",
                 d.n, d.M, (long long)d.E, mb, nb, Z, Z);
    for (int32_t t = 0; t < mb * nb; ++t)
        if (shifts[t] < 0 || shifts[t] >= Z) QKD_FAIL(QKDREC_ERR_ARG, "shift %d outside [0, %d)", shifts[t], Z);
    std::vector<int32_t> rp((size_t)d.M + 1), ci((size_t)d.E);
    QKD_CUDA(cudaMemcpy(rp.data(), d.rp, rp.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    QKD_CUDA(cudaMemcpy(ci.data(), d.ci, ci.size() * sizeof(int32_t), cudaMemcpyDeviceToHost));
    for (int32_t c = 0; c < d.M; ++c) {
        const int32_t i = c / Z, z = c - i * Z;
        if (rp[c] != (int64_t)c * nb) QKD_FAIL(QKDREC_ERR_CSR, "check %d does not have degree %d", c, nb);
        for (int32_t k = 0; k < nb; ++k)
            if (ci[(size_t)c * nb + k] != k * Z + (z + shifts[i * nb + k]) % Z)
                QKD_FAIL(QKDREC_ERR_CSR, "check %d edge %d is not the circulant entry of base (%d, %d)", c, k, i, k);
        if (d.h_layer_of[c] != i)
            QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "layer partition differs from the base rows at check %d", c);
    }
    if (d.n_layers != mb) QKD_FAIL(QKDREC_ERR_UNSUPPORTED, "%d layers for %d base rows", d.n_layers, mb);
    int32_t *dev = nullptr;
    QKD_CUDA(cudaMalloc(&dev, sizeof(int32_t) * (size_t)mb * nb));
    cudaError_t e = cudaMemcpy(dev, shifts, sizeof(int32_t) * (size_t)mb * nb, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        QKD_FAIL(QKDREC_ERR_CUDA, "cudaMemcpy: %s", cudaGetErrorString(e));
    }
    cudaFree(d.qc_shift);
    d.qc_shift = dev;
    d.qc_Z = Z;
    d.qc_mb = mb;
    d.qc_nb = nb;
    d.qc_tma = tma_staging ? 1 : 0;
    return QKDREC_OK;
}

qkdrec_status qkdrec_make_regular_code(uint64_t seed, int32_t n, int32_t m_checks, int32_t dv,
                                       int32_t **row_ptr, int32_t **col_idx, int32_t *cycles4_left) {
    clear_error();
    if (!row_ptr || !col_idx) QKD_FAIL(QKDREC_ERR_ARG, "row_ptr/col_idx NULL");
    *row_ptr = nullptr;
    *col_idx = nullptr;
    const int64_t E = (int64_t)dv * n;
    if (n <= 0 || dv <= 0 || m_checks <= 0 || m_checks > E || E > INT32_MAX)
        QKD_FAIL(QKDREC_ERR_ARG, "n=%d m_checks=%d dv=%d: need n, dv > 0 and 0 < m_checks <= dv n < 2^31", n,
                 m_checks, dv);
    if ((E + m_checks - 1) / m_checks > n)
        QKD_FAIL(QKDREC_ERR_ARG, "check degree %lld above n=%d", (long long)((E + m_checks - 1) / m_checks), n);
    int32_t *rp = (int32_t *)malloc(sizeof(int32_t) * ((size_t)m_checks + 1));
    int32_t *ci = (int32_t *)malloc(sizeof(int32_t) * (size_t)E);
    if (!rp || !ci) {
        free(rp);
        free(ci);
        QKD_FAIL(QKDREC_ERR_NOMEM, "host allocation of %lld edges", (long long)E);
    }
    const int64_t res = synth_make_regular_code(seed, n, m_checks, dv, 100, rp, ci);
    if (res < 0) {
        free(rp);
        free(ci);
        QKD_FAIL(QKDREC_ERR_NOMEM, "code construction ran out of host memory");
    }
    *row_ptr = rp;
    *col_idx = ci;
    if (cycles4_left) *cycles4_left = res > INT32_MAX ? INT32_MAX : (int32_t)res;
    return QKDREC_OK;
}

void qkdrec_free(void *p) { free(p); }

qkdrec_status qkdrec_code_rate(double capacity, double fraction, int32_t denom, double *rate) {
    clear_error();
    if (!rate) QKD_FAIL(QKDREC_ERR_ARG, "rate is NULL");
    if (!isfinite(capacity) || !isfinite(fraction) || fraction < 0.0 || denom < 2 || denom > (1 << 20))
        QKD_FAIL(QKDREC_ERR_ARG, "capacity=%g fraction=%g denom=%d", capacity, fraction, denom);
    // nearest multiple of 1/denom, ties up; at most (denom - 1)/denom; 0 = disclosed
    double k = floor(fraction * capacity * denom + 0.5);
    k = std::min(std::max(k, 0.0), (double)(denom - 1));
    *rate = k / denom;
    return QKDREC_OK;
}

qkdrec_status qkdrec_checks_for_rate(int32_t n, double rate, int32_t *m_checks) {
    clear_error();
    if (!m_checks) QKD_FAIL(QKDREC_ERR_ARG, "m_checks is NULL");
    if (n <= 0 || !(rate >= 0.0) || !(rate < 1.0)) QKD_FAIL(QKDREC_ERR_ARG, "n=%d rate=%g", n, rate);
    const double m = nearbyint((double)n * (1.0 - rate));   // nearest, ties to even
    if (m < 1.0 || m > n) QKD_FAIL(QKDREC_ERR_ARG, "rate %g gives %g checks for n=%d", rate, m, n);
    *m_checks = (int32_t)m;
    return QKDREC_OK;
}

qkdrec_status qkdrec_quantiser_range(double snr, double va, double *lo, double *hi) {
    clear_error();
    if (!lo || !hi) QKD_FAIL(QKDREC_ERR_ARG, "lo/hi NULL");
    if (!(snr > 0.0) || !(va > 0.0) || !isfinite(snr) || !isfinite(va))
        QKD_FAIL(QKDREC_ERR_ARG, "snr=%g va=%g must be positive", snr, va);
    const double sy = sqrt(va + 1.0 / snr);   // model sigma_y of y = x + n
    *lo = -4.0 * sy;
    *hi = 4.0 * sy;
    return QKDREC_OK;
}

qkdrec_status qkdrec_reconciliation_efficiency(double snr, int32_t m, double lo, double hi, double va,
                                               const double *rates, double *beta, double *entropy) {
    clear_error();
    if (!rates || !beta) QKD_FAIL(QKDREC_ERR_ARG, "rates/beta NULL");
    if (!(snr > 0) || !(va > 0) || m < 1 || m > 16 || !(lo < hi))
        QKD_FAIL(QKDREC_ERR_ARG, "bad arguments (snr=%g m=%d lo=%g hi=%g va=%g)", snr, m, lo, hi, va);
    // Pi(M(Y)): entropy of Bob's quantised value, y ~ N(0, va + 1/snr), 2^m bins
    const int K = 1 << m;
    const double sy = sqrt(va + 1.0 / snr), r2 = 0.70710678118654752440;
    auto cdf = [&](double t) { return isinf(t) ? (t > 0 ? 1.0 : 0.0) : 0.5 * erfc(-t / sy * r2); };
    double H = 0.0, sum_r = 0.0;
    for (int k = 0; k < K; ++k) {
        const double a = k == 0 ? -INFINITY : lo + (hi - lo) * k / K;
        const double b = k == K - 1 ? INFINITY : lo + (hi - lo) * (k + 1) / K;
        // the smaller tail difference, so an outer bin keeps its relative precision
        const double P = (a >= 0.0) ? 0.5 * (erfc(a / sy * r2) - erfc(b / sy * r2)) : cdf(b) - cdf(a);
        if (P > 0) H -= P * log2(P);
    }
    for (int j = 0; j < m; ++j) {
        if (!(rates[j] >= 0.0 && rates[j] < 1.0)) QKD_FAIL(QKDREC_ERR_ARG, "rate[%d]=%g outside [0, 1)", j, rates[j]);
        sum_r += rates[j];
    }
    const double iab = 0.5 * log2(1.0 + va * snr);   // I(X;Y) of the Gaussian channel, bits per sample
    *beta = (H - m + sum_r) / iab;
    if (entropy) *entropy = H;
    return QKDREC_OK;
}

qkdrec_status qkdrec_code_layers(qkdrec_code_t code, int32_t *layer_of_check) {
    clear_error();
    if (!code || !layer_of_check) QKD_FAIL(QKDREC_ERR_ARG, "NULL argument");
    memcpy(layer_of_check, code->d.h_layer_of, sizeof(int32_t) * (size_t)code->d.M);
    return QKDREC_OK;
}

// ------------------------------------------------------------------ capacity
// Interval probability P(k | x) = Phi(b) - Phi(a), from complementary error
// functions on the side of x the interval lies on.
static double host_interval_prob(double tlo, double thi, double x, double sn) {
    const double r2 = 0.70710678118654752440;
    double a = (tlo - x) / sn, b = (thi - x) / sn;
    if (a >= 0.0) return 0.5 * (erfc(a * r2) - erfc(b * r2));
    if (b <= 0.0) return 0.5 * (erfc(-b * r2) - erfc(-a * r2));
    return 1.0 - 0.5 * erfc(-a * r2) - 0.5 * erfc(b * r2);
}

qkdrec_status qkdrec_slice_capacity(double snr, int32_t m, int32_t j, double lo, double hi,
                                    qkdrec_label label, double va, double *capacity) {
    clear_error();
    if (!capacity) QKD_FAIL(QKDREC_ERR_ARG, "capacity is NULL");
    if (!(snr > 0) || !(va > 0) || m < 1 || m > 8 || j < 0 || j >= m || !(lo < hi))
        QKD_FAIL(QKDREC_ERR_ARG, "bad arguments (snr=%g m=%d j=%d lo=%g hi=%g va=%g)", snr, m, j, lo, hi, va);
    const int K = 1 << m;
    const double sn = 1.0 / sqrt(snr);
    std::vector<double> t(K + 1);
    t[0] = -INFINITY;
    t[K] = INFINITY;
    for (int k = 1; k < K; ++k) t[k] = lo + (hi - lo) * k / K;
    std::vector<int> lab(K);
    for (int k = 0; k < K; ++k) lab[k] = label == QKDREC_LABEL_BINARY ? k : (k ^ (k >> 1));
    const int npts = 20001;  // composite Simpson, odd point count
    const double L = 12.0 * sqrt(va), h = 2.0 * L / (npts - 1);
    const int lowmask = (1 << j) - 1;
    std::vector<double> P(K), p0(1 << j), p1(1 << j);
    double acc = 0.0;
    for (int i = 0; i < npts; ++i) {
        double x = -L + h * i;
        for (int k = 0; k < K; ++k) P[k] = host_interval_prob(t[k], t[k + 1], x, sn);
        std::fill(p0.begin(), p0.end(), 0.0);
        std::fill(p1.begin(), p1.end(), 0.0);
        for (int k = 0; k < K; ++k) {
            int low = lab[k] & lowmask;
            if ((lab[k] >> j) & 1) p1[low] += P[k];
            else p0[low] += P[k];
        }
        double Hx = 0.0;
        for (int low = 0; low < (1 << j); ++low) {
            double s = p0[low] + p1[low];
            if (p0[low] > 0) Hx -= p0[low] * log2(p0[low] / s);
            if (p1[low] > 0) Hx -= p1[low] * log2(p1[low] / s);
        }
        double w = (i == 0 || i == npts - 1) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        double dens = exp(-x * x / (2.0 * va)) / sqrt(2.0 * M_PI * va);
        acc += w * dens * Hx;
    }
    *capacity = 1.0 - acc * h / 3.0;
    return QKDREC_OK;
}

}  // extern "C"
