/*
 * Self-test hooks of libqkdrec: entry points that expose internal device
 * functions so that tests can check them against reference values.  They are
 * not part of the reconciliation path.
 */
#ifndef QKDREC_SELFTEST_H
#define QKDREC_SELFTEST_H

#include "qkdrec.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * out[i] = phi(clamp(x[i], 1e-30, 30)) as the sum-product check kernels
 * evaluate it, phi(x) = -ln tanh(x / 2) (the check-node function of Sec. III-C's
 * BP decoder in the log-magnitude domain).
 *   x, out  DEVICE float [count].
 * Errors: QKDREC_ERR_ARG (count < 0, NULL with count > 0).
 */
qkdrec_status qkdrec_selftest_phi(const float *x, int64_t count, float *out, void *stream);

/*
 * The same function as the two-frames-per-lane sum-product check kernel
 * evaluates it (pairs of values in packed FP32x2 arithmetic):
 * out[i] = phi(clamp(|x[i]|, 1e-30, 30)).
 *   x, out  DEVICE float [count], 8-byte aligned; count even.
 * Errors: QKDREC_ERR_ARG (count odd or < 0, NULL, misaligned).
 */
qkdrec_status qkdrec_selftest_phi_pair(const float *x, int64_t count, float *out, void *stream);

/*
 * out[i] = Q(|z[i]|), the Gaussian upper tail P(N(0,1) > |z|), as the slice LLR
 * kernel evaluates it at a standardised interval bound (Sec. III-B step 4:
 * P(k | x) is the Gaussian mass of interval k), pairs of values in packed
 * FP32x2 arithmetic.
 *   z, out  DEVICE float [count], 8-byte aligned; count even.
 * Errors: QKDREC_ERR_ARG (count odd or < 0, NULL, misaligned).
 */
qkdrec_status qkdrec_selftest_gauss_tail(const float *z, int64_t count, float *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* QKDREC_SELFTEST_H */
