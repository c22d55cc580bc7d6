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

#ifdef __cplusplus
}
#endif
#endif /* QKDREC_SELFTEST_H */
