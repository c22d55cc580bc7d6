"""Seeded workloads shared by the tests (inputs only; no method arithmetic).

Decoder-parity inputs are synthetic: random words b and BPSK-shaped channel
LLRs (2/s^2)((1 - 2b) + s z), so the decoder is exercised from the waterfall
to the error floor; the full slice pipeline (quantiser -> LLR -> decoder) is
exercised separately on the paper's Gaussian quadratures.
"""
import numpy as np

import synth

TOL = 1e-4          # |gpu - oracle| <= TOL * max(|oracle|, 1)  (FP32 vs FP64)


def rel_ok(got, ref, tol=TOL):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.abs(got - ref) <= tol * np.maximum(np.abs(ref), 1.0)


def code(seed, n, rate, dv=3):
    M = synth.checks_for_rate(n, rate)
    rp, ci, _ = synth.make_regular_code(seed, n, M, dv)
    return rp, ci, M


def bpsk_frames(seed, F, n, sigma):
    """Random words uint8 [F][n] and float32 LLRs of them seen through AWGN."""
    g = synth.philox(seed)
    b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
    z = g.standard_normal((F, n))
    llr = (2.0 / sigma**2) * ((1.0 - 2.0 * b) + sigma * z)
    return b, llr.astype(np.float32)


def wilson(k, n, z=1.96):
    """Wilson 95% interval of a binomial proportion."""
    if n == 0:
        return 0.0, 1.0
    p = k / n
    den = 1 + z * z / n
    c = (p + z * z / (2 * n)) / den
    h = z * np.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / den
    return max(0.0, c - h), min(1.0, c + h)
