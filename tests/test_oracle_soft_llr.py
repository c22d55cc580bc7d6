"""Pins for the oracle's soft-conditioned slice LLR (lower slices known softly).

* Known lower bits (infinite lower LLRs) reduce it to the hard-conditioned
  slice LLR; large finite lower LLRs come within e^-L of it.
* No lower information (lower LLRs 0): the Gray MSB is the sign of y, so its
  LLR is the textbook ln Phi(-x/s) / Phi(x/s) whatever the quantiser.
* Brute force at 50 digits (mpmath) on a 2-slice quantiser with random lower
  LLRs: enumerate every interval, weight by the exact lower-bit probabilities.
"""
import mpmath as mp
import numpy as np
import pytest
from scipy.special import log_ndtr

import oracle
import synth


@pytest.mark.parametrize("m,j,label", [(5, 2, "gray"), (5, 4, "gray"), (4, 3, "binary"), (5, 1, "gray")])
def test_infinite_lower_llrs_reduce_to_hard_conditioning(m, j, label):
    snr = 3.0
    lo, hi = oracle.quantiser_range(snr)
    x, y = synth.gaussian_pair(90, 4000, snr)
    _, bits = oracle.quantise(y, m, lo, hi, label)
    post = np.where(bits[:j] == 0, np.inf, -np.inf)
    soft = oracle.slice_llr_soft(x, post, j, m, lo, hi, snr ** -0.5, label)
    hard = oracle.slice_llr(x, bits[:j], j, m, lo, hi, snr ** -0.5, label)
    assert np.max(np.abs(soft - hard)) < 1e-9
    # large but finite lower LLRs: the other candidates enter with weight e^-60
    post60 = np.where(bits[:j] == 0, 60.0, -60.0)
    soft60 = oracle.slice_llr_soft(x, post60, j, m, lo, hi, snr ** -0.5, label)
    assert np.max(np.abs(soft60 - hard)) < 1e-6


@pytest.mark.parametrize("snr,m", [(3.0, 5), (15.0, 4), (2.0, 6)])
def test_no_lower_information_gray_msb_is_the_sign_of_y(snr, m):
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    x = np.linspace(-3.0, 3.0, 301)
    j = m - 1
    soft = oracle.slice_llr_soft(x, np.zeros((j, x.size)), j, m, lo, hi, s, "gray")
    ref = np.clip(log_ndtr(-x / s) - log_ndtr(x / s), -oracle.LLR_CLIP, oracle.LLR_CLIP)
    assert np.max(np.abs(soft - ref)) < 1e-9


def test_brute_force_two_slices_random_lower_llrs():
    mp.mp.dps = 50
    m, j, snr = 2, 1, 3.0
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    g = np.random.default_rng(7)
    x = g.normal(size=40) * 1.3
    L0 = g.normal(size=40) * 3.0
    got = oracle.slice_llr_soft(x, L0[None, :], j, m, lo, hi, s, "gray")
    t = [mp.mpf(lo + (hi - lo) * k / 4) for k in range(1, 4)]
    edges = [mp.ninf] + t + [mp.inf]
    lab = [k ^ (k >> 1) for k in range(4)]
    for i in range(x.size):
        xi, Li = mp.mpf(x[i]), mp.mpf(L0[i])
        num = [mp.mpf(0), mp.mpf(0)]
        for k in range(4):
            p = mp.ncdf((edges[k + 1] - xi) / s) - mp.ncdf((edges[k] - xi) / s)
            b0 = lab[k] & 1
            w = 1 / (1 + mp.exp(-Li)) if b0 == 0 else 1 / (1 + mp.exp(Li))
            num[(lab[k] >> 1) & 1] += p * w
        ref = float(mp.log(num[0]) - mp.log(num[1]))
        ref = min(max(ref, -oracle.LLR_CLIP), oracle.LLR_CLIP)
        assert abs(got[i] - ref) < 1e-9 * max(1.0, abs(ref)), (i, got[i], ref)
