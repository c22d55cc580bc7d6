"""Pins for the oracle's quantiser, labelling, interval probabilities and slice LLRs.

Each check compares the oracle with something other than itself: a hand-worked
fixture, the Gray-code property, Monte-Carlo draws, arbitrary-precision
(mpmath) evaluation of the defining integrals, symmetry, and the textbook sign
quantiser.
"""
import os

import mpmath as mp
import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_quantiser_hand_example():
    rows = np.loadtxt(os.path.join(GOLDEN, "quantiser_m2.txt"))
    y, k, b0, b1 = rows[:, 0], rows[:, 1], rows[:, 2], rows[:, 3]
    idx, bits = oracle.quantise(y, 2, -2.0, 2.0, "gray")
    assert np.array_equal(idx, k.astype(np.uint8))
    assert np.array_equal(bits[0], b0.astype(np.uint8))
    assert np.array_equal(bits[1], b1.astype(np.uint8))


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5, 6])
def test_gray_labels_are_a_gray_code(m):
    lab = oracle.labels(m, "gray")
    assert sorted(lab.tolist()) == list(range(1 << m))
    for k in range(1, 1 << m):
        assert bin(int(lab[k] ^ lab[k - 1])).count("1") == 1
    assert np.array_equal(oracle.labels(m, "binary"), np.arange(1 << m))


@pytest.mark.parametrize("m", [3, 5])
def test_quantiser_brute_force_sweep(m):
    lo, hi = -2.5, 3.5
    K = 1 << m
    delta = (hi - lo) / K
    # every threshold exactly, plus its float neighbours, plus the far tails
    t = [lo + kk * delta for kk in range(1, K)]
    ys = []
    for tk in t:
        ys += [np.nextafter(tk, -np.inf), tk, np.nextafter(tk, np.inf)]
    ys += [-1e30, lo - 1, hi + 1, 1e30]
    ys = np.array(ys)
    idx, bits = oracle.quantise(ys, m, lo, hi, "binary")
    for y, k in zip(ys, idx):
        # brute force: interval k means t_k <= y < t_{k+1}
        expect = sum(1 for tk in t if y >= tk)
        assert k == expect
    for j in range(m):
        assert np.array_equal(bits[j], (idx >> j) & 1)


def test_quantiser_frequencies_match_model():
    snr, m = 3.0, 5
    lo, hi = oracle.quantiser_range(snr)
    _, y = synth.gaussian_pair(11, 400_000, snr)
    idx, _ = oracle.quantise(y, m, lo, hi)
    sy = np.sqrt(1 + 1 / snr)
    t = [-mp.inf] + [mp.mpf(lo) + k * mp.mpf(hi - lo) / 32 for k in range(1, 32)] + [mp.inf]
    cnt = np.bincount(idx, minlength=32)
    for k in range(32):
        p = float(mp.ncdf(t[k + 1] / sy) - mp.ncdf(t[k] / sy))
        sd = np.sqrt(p * (1 - p) * len(y))
        assert abs(cnt[k] - p * len(y)) <= 5 * sd + 1


def _mp_interval_prob(tlo, thi, x, sigma):
    mp.mp.dps = 60
    a = (mp.mpf(tlo) - mp.mpf(x)) / sigma if np.isfinite(tlo) else -mp.inf
    b = (mp.mpf(thi) - mp.mpf(x)) / sigma if np.isfinite(thi) else mp.inf
    # Phi(b) - Phi(a) = Phi(-a) - Phi(-b): take the form whose terms are small,
    # so 60 digits are never spent on a difference of two numbers near 1.
    if a > 0:
        return mp.ncdf(-a) - mp.ncdf(-b)
    return mp.ncdf(b) - mp.ncdf(a)


def test_interval_probabilities_vs_arbitrary_precision():
    m, lo, hi, sn = 5, -4.6188, 4.6188, 0.25
    t = np.concatenate([[-np.inf], oracle.thresholds(m, lo, hi), [np.inf]])
    xs = np.array([-6.0, -2.2, -0.01, 0.0, 0.3, 1.7, 4.9, 7.5])
    lp = oracle.interval_logprob(xs, m, lo, hi, sn)
    for i, x in enumerate(xs):
        for k in range(32):
            ref = _mp_interval_prob(t[k], t[k + 1], x, mp.mpf(sn))
            ref_log = float(mp.log(ref))
            assert abs(lp[i, k] - ref_log) <= 1e-12 * max(1.0, abs(ref_log)), (x, k)


def test_interval_probabilities_sum_to_one_and_mirror():
    m = 5
    lo, hi = oracle.quantiser_range(15.0)
    xs = np.linspace(-7, 7, 301)
    P = np.exp(oracle.interval_logprob(xs, m, lo, hi, 15.0 ** -0.5))
    assert np.max(np.abs(P.sum(axis=1) - 1.0)) < 1e-14
    Pm = np.exp(oracle.interval_logprob(-xs, m, lo, hi, 15.0 ** -0.5))
    # symmetric quantiser: P(k | x) = P(2^m - 1 - k | -x)
    assert np.max(np.abs(P - Pm[:, ::-1])) < 1e-14


def test_interval_probabilities_monte_carlo():
    m, snr = 4, 3.0
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    g = synth.philox(5)
    N = 2_000_000
    for x in (-1.3, 0.2, 2.4):
        y = x + sn * g.standard_normal(N)
        idx, _ = oracle.quantise(y, m, lo, hi)
        freq = np.bincount(idx, minlength=16) / N
        P = np.exp(oracle.interval_logprob(np.array([x]), m, lo, hi, sn))[0]
        sd = np.sqrt(P * (1 - P) / N)
        assert np.all(np.abs(freq - P) <= 5 * sd + 1e-7)


def test_sign_quantiser_llr_is_textbook():
    # m = 1 with a symmetric range: one threshold at 0, interval 0 <-> y < 0 <-> bit 0,
    # so LLR = ln P(y<0|x)/P(y>=0|x) = ln Phi(-x/s) / Phi(x/s).
    sn = 0.7
    xs = np.array([-9.0, -3.0, -0.5, 0.0, 0.1, 2.0, 8.0])
    llr = oracle.slice_llr(xs, None, 0, 1, -3.0, 3.0, sn, clip=1e9)
    mp.mp.dps = 50
    for x, l in zip(xs, llr):
        ref = mp.log(mp.ncdf(-x / mp.mpf(sn))) - mp.log(mp.ncdf(x / mp.mpf(sn)))
        assert abs(l - float(ref)) <= 1e-12 * max(1.0, abs(float(ref)))


def test_slice_llr_vs_brute_force_candidate_sums():
    # brute force: enumerate all intervals, keep those whose label agrees with the
    # lower bits, split by bit j, sum probabilities at 60 digits.
    m, snr = 4, 3.0
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    t = np.concatenate([[-np.inf], oracle.thresholds(m, lo, hi), [np.inf]])
    g = synth.philox(9)
    xs = g.standard_normal(12) * 1.5
    gray = [k ^ (k >> 1) for k in range(16)]
    for j in range(m):
        low = g.integers(0, 2, size=(j, xs.size)).astype(np.uint8)
        llr = oracle.slice_llr(xs, low if j else None, j, m, lo, hi, sn, clip=1e9)
        for i, x in enumerate(xs):
            lowv = sum(int(low[b, i]) << b for b in range(j))
            s = [mp.mpf(0), mp.mpf(0)]
            for k in range(16):
                if gray[k] & ((1 << j) - 1) != lowv:
                    continue
                s[(gray[k] >> j) & 1] += _mp_interval_prob(t[k], t[k + 1], x, mp.mpf(sn))
            ref = float(mp.log(s[0]) - mp.log(s[1]))
            assert abs(llr[i] - ref) <= 1e-11 * max(1.0, abs(ref)), (j, i)


def test_slice_llr_clip():
    m, snr = 5, 15.0
    lo, hi = oracle.quantiser_range(snr)
    xs = np.array([3.0, -3.0])
    low = np.array([[0, 0], [0, 0], [0, 0], [0, 0]], dtype=np.uint8)
    llr = oracle.slice_llr(xs, low, 4, m, lo, hi, snr ** -0.5)
    assert np.all(np.abs(llr) == oracle.LLR_CLIP)
    # the MSB of the Gray label is the sign of y: positive x -> bit 1 likely -> LLR < 0
    assert llr[0] < 0 < llr[1]
