"""Pins for the oracle's conditional slice capacities and the code-rate rule.

The capacities follow Sec. II Step 5 / Sec. III-B ("closest to the capacity")
and are bound by the chain rule and the Slepian-Wolf inequality of Eqs. beta2
and SWB; the checks below use those identities, an independent direct
entropy of the quantised output, the Shannon bound 1/2 log2(1 + SNR), and a
special case (one slice) that reduces to a binary-input textbook integral.
"""
import mpmath as mp
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("snr,m", [(3.0, 4), (15.0, 5), (2.0, 3)])
def test_chain_rule(snr, m):
    hs = [oracle.slice_cond_entropy(snr, m, j) for j in range(m)]
    assert abs(sum(hs) - oracle.total_cond_entropy(snr, m)) < 1e-9


@pytest.mark.parametrize("snr,m", [(3.0, 4), (15.0, 5)])
def test_two_integrators_agree(snr, m):
    for j in range(m):
        a = oracle.slice_cond_entropy(snr, m, j, method="simpson")
        b = oracle.slice_cond_entropy(snr, m, j, method="quad")
        assert abs(a - b) < 1e-9


@pytest.mark.parametrize("snr", [2.0, 3.0, 15.0])
def test_mutual_information_below_shannon_and_converging(snr):
    cap = 0.5 * np.log2(1 + snr)
    prev = 0.0
    for m in (2, 4, 6):
        ikx = oracle.label_entropy(snr, m) - oracle.total_cond_entropy(snr, m)
        # Slepian-Wolf / data processing: I(M(Y);X) <= I(X;Y) = 1/2 log2(1+SNR)
        assert ikx <= cap + 1e-12
        assert ikx >= prev - 1e-12      # finer quantiser keeps more information
        prev = ikx
    assert prev > 0.95 * cap


def test_one_slice_is_binary_textbook_integral():
    # m = 1, symmetric range: B = [y >= 0]; H(B|X) = E_x h2(Phi(x / sigma_n)).
    snr = 3.0
    sn = 1 / mp.sqrt(snr)
    mp.mp.dps = 30

    def h2(p):
        return 0 if p <= 0 or p >= 1 else -(p * mp.log(p, 2) + (1 - p) * mp.log(1 - p, 2))

    ref = mp.quad(lambda x: mp.npdf(x) * h2(mp.ncdf(x / sn)), [-12, -3, 0, 3, 12])
    assert abs(oracle.slice_cond_entropy(snr, 1, 0) - float(ref)) < 1e-9


def test_capacities_in_unit_interval_and_rates():
    for snr in (2.0, 3.0, 15.0):
        for j in range(5):
            c = oracle.slice_capacity(snr, 5, j)
            assert -1e-12 <= c <= 1 + 1e-12


def test_rate_rule_hand_values():
    # r = round(0.95 C * 64) / 64, ties up, capped at 63/64, r <= 0 disclosed
    assert oracle.code_rate(0.5) == 30 / 64          # 30.4 -> 30
    assert oracle.code_rate(30.5 / 64 / 0.95) == 31 / 64   # exact tie -> up
    assert oracle.code_rate(0.999) == 61 / 64        # 60.7 -> 61
    assert oracle.code_rate(1.0) == 61 / 64          # 60.8 -> 61
    assert oracle.code_rate(0.005) == 0.0            # 0.304 -> 0: disclosed
    assert oracle.code_rate(2.0) == 63 / 64          # cap


def test_beta_identity():
    # Eq. beta vs Eq. beta2: Pi(M(Y)) - m + sum R_j  ==  Pi(M(Y)) - R_s, R_s = sum (1 - R_j),
    # and with R_j = C_j the efficiency numerator equals I(M(Y); X) (Slepian-Wolf tight).
    snr, m = 3.0, 5
    caps = [oracle.slice_capacity(snr, m, j) for j in range(m)]
    HK = oracle.label_entropy(snr, m)
    num = HK - m + sum(caps)
    ikx = HK - oracle.total_cond_entropy(snr, m)
    assert abs(num - ikx) < 1e-9
