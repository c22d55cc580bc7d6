"""Pins for the oracle's unrolled weighted offset min-sum and its reverse-mode gradient.

* With every scale alpha = 1 and offset beta = b the posteriors must equal the
  plain flooding offset min-sum decoder run for the same number of iterations
  (a separate oracle function).
* The gradient must match central finite differences of the oracle's own loss
  where the loss is smooth; a kink (a min/argmin switch, max(x, 0) at 0, a sign
  change) inside the step is detected by comparing two step sizes, and that
  parameter is skipped.
* On a regular code every check is in degree class 0, so class-1 gradients are
  exactly zero; where alpha = 0 the offset carries no gradient.
"""
import numpy as np
import pytest

import oracle
from _workloads import bpsk_frames, code


def _setup(seed, n, rate, F, sigma):
    rp, ci, M = code(seed, n, rate)
    b, llr = bpsk_frames(seed + 1, F, n, sigma)
    s = oracle.syndrome(rp, ci, b)
    return rp, ci, b, s, llr.astype(np.float64)


def test_unit_weights_reduce_to_offset_min_sum():
    rp, ci, b, s, llr = _setup(500, 256, 0.5, 4, 0.85)
    T = 7
    out = oracle.woms(rp, ci, llr, s, b, np.ones((T, 2)), np.full((T, 2), 0.5), want_post=True)
    ref = oracle.decode(rp, ci, llr, s, "oms_flood", max_iter=T, early_stop=False, offset=0.5)
    assert np.max(np.abs(out["post"] - ref["post"])) < 1e-12
    # loss is the mean binary cross-entropy of P(b=1) = sigmoid(-L)
    L = ref["post"]
    p1 = 1.0 / (1.0 + np.exp(L))
    bce = -(b * np.log(p1) + (1 - b) * np.log(1 - p1))
    assert abs(out["loss"] - bce.mean()) < 1e-12


def _fd_check(rp, ci, b, s, llr, alpha, beta, classes):
    out = oracle.woms(rp, ci, llr, s, b, alpha, beta)
    checked, total = 0, 0
    for name, P, G in (("alpha", alpha, out["galpha"]), ("beta", beta, out["gbeta"])):
        for t in range(P.shape[0]):
            for d in classes:
                total += 1
                fd = []
                for h in (1e-4, 1e-5):
                    pp, pm = P.copy(), P.copy()
                    pp[t, d] += h
                    pm[t, d] -= h
                    a_p, b_p = (pp, beta) if name == "alpha" else (alpha, pp)
                    a_m, b_m = (pm, beta) if name == "alpha" else (alpha, pm)
                    lp = oracle.woms(rp, ci, llr, s, b, a_p, b_p)["loss"]
                    lm = oracle.woms(rp, ci, llr, s, b, a_m, b_m)["loss"]
                    fd.append((lp - lm) / (2 * h))
                if abs(fd[0] - fd[1]) > 1e-9 + 1e-6 * abs(fd[1]):
                    continue                       # a kink inside the step
                checked += 1
                assert abs(G[t, d] - fd[1]) <= 1e-9 + 1e-6 * abs(fd[1]), (name, t, d, G[t, d], fd)
    return out, checked, total


def test_gradient_matches_finite_differences_regular_code():
    rp, ci, b, s, llr = _setup(510, 96, 0.5, 3, 0.9)
    T = 5
    g = np.random.default_rng(1)
    alpha = g.uniform(0.6, 1.2, size=(T, 2))
    beta = g.uniform(0.1, 0.8, size=(T, 2))
    out, checked, total = _fd_check(rp, ci, b, s, llr, alpha, beta, classes=(0,))
    assert checked >= 0.6 * total
    assert np.all(out["galpha"][:, 1] == 0.0) and np.all(out["gbeta"][:, 1] == 0.0)
    assert np.max(np.abs(out["galpha"][:, 0])) > 1e-4


def test_gradient_matches_finite_differences_two_degree_classes():
    rp, ci, b, s, llr = _setup(520, 90, 40 / 90, 3, 0.9)     # 3n/M not an integer
    assert len(set(np.diff(rp).tolist())) == 2
    T = 4
    g = np.random.default_rng(2)
    alpha = g.uniform(0.6, 1.2, size=(T, 2))
    beta = g.uniform(0.1, 0.8, size=(T, 2))
    out, checked, total = _fd_check(rp, ci, b, s, llr, alpha, beta, classes=(0, 1))
    assert checked >= 0.6 * total
    assert np.max(np.abs(out["galpha"][:, 1])) > 1e-5


def test_zero_scale_blocks_offset_gradient():
    rp, ci, b, s, llr = _setup(530, 128, 0.5, 2, 0.9)
    T = 4
    alpha = np.ones((T, 2))
    alpha[2] = 0.0
    out = oracle.woms(rp, ci, llr, s, b, alpha, np.full((T, 2), 0.3))
    assert np.all(out["gbeta"][2] == 0.0)
