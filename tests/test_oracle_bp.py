"""Pins for the oracle's BP decoders (Sec. III-C: "the well-known BP decoder").

BP is exact on cycle-free factor graphs: on random trees the sum-product
posteriors must equal the brute-force bit marginals over all 2^n words that
satisfy the syndrome, and offset min-sum with offset 0 must equal the max-log
(max-product) marginals.  Further invariants: a converged output satisfies its
syndrome (checked with a dense GF(2) product, not the oracle's own XOR), a
channel that already agrees with the syndrome stops at iteration 0, the 2-edge
check passes the other LLR through unchanged, and the integer decoder on
exactly representable inputs equals the float decoder scaled by the LSB.
"""
import itertools

import numpy as np
import pytest

import oracle
import synth
from _workloads import bpsk_frames


def random_tree_code(rng, n_target, max_dc=4):
    """Cycle-free factor graph: every new check joins one existing variable to
    d-1 new ones.  Returns CSR (row_ptr, col_idx) and n."""
    rows = []
    n = 1
    while n < n_target:
        d = int(rng.integers(2, max_dc + 1))
        d = min(d, n_target - n + 1)
        old = int(rng.integers(0, n))
        new = list(range(n, n + d - 1))
        row = [old] + new
        rng.shuffle(row)
        rows.append(row)
        n += d - 1
    # shuffle check order and variable labels to avoid structure
    perm = rng.permutation(n)
    rows = [[int(perm[v]) for v in r] for r in rows]
    order = rng.permutation(len(rows))
    rows = [rows[i] for i in order]
    rp = np.zeros(len(rows) + 1, dtype=np.int32)
    rp[1:] = np.cumsum([len(r) for r in rows])
    ci = np.array([v for r in rows for v in r], dtype=np.int32)
    return rp, ci, n


def dense_H(rp, ci, n):
    M = len(rp) - 1
    H = np.zeros((M, n), dtype=np.int64)
    for c in range(M):
        H[c, ci[rp[c]:rp[c + 1]]] = 1
    return H


def brute_marginals(H, s, llr, maxlog):
    """Exact (or max-log) posterior LLRs by enumerating all words with H b = s."""
    n = H.shape[1]
    words = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.int64)
    ok = np.all((words @ H.T) % 2 == s[None, :], axis=1)
    words = words[ok]
    score = ((1 - 2 * words) * llr[None, :] / 2).sum(axis=1)   # log prod P(b_v) + const
    out = np.zeros(n)
    for v in range(n):
        s0, s1 = score[words[:, v] == 0], score[words[:, v] == 1]
        if maxlog:
            out[v] = s0.max() - s1.max()
        else:
            m0, m1 = s0.max(), s1.max()
            out[v] = (m0 + np.log(np.exp(s0 - m0).sum())) - (m1 + np.log(np.exp(s1 - m1).sum()))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_sp_exact_on_trees(seed):
    rng = np.random.default_rng(100 + seed)
    rp, ci, n = random_tree_code(rng, 12)
    H = dense_H(rp, ci, n)
    llr = rng.normal(0.0, 2.0, size=n)
    s = rng.integers(0, 2, size=H.shape[0])
    ref = brute_marginals(H, s, llr, maxlog=False)
    out = oracle.decode(rp, ci, llr[None, :], s[None, :].astype(np.uint8), "sp_flood",
                        max_iter=2 * n, early_stop=False)
    assert np.max(np.abs(out["post"][0] - ref)) < 1e-10


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("algo", ["oms_flood", "oms_layered"])
def test_min_sum_offset0_is_maxlog_on_trees(seed, algo):
    rng = np.random.default_rng(200 + seed)
    rp, ci, n = random_tree_code(rng, 12)
    H = dense_H(rp, ci, n)
    llr = rng.normal(0.0, 2.0, size=n)
    s = rng.integers(0, 2, size=H.shape[0])
    ref = brute_marginals(H, s, llr, maxlog=True)
    out = oracle.decode(rp, ci, llr[None, :], s[None, :].astype(np.uint8), algo,
                        max_iter=2 * n, early_stop=False, offset=0.0)
    assert np.max(np.abs(out["post"][0] - ref)) < 1e-10


def test_single_check_maxlog_and_offset():
    # one check over 5 variables: OMS posterior = L_v + (-1)^s prod sgn * max(min|L_other| - beta, 0)
    rp = np.array([0, 5], dtype=np.int32)
    ci = np.arange(5, dtype=np.int32)
    llr = np.array([[1.5, -0.25, 3.0, -2.0, 0.75]])
    H = np.ones((1, 5), dtype=np.int64)
    for s in (0, 1):
        ref = brute_marginals(H, np.array([s]), llr[0], maxlog=True)
        out = oracle.decode(rp, ci, llr, np.array([[s]], dtype=np.uint8), "oms_flood",
                            max_iter=1, early_stop=False, offset=0.0)
        assert np.allclose(out["post"][0], ref, atol=1e-12)
    # with offset 0.5 the hand-computed messages (s=0): others' min magnitudes
    # v0: min(.25,3,2,.75)=.25 -> 0 ; v1: min(1.5,3,2,.75)=.75 -> .25 with sign(+,+,-,+) = -,
    # every other variable sees |-0.25| as its minimum -> 0.
    out = oracle.decode(rp, ci, llr, np.array([[0]], dtype=np.uint8), "oms_flood",
                        max_iter=1, early_stop=False, offset=0.5)
    m = out["post"][0] - llr[0]
    assert np.allclose(m, [0.0, -0.25, 0.0, 0.0, 0.0], atol=1e-12)


def test_sp_two_edge_check_passes_llr_through():
    # a degree-2 check forwards phi(phi(|q|)) = |q| with the syndrome-adjusted sign
    rp = np.array([0, 2], dtype=np.int32)
    ci = np.array([0, 1], dtype=np.int32)
    llr = np.array([[0.8, -2.5]])
    for s in (0, 1):
        out = oracle.decode(rp, ci, llr, np.array([[s]], dtype=np.uint8), "sp_flood",
                            max_iter=1, early_stop=False)
        sign = -1.0 if s else 1.0
        assert np.allclose(out["post"][0], llr[0] + sign * llr[0][::-1], atol=1e-12)


def _random_frames(seed, n=512, rate=0.5, F=6, snr_db=3.0):
    M = synth.checks_for_rate(n, rate)
    rp, ci, _ = synth.make_regular_code(seed, n, M)
    g = synth.philox(seed + 1)
    b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
    H = dense_H(rp, ci, n)
    s = ((b.astype(np.int64) @ H.T) % 2).astype(np.uint8)
    sigma = 10 ** (-snr_db / 20)
    # BPSK-like soft information: llr = 2/sigma^2 * (1 - 2b + noise)
    llr = 2 / sigma**2 * ((1 - 2 * b.astype(np.float64)) + sigma * g.standard_normal((F, n)))
    return rp, ci, b, s, llr, H


@pytest.mark.parametrize("algo", ["sp_flood", "oms_flood", "oms_layered", "ioms_flood", "ioms_layered"])
def test_converged_frames_satisfy_syndrome(algo):
    rp, ci, b, s, llr, H = _random_frames(7)
    out = oracle.decode(rp, ci, llr, s, algo, max_iter=30)
    got = (out["bits"].astype(np.int64) @ H.T) % 2
    for f in range(b.shape[0]):
        sat = np.array_equal(got[f], s[f])
        assert bool(out["converged"][f]) == sat
    assert out["converged"].mean() > 0.5       # the channel is good enough to decode


@pytest.mark.parametrize("algo", ["sp_flood", "oms_flood", "oms_layered", "ioms_flood", "ioms_layered"])
def test_consistent_channel_stops_at_zero(algo):
    rp, ci, b, s, _, _ = _random_frames(8)
    llr = 8.0 * (1 - 2 * b.astype(np.float64))
    out = oracle.decode(rp, ci, llr, s, algo, max_iter=30)
    assert np.all(out["iters"] == 0) and np.all(out["converged"] == 1)
    assert np.array_equal(out["bits"], b)


@pytest.mark.parametrize("layered", [False, True])
def test_integer_min_sum_equals_scaled_float_min_sum(layered):
    # inputs on the 0.5 grid, small enough that no 6-bit clip or int16 saturation
    # occurs: integer OMS (offset 1 LSB) * 0.5 == float OMS with offset 0.5.
    rng = np.random.default_rng(3)
    rp, ci, n = random_tree_code(rng, 14)
    s = rng.integers(0, 2, size=len(rp) - 1).astype(np.uint8)
    llr = rng.integers(-6, 7, size=n) * 0.5
    a1 = "ioms_layered" if layered else "ioms_flood"
    a2 = "oms_layered" if layered else "oms_flood"
    for it in (1, 2, 3, 5):
        oi = oracle.decode(rp, ci, llr[None], s[None], a1, max_iter=it, early_stop=False, llr_step=0.5)
        of = oracle.decode(rp, ci, llr[None], s[None], a2, max_iter=it, early_stop=False, offset=0.5)
        assert np.array_equal(oi["post"], of["post"])


def test_integer_min_sum_hand_example():
    # one check, 3 variables, step 0.5: llr (1.2, -0.3, 20) -> q = (2, -1, 31) after
    # round-half-away and the +-31 clip.  Messages (s = 0): v0 <- sgn(-1*31)=- * (min(1,31)-1)=0,
    # v1 <- + * (min(2,31)-1) = 1, v2 <- - * (min(2,1)-1) = 0.  Posteriors: 2, 0, 31.
    rp = np.array([0, 3], dtype=np.int32)
    ci = np.array([0, 1, 2], dtype=np.int32)
    out = oracle.decode(rp, ci, np.array([[1.2, -0.3, 20.0]]), np.array([[0]], dtype=np.uint8),
                        "ioms_flood", max_iter=1, early_stop=False, llr_step=0.5)
    assert np.array_equal(out["post"][0], np.array([2, 0, 31]) * 0.5)
    # round half away from zero: 0.25/0.5 = 0.5 -> 1, -0.25/0.5 = -0.5 -> -1
    out = oracle.decode(rp, ci, np.array([[0.25, -0.25, 0.75]]), np.array([[0]], dtype=np.uint8),
                        "ioms_flood", max_iter=0, early_stop=False, llr_step=0.5)
    assert np.array_equal(out["post"][0], np.array([1, -1, 2]) * 0.5)


def saturating_codes():
    """Hand codes where the 6-bit clip and the int16 posterior saturation both fire.
    A: n = 2, 1100 checks {0, 1}.  B: A plus a last check {0, 1, 2}.  Every check
    of A meets every other, so the first-fit layers are one check each, in index
    order; B's last check is the last layer."""
    K = 1100
    rpA = np.arange(0, 2 * K + 1, 2, dtype=np.int32)
    ciA = np.tile(np.array([0, 1], np.int32), K)
    rpB = np.append(rpA, 2 * K + 3).astype(np.int32)
    ciB = np.append(ciA, np.array([0, 1, 2], np.int32))
    return (rpA, ciA, 2), (rpB, ciB, 3)


@pytest.mark.parametrize("layered", [False, True])
def test_integer_min_sum_saturation_by_hand(layered):
    """Step 0.5, llr 20 -> 40 LSB, clipped to q = 31.  Code A, syndrome 0:
    every check sends 31 - 1 = 30 to both variables.  Layered: after the k-th
    check L = 31 + 30 k (the v->c value stays clipped at 31 while L grows, so
    L = q_full + m uses the UNclipped q), saturating at 32767 after 1092 checks;
    flooding: L = 31 + 1100 * 30 added in edge order, saturating likewise.  A
    second iteration keeps 32767 (q_full = 32767 - 30, clipped to 31, + 30).
    Clipping q before forming L would give 61; no clip would give a message of
    32766 that int8 cannot hold; no saturation would give 33031."""
    (rp, ci, n), _ = saturating_codes()
    algo = "ioms_layered" if layered else "ioms_flood"
    s = np.zeros((1, len(rp) - 1), np.uint8)
    for it in (1, 2):
        out = oracle.decode(rp, ci, np.array([[20.0, 20.0]]), s, algo, max_iter=it, early_stop=False,
                            llr_step=0.5)
        assert np.array_equal(out["post"][0], [32767 * 0.5, 32767 * 0.5])
    # with the second variable negative the messages cancel to zero after one check
    out = oracle.decode(rp, ci, np.array([[20.0, -20.0]]), s, algo, max_iter=1, early_stop=False, llr_step=0.5)
    # layered: check 0 sends -30 / +30 -> L = (1, -1); every later check then sends
    # max(1 - 1, 0) = 0.  Flooding: all 1100 checks send -30 / +30 from q = (31, -31).
    expect = [1, -1] if layered else [-32767, 32767]
    assert np.array_equal(out["post"][0], np.array(expect) * 0.5)


@pytest.mark.parametrize("layered", [False, True])
def test_integer_min_sum_clip_then_saturation_by_hand(layered):
    """Code B, llr (20, 20, -2) -> (31, 31, -4).  Iteration 1: the 1100 checks
    {0, 1} drive L0 = L1 to 32767; the last check sees q_full = (32767, 32767, -4),
    clipped q = (31, 31, -4): to v0 and v1 sign(31 * -4) (min(31, 4) - 1) = -3, to
    v2 +(31 - 1) = 30.  So L = (32764, 32764, 26) in both schedules (flooding adds
    the last check's -3 after the 1100 saturating +30s, in edge order)."""
    _, (rp, ci, n) = saturating_codes()
    algo = "ioms_layered" if layered else "ioms_flood"
    s = np.zeros((1, len(rp) - 1), np.uint8)
    out = oracle.decode(rp, ci, np.array([[20.0, 20.0, -2.0]]), s, algo, max_iter=1, early_stop=False,
                        llr_step=0.5)
    assert np.array_equal(out["post"][0], np.array([32764, 32764, 26]) * 0.5)
    assert np.array_equal(out["bits"][0], [0, 0, 0])


def test_layered_integer_min_sum_equals_float_min_sum_on_a_real_code():
    """Below the clip and saturation limits the layered integer decoder is the
    float offset min-sum (offset 0.5) on the 0.5 grid, on a real regular code
    (not only trees): LLRs on the grid with |llr| <= 3, so every |q| stays
    below 31 for two iterations (|L| <= 3 + 3 * 3) and nothing saturates."""
    rp, ci, n = (*synth.make_regular_code(77, 256, 128)[:2], 256)
    g = np.random.default_rng(5)
    llr = g.integers(-6, 7, size=(4, n)) * 0.5
    s = g.integers(0, 2, size=(4, len(rp) - 1)).astype(np.uint8)
    for it in (1, 2):
        oi = oracle.decode(rp, ci, llr, s, "ioms_layered", max_iter=it, early_stop=False, llr_step=0.5)
        of = oracle.decode(rp, ci, llr, s, "oms_layered", max_iter=it, early_stop=False, offset=0.5)
        assert np.abs(of["post"]).max() < 31 * 0.5
        assert np.array_equal(oi["post"], of["post"])


def test_layer_partition_valid_and_first_fit():
    rp, ci, _, _, _, _ = _random_frames(9, n=256)
    n = 256
    layer_of, lptr, lchk = oracle.greedy_layers(rp, ci, n)
    M = len(rp) - 1
    assert sorted(lchk.tolist()) == list(range(M))
    for l in range(len(lptr) - 1):
        vs = np.concatenate([ci[rp[c]:rp[c + 1]] for c in lchk[lptr[l]:lptr[l + 1]]])
        assert len(np.unique(vs)) == len(vs)                  # no shared variable in a layer
        assert np.all(layer_of[lchk[lptr[l]:lptr[l + 1]]] == l)
    # first fit: a check in layer l conflicts with an earlier check in every layer < l
    for c in range(M):
        vc = set(ci[rp[c]:rp[c + 1]].tolist())
        for l in range(layer_of[c]):
            assert any(vc & set(ci[rp[d]:rp[d + 1]].tolist()) for d in range(c) if layer_of[d] == l)


def test_syndrome_vs_dense_product():
    rp, ci, b, s, _, H = _random_frames(10)
    assert np.array_equal(oracle.syndrome(rp, ci, b), s)


def test_sum_product_threshold_of_the_regular_3_6_ensemble():
    """Density evolution puts the BP threshold of the regular (3,6) ensemble on the
    binary-input AWGN channel at sigma* = 0.881 (a textbook value of the theory of
    iterative decoding).  A length-8192 code of the seeded construction decodes
    every frame 5 % below it and none 5 % above it within 100 iterations; a
    dropped exclusion term, a sign error or a wrong phi moves that transition."""
    n = 8192
    rp, ci, _ = synth.make_regular_code(190, n, synth.checks_for_rate(n, 0.5))
    for sigma, seed, want in ((0.84, 191, 8), (0.93, 192, 0)):
        b, llr = bpsk_frames(seed, 8, n, sigma)
        out = oracle.decode(rp, ci, llr.astype(np.float64), oracle.syndrome(rp, ci, b), "sp_flood", max_iter=100)
        assert int((out["bits"] == b).all(axis=1).sum()) == want, sigma
        assert int(out["converged"].sum()) == want, sigma
