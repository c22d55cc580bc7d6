"""GPU parity of the low-precision decoder forms against the FP64 oracle.

FP16 messages (FP32 arithmetic, messages stored in binary16): the posteriors
after a fixed number of iterations (no stopping test) must lie within the
oracle's forward error radius of the FP64 posteriors (oracle.decode_bound:
2^-11 relative per stored message, 2^-24 per FP32 operation, the check
function's stated accuracy, propagated through the iterations), and the hard
decisions must equal the oracle's wherever the radius cannot flip them.  Full
decodes: identical words where both converge, FER inside the oracle's Wilson
interval.

6-bit integer min-sum: bit-exact against the oracle on the hand-traced codes
where the +-31 clip and the int16 posterior saturation both fire.
"""
import numpy as np
import pytest

import oracle
from _workloads import bpsk_frames, code, wilson

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402

PHI_REL = 4e-6        # the kernels' phi accuracy, asserted by test_gpu_phi.py


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("algo,T", [("oms_flood", 4), ("sp_flood", 4), ("oms_layered", 3)])
@pytest.mark.parametrize("n,rate,F,sigma", [(2048, 0.5, 40, 0.8), (1024, 0.75, 131, 0.55)])
def test_f16_posteriors_within_the_derived_bound_of_the_fp64_oracle(algo, T, n, rate, F, sigma):
    rp, ci, _ = code(610 + int(rate * 64), n, rate)
    b, llr = bpsk_frames(611, F, n, sigma)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    sh = oracle.syndrome(rp, ci, b)
    worst = 0.0
    for t in range(1, T + 1):
        out = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec="f16", max_iter=t,
                                                                   early_stop=False), want_post=True)
        ref, rad = oracle.decode_bound(rp, ci, llr, sh, algo, t, f16=True, phi_rel=PHI_REL)
        got = host(out["post"]).astype(np.float64)
        gap = np.abs(got - ref)
        bad = gap > rad
        assert not bad.any(), (t, np.argwhere(bad)[:5], got[bad][:5], ref[bad][:5], rad[bad][:5])
        worst = max(worst, float(np.max(gap / np.maximum(rad, 1e-300))))
        sure = np.abs(ref) > rad
        assert sure.mean() > 0.9
        assert np.array_equal(host(out["bits"])[sure], (ref[sure] < 0).astype(np.uint8))
        assert np.all(host(out["iters"]) == t)
    print(f"{algo} n={n}: largest |gpu - oracle| / bound = {worst:.3f}")


@pytest.mark.parametrize("algo", ["oms_flood", "oms_layered", "sp_flood"])
def test_f16_full_decodes_match_the_fp64_oracle(algo):
    n, F = 2048, 96
    rp, ci, _ = code(620, n, 0.5)
    b, llr = bpsk_frames(621, F, n, 0.84)
    c = q.Code(n, rp, ci)
    out = q.qkdrec_decode_batch(c, dev(llr), q.qkdrec_syndrome(c, dev(b)),
                                q.DecodeOpts(algo=algo, prec="f16", max_iter=50))
    ref = oracle.decode(rp, ci, llr, oracle.syndrome(rp, ci, b), algo, max_iter=50)
    gb, gc = host(out["bits"]), host(out["converged"]).astype(bool)
    both = gc & ref["converged"].astype(bool)
    assert both.sum() > F // 2
    assert np.array_equal(gb[both], ref["bits"][both])
    # a converged output satisfies the syndrome
    assert np.array_equal(oracle.syndrome(rp, ci, gb[gc]), oracle.syndrome(rp, ci, b)[gc])
    e_gpu = int(np.sum(np.any(gb != b, axis=1)))
    e_ref = int(np.sum(np.any(ref["bits"] != b, axis=1)))
    lo, hi = wilson(e_ref, F)
    assert lo <= e_gpu / F <= hi, (e_gpu, e_ref)


def saturating_codes():
    """The hand codes of the oracle's saturation pins (tests/test_oracle_bp.py)."""
    K = 1100
    rpA = np.arange(0, 2 * K + 1, 2, dtype=np.int32)
    ciA = np.tile(np.array([0, 1], np.int32), K)
    rpB = np.append(rpA, 2 * K + 3).astype(np.int32)
    ciB = np.append(ciA, np.array([0, 1, 2], np.int32))
    return (rpA, ciA, 2), (rpB, ciB, 3)


@pytest.mark.parametrize("algo", ["oms_flood", "oms_layered"])
def test_integer_min_sum_clip_and_saturation_bit_exact(algo):
    (rpA, ciA, nA), (rpB, ciB, nB) = saturating_codes()
    cases = [(rpA, ciA, nA, [20.0, 20.0]), (rpA, ciA, nA, [20.0, -20.0]), (rpB, ciB, nB, [20.0, 20.0, -2.0])]
    for rp, ci, n, row in cases:
        F = 5                                      # one ragged frame block
        llr = np.tile(np.array(row, np.float32), (F, 1))
        llr[1] *= -1.0                             # and sign-mirrored frames
        llr[3] *= 0.5
        synd = np.zeros((F, len(rp) - 1), np.uint8)
        synd[2, ::3] = 1                           # a syndrome that flips some checks
        c = q.Code(n, rp, ci)
        for it in (0, 1, 2):
            out = q.qkdrec_decode_batch(c, dev(llr), dev(synd), q.DecodeOpts(algo=algo, prec="i8", max_iter=it,
                                                                              early_stop=False), want_post=True)
            ref = oracle.decode(rp, ci, llr, synd, "i" + algo, max_iter=it, early_stop=False, llr_step=0.5)
            assert np.array_equal(host(out["post"]).astype(np.float64), ref["post"]), (row, it)
            assert np.array_equal(host(out["bits"]), ref["bits"])
            assert np.array_equal(host(out["converged"]), ref["converged"])
        if it and row == [20.0, 20.0]:
            assert np.all(ref["post"][0] == 32767 * 0.5)
