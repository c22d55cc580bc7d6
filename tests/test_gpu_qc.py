"""GPU: layered offset min-sum of quasi-cyclic codes with TMA-staged posteriors.

The QC path must give exactly the results of the generic layered decoder on the
same parity-check matrix (bits, iterations, flags, posteriors), match the
oracle's layered decoder after fixed iterations, report no tile-copy timeout,
and reject a structure that does not match the CSR.
"""
import numpy as np
import pytest

import oracle
import synth
from _workloads import bpsk_frames, rel_ok

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def pair(seed, Z, nb):
    rp, ci, S, res = synth.make_qc_code(seed, Z, nb)
    assert res == 0
    n = nb * Z
    plain = q.Code(n, rp, ci)
    qc = q.Code(n, rp, ci)
    qc.set_qc(Z, 3, nb, S)
    return rp, ci, S, plain, qc


def decode(code, llr, s, iters, early):
    return q.qkdrec_decode_batch(code, dev(llr), s, q.DecodeOpts(algo="oms_layered", prec="f32", max_iter=iters,
                                                                 early_stop=early), want_post=True)


@pytest.mark.parametrize("Z,nb,F,sigma", [(512, 6, 37, 0.85), (128, 24, 70, 0.42), (1000, 8, 5, 0.7),
                                           (8192, 24, 64, 0.42)])
@pytest.mark.parametrize("iters,early", [(40, True), (6, False)])
def test_qc_path_identical_to_generic_layered(Z, nb, F, sigma, iters, early):
    rp, ci, S, plain, qc = pair(70 + nb, Z, nb)
    n = nb * Z
    b, llr = bpsk_frames(71 + Z, F, n, sigma)
    s = q.qkdrec_syndrome(plain, dev(b))
    before = q.qkdrec_qc_timeouts()
    g = decode(plain, llr, s, iters, early)
    t = decode(qc, llr, s, iters, early)
    torch.cuda.synchronize()
    for k in ("bits", "iters", "converged", "post"):
        assert torch.equal(g[k], t[k]), k
    assert q.qkdrec_qc_timeouts() == before


def test_qc_path_vs_oracle_after_fixed_iterations():
    Z, nb, F = 256, 6, 9
    rp, ci, S, plain, qc = pair(80, Z, nb)
    b, llr = bpsk_frames(81, F, nb * Z, 0.85)
    s_ref = oracle.syndrome(rp, ci, b)
    t = decode(qc, llr, dev(s_ref), 3, False)
    ref = oracle.decode(rp, ci, llr.astype(np.float64), s_ref, "oms_layered", max_iter=3, early_stop=False,
                        offset=0.5)
    assert rel_ok(t["post"].cpu().numpy(), ref["post"]).all()


def test_set_qc_rejects_a_structure_that_does_not_match():
    Z, nb = 64, 6
    rp, ci, S, res = synth.make_qc_code(90, Z, nb)
    c = q.Code(nb * Z, rp, ci)
    bad = S.copy()
    bad[1, 2] = (bad[1, 2] + 1) % Z
    with pytest.raises(RuntimeError):
        c.set_qc(Z, 3, nb, bad)
    with pytest.raises(RuntimeError):
        c.set_qc(Z + 1, 3, nb, S)
    c.set_qc(Z, 3, nb, S)
