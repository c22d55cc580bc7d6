"""Re-packing of the still-decoding frames during a flooding decode.

After iterations 16, 32 and 64 (flooding schedule, every message precision)
the frames that have not stopped move, with
their messages, posteriors, channel values and syndrome bits, to the front of
the other half of the workspace, and the stopped ones leave with their final
outputs.  Every frame is decoded on its own, so where it sits must not change
anything: the same frames decoded in another order (and so re-packed into
other positions) give bit-identical bits, posteriors, iteration counts and
flags.
"""
import numpy as np
import pytest

import oracle
from _workloads import bpsk_frames, code

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


@pytest.mark.parametrize("algo,prec", [("sp_flood", "f32"), ("oms_flood", "f32"), ("oms_flood", "f16"),
                                       ("oms_flood", "i8"), ("sp_flood", "f16")])
def test_repacking_leaves_every_frame_unchanged(algo, prec):
    n, F = 1024, 333
    rp, ci, _ = code(700, n, 0.5)
    b, llr = bpsk_frames(701, F, n, 0.9)          # near the threshold: 1 to 100 iterations
    c = q.Code(n, rp, ci)
    s = oracle.syndrome(rp, ci, b)
    opts = q.DecodeOpts(algo=algo, prec=prec, max_iter=100)
    res = []
    for perm in (np.arange(F), np.arange(F)[::-1], np.random.default_rng(2).permutation(F)):
        out = q.qkdrec_decode_batch(c, dev(llr[perm]), dev(s[perm]), opts, want_post=True)
        inv = np.argsort(perm)
        res.append({k: out[k].cpu().numpy()[inv] for k in ("bits", "iters", "converged", "post")})
    it = res[0]["iters"]
    assert (it > 16).sum() > 10 and (it > 32).sum() > 2 and (it == 100).sum() > 0   # every re-packing ran
    for r in res[1:]:
        for k in r:
            assert np.array_equal(r[k], res[0][k]), k
    # and the decodes are right: converged words satisfy the syndrome
    conv = res[0]["converged"].astype(bool)
    assert np.array_equal(oracle.syndrome(rp, ci, res[0]["bits"][conv]), s[conv])


def test_repacking_matches_the_oracle_iteration_by_iteration_for_converging_frames():
    """Frames that converge after a re-packing: identical words to the FP64 oracle
    and the same stopping iteration wherever the oracle's margin is clear."""
    n, F = 2048, 64
    rp, ci, _ = code(710, n, 0.5)
    b, llr = bpsk_frames(711, F, n, 0.88)
    c = q.Code(n, rp, ci)
    s = oracle.syndrome(rp, ci, b)
    out = q.qkdrec_decode_batch(c, dev(llr), dev(s), q.DecodeOpts(algo="sp_flood", max_iter=100))
    ref = oracle.decode(rp, ci, llr, s, "sp_flood", max_iter=100)
    gi, oi = out["iters"].cpu().numpy(), ref["iters"]
    both = out["converged"].cpu().numpy().astype(bool) & ref["converged"].astype(bool)
    late = both & (oi > 16)
    assert late.sum() > 0
    assert np.array_equal(out["bits"].cpu().numpy()[both], ref["bits"][both])
    assert np.mean(gi[both] == oi[both]) > 0.9
