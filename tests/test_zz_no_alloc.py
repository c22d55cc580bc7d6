"""The no-allocation decoder entry point (qkdrec_decode_batch_static).

Callers that may not allocate device memory at decode time use the decoder
through a workspace compiled into the library.  Through the C ABI, two calls
in a row (different codes, algorithms and frame counts) must give what the
ordinary entry point gives on the same inputs, and an over-size request must
be refused before anything runs.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from _workloads import bpsk_frames, code

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def _case(seed, n, rate, F, sigma, opts):
    rp, ci, _ = code(seed, n, rate)
    c = q.Code(n, rp, ci)
    b, llr = bpsk_frames(seed + 1, F, n, sigma)
    bd, ld = torch.from_numpy(b).cuda(), torch.from_numpy(llr).cuda()
    s = q.qkdrec_syndrome(c, bd)
    return c, ld, s, opts


def test_static_matches_workspace_entry_point_twice():
    """Two calls in a row on the shared array, then low-precision passes with the
    FP32 re-decode of their failed frames (two layouts laid over the same bytes
    in one call): every output equals the ordinary entry point's, bit for bit
    (both run the same kernels on the same inputs)."""
    cases = [_case(300, 2048, 0.5, 37, 0.85, q.DecodeOpts(algo="sp_flood", max_iter=20)),
             _case(310, 4096, 0.84375, 70, 0.5, q.DecodeOpts(algo="oms_layered", max_iter=15)),
             _case(330, 2048, 0.5, 45, 0.86, q.DecodeOpts(algo="oms_flood", prec="i8", max_iter=12,
                                                          fallback_f32=True)),
             _case(340, 2048, 0.5, 45, 0.86, q.DecodeOpts(algo="oms_flood", prec="f16", max_iter=12,
                                                          fallback_f32="sp"))]
    redone = 0
    for c, ld, s, opts in cases:
        got = q.qkdrec_decode_batch_static(c, ld, s, opts, want_post=True)
        ref = q.qkdrec_decode_batch(c, ld, s, opts, want_post=True)
        torch.cuda.synchronize()
        for k in ("bits", "iters", "converged", "post"):
            assert torch.equal(got[k], ref[k]), (opts, k)
        if opts.fallback_f32:
            first = q.qkdrec_decode_batch(c, ld, s, q.DecodeOpts(algo=opts.algo, prec=opts.prec, max_iter=12))
            redone += int((first["converged"] == 0).sum())
    assert redone > 0          # the re-decode really ran on the shared array


def test_static_rejects_requests_above_its_capacity():
    c, ld, s, opts = _case(320, 4096, 0.5, 8, 0.8, q.DecodeOpts())
    cap = q.qkdrec_decode_static_capacity()
    F = 1
    while q.qkdrec_decode_workspace_size(c, F, opts) <= cap:
        F *= 2
    big_llr = torch.zeros((F, c.n), device="cuda")
    big_s = torch.zeros((F, c.M), dtype=torch.uint8, device="cuda")
    with pytest.raises(q.QkdrecError) as e:
        q.qkdrec_decode_batch_static(c, big_llr, big_s, opts)
    assert e.value.status == q.ERR_ARG and "built-in workspace" in str(e.value)
