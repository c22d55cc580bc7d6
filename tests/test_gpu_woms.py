"""GPU unrolled weighted offset min-sum and its adjoint against the FP64 oracle.

Forward posteriors and loss within 1e-4 relative; the gradient within 1e-4 of
the oracle's FP64 gradient (relative to its largest component); identical
gradients for every checkpoint interval; central finite differences (step
1e-3) of the GPU loss; the full-size workload (1024 frames of a rate-1/2
dv=3/dc=6 code with n = 16384, 20 iterations, checkpoints every 5); and a few
optimiser steps that lower the loss.
"""
import numpy as np
import pytest

import oracle
import synth
from _workloads import TOL, bpsk_frames, code, rel_ok

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


def setup(seed, n, rate, F, sigma):
    rp, ci, M = code(seed, n, rate)
    c = q.Code(n, rp, ci)
    b, llr = bpsk_frames(seed + 1, F, n, sigma)
    s_ref = oracle.syndrome(rp, ci, b)
    s = q.qkdrec_syndrome(c, dev(b))
    assert np.array_equal(s.cpu().numpy(), s_ref)
    return rp, ci, c, b, llr, s, s_ref


def run(c, llr, s, b, alpha, beta, K, want_post=False):
    F = b.shape[0]
    T = alpha.shape[0]
    ws = torch.empty(q.qkdrec_woms_workspace_size(c, F, T, K), dtype=torch.uint8, device="cuda")
    a, bt = dev(alpha.astype(np.float32)), dev(beta.astype(np.float32))
    loss, post = q.qkdrec_woms_forward(c, dev(llr), s, dev(b), a, bt, K, ws, want_post)
    ga, gb = q.qkdrec_woms_backward(c, dev(llr), s, dev(b), a, bt, K, ws)
    return (float(loss.item()), post.cpu().numpy() if want_post else None, ga.cpu().numpy().astype(np.float64),
            gb.cpu().numpy().astype(np.float64))


@pytest.mark.parametrize("n,rate,F", [(512, 0.5, 12), (720, 40 / 90, 9)])
def test_forward_and_gradient_vs_oracle(n, rate, F):
    rp, ci, c, b, llr, s, s_ref = setup(600 + F, n, rate, F, 0.85)
    T = 6
    g = np.random.default_rng(3)
    alpha = g.uniform(0.7, 1.1, size=(T, 2))
    beta = g.uniform(0.1, 0.7, size=(T, 2))
    loss, post, ga, gb = run(c, llr, s, b, alpha, beta, K=2, want_post=True)
    ref = oracle.woms(rp, ci, llr.astype(np.float64), s_ref, b, alpha.astype(np.float32).astype(np.float64),
                      beta.astype(np.float32).astype(np.float64), want_post=True)
    assert rel_ok(post, ref["post"]).all()
    assert abs(loss - ref["loss"]) <= TOL * abs(ref["loss"])
    scale = max(np.max(np.abs(ref["galpha"])), np.max(np.abs(ref["gbeta"])))
    assert np.all(np.abs(ga - ref["galpha"]) <= TOL * scale), (ga, ref["galpha"])
    assert np.all(np.abs(gb - ref["gbeta"]) <= TOL * scale), (gb, ref["gbeta"])
    if len(set(np.diff(rp).tolist())) == 1:
        assert np.all(ga[:, 1] == 0) and np.all(gb[:, 1] == 0)


def test_unit_weights_match_offset_min_sum_decoder():
    rp, ci, c, b, llr, s, s_ref = setup(640, 1024, 0.5, 8, 0.85)
    T = 5
    _, post, _, _ = run(c, llr, s, b, np.ones((T, 2)), np.full((T, 2), 0.5), K=5, want_post=True)
    ref = oracle.decode(rp, ci, llr.astype(np.float64), s_ref, "oms_flood", max_iter=T, early_stop=False, offset=0.5)
    assert rel_ok(post, ref["post"]).all()


def test_checkpoint_interval_does_not_change_gradient():
    rp, ci, c, b, llr, s, _ = setup(650, 1024, 0.5, 32, 0.85)
    T = 10
    g = np.random.default_rng(4)
    alpha, beta = g.uniform(0.7, 1.1, size=(T, 2)), g.uniform(0.1, 0.7, size=(T, 2))
    base = run(c, llr, s, b, alpha, beta, K=T)
    for K in (1, 3, 5):
        other = run(c, llr, s, b, alpha, beta, K=K)
        assert other[0] == base[0]
        assert np.allclose(other[2], base[2], rtol=1e-6, atol=1e-12)
        assert np.allclose(other[3], base[3], rtol=1e-6, atol=1e-12)


def test_gradient_vs_central_differences_of_gpu_loss():
    rp, ci, c, b, llr, s, _ = setup(660, 2048, 0.5, 64, 0.85)
    T = 6
    g = np.random.default_rng(5)
    alpha, beta = g.uniform(0.7, 1.1, size=(T, 2)), g.uniform(0.1, 0.7, size=(T, 2))
    _, _, ga, gb = run(c, llr, s, b, alpha, beta, K=3)
    scale = max(np.abs(ga).max(), np.abs(gb).max())
    checked = 0
    for name, P, G in (("alpha", alpha, ga), ("beta", beta, gb)):
        for t in range(T):
            fds = []
            for h in (1e-3, 2e-3):
                pp, pm = P.copy(), P.copy()
                pp[t, 0] += h
                pm[t, 0] -= h
                lp = run(c, llr, s, b, pp if name == "alpha" else alpha, pp if name == "beta" else beta, K=3)[0]
                lm = run(c, llr, s, b, pm if name == "alpha" else alpha, pm if name == "beta" else beta, K=3)[0]
                fds.append((lp - lm) / (2 * h))
            if abs(fds[0] - fds[1]) > 0.02 * scale:
                continue          # a kink inside the step
            checked += 1
            assert abs(G[t, 0] - fds[0]) <= 0.02 * scale, (name, t, G[t, 0], fds)
    assert checked >= T


def test_full_size_twenty_iterations_checkpoint_five():
    """1024 frames of n = 16384, rate 1/2 (dv 3, dc 6), 20 iterations, checkpoints
    every 5: against the oracle on two of those frames run alone, and against the
    uncheckpointed backward on all frames."""
    n, F, T = 16384, 1024, 20
    rp, ci, M = code(5000, n, 0.5)
    c = q.Code(n, rp, ci)
    x, y = synth.gaussian_pair(5, F * n, 3.0)
    lo, hi = oracle.quantiser_range(3.0)
    _, bits = q.qkdrec_quantise_slices(dev(y), 5, lo, hi)
    j = 4      # the slice whose capacity (0.545) is closest above 0.5/0.95
    target = bits[j].reshape(F, n).contiguous()
    llr = q.qkdrec_slice_llr(dev(x), 5, j, lo, hi, 3.0 ** -0.5, bits[:j]).reshape(F, n)
    s = q.qkdrec_syndrome(c, target)
    alpha = np.ones((T, 2))
    beta = np.full((T, 2), 0.5)
    ws = torch.empty(q.qkdrec_woms_workspace_size(c, F, T, 5), dtype=torch.uint8, device="cuda")
    a, bt = dev(alpha.astype(np.float32)), dev(beta.astype(np.float32))
    loss5, _ = q.qkdrec_woms_forward(c, llr, s, target, a, bt, 5, ws)
    ga5, gb5 = q.qkdrec_woms_backward(c, llr, s, target, a, bt, 5, ws)
    ws20 = torch.empty(q.qkdrec_woms_workspace_size(c, F, T, 20), dtype=torch.uint8, device="cuda")
    loss20, _ = q.qkdrec_woms_forward(c, llr, s, target, a, bt, 20, ws20)
    ga20, gb20 = q.qkdrec_woms_backward(c, llr, s, target, a, bt, 20, ws20)
    assert loss5.item() == loss20.item()
    assert torch.allclose(ga5, ga20, rtol=1e-5, atol=1e-9) and torch.allclose(gb5, gb20, rtol=1e-5, atol=1e-9)
    assert torch.isfinite(ga5).all() and torch.isfinite(gb5).all()
    # two frames through both implementations
    sel = [3, 700]
    tl = target[sel].contiguous()
    ll = llr[sel].contiguous()
    ss = s[sel].contiguous()
    loss2, _, g2a, g2b = run(c, ll.cpu().numpy(), ss, tl.cpu().numpy(), alpha, beta, K=5)
    ref = oracle.woms(rp, ci, ll.cpu().numpy().astype(np.float64), ss.cpu().numpy(), tl.cpu().numpy(),
                      alpha, beta)
    assert abs(loss2 - ref["loss"]) <= TOL * abs(ref["loss"])
    scale = max(np.abs(ref["galpha"]).max(), np.abs(ref["gbeta"]).max())
    assert np.all(np.abs(g2a - ref["galpha"]) <= TOL * scale)
    assert np.all(np.abs(g2b - ref["gbeta"]) <= TOL * scale)


def test_training_lowers_the_loss():
    from paper_2108_08418_b300.woms import woms_loss
    rp, ci, c, b, llr, s, _ = setup(670, 2048, 0.5, 128, 0.88)
    T = 8
    alpha = torch.ones((T, 2), device="cuda", requires_grad=True)
    beta = torch.full((T, 2), 0.5, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([alpha, beta], lr=0.03)
    ld, bd = dev(llr), dev(b)
    losses = []
    for _ in range(15):
        opt.zero_grad()
        loss = woms_loss(c, ld, s, bd, alpha, beta, 4)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert losses[-1] < losses[0]
