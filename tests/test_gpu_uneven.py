"""GPU: reverse reconciliation of an uneven batch (frames of several lengths and
SNRs, per-frame slice rates) as one CUDA graph.

* The graph's results (Bob's planes, Alice's reconciled planes, iteration
  counts, flags) equal those of the same reconciliation done frame group by
  frame group through the single-code entry points (quantiser, syndrome,
  slice LLR, batch decoder with layered offset min-sum).
* Graph replay with new inputs written in place equals an eager step, with
  the batch's frames in one to three parts decoded on their own streams.
* Against the FP64 oracle: for sampled frames the oracle reconciles the frame
  on its own (quantiser, syndromes, LLRs from its own lower slices, layered
  offset min-sum); both sides agree on every slice where both converge.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402
from paper_2108_08418_b300.uneven import UnevenBatch  # noqa: E402

M_SLICES = 5


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def frame_rates(snrs, fraction=0.75):
    """Rate of each (slice, frame): `fraction` x capacity on the 1/64 grid, at most
    60/64; below 0.10 the slice is disclosed (rate 0).  Codes well below capacity
    at these short lengths, so that most frames converge."""
    r = np.zeros((M_SLICES, len(snrs)))
    for f, s in enumerate(snrs):
        lo, hi = q.quantiser_range(s)
        for j in range(M_SLICES):
            k = int(np.floor(fraction * q.qkdrec_slice_capacity(s, M_SLICES, j, lo, hi) * 64 + 0.5))
            v = min(k, 60) / 64
            r[j, f] = v if v >= 0.10 else 0.0
    return r


def make_batch(seed, F, lengths=(1024, 2048, 4096), fraction=0.75):
    n, snr = synth.uneven_frames(seed, F, lengths, (2.0, 15.0))
    order = np.lexsort((snr, n))
    n, snr = n[order], snr[order]
    rates = frame_rates(snr, fraction)
    keys = {(int(n[f]), float(rates[j, f])) for j in range(M_SLICES) for f in range(F) if rates[j, f] > 0}
    csr, codes = {}, {}
    for i, (nn, r) in enumerate(sorted(keys)):
        rp, ci, _ = synth.make_regular_code(3000 + i, nn, synth.checks_for_rate(nn, r))
        csr[(nn, r)], codes[(nn, r)] = (rp, ci), q.Code(nn, rp, ci)
    x, y = synth.gaussian_frames(seed, n, snr)
    return n, snr, rates, codes, csr, x, y


def per_group_reference(ub, x, y):
    """The same reconciliation through the single-code entry points."""
    dev = ub.device
    off = ub.offsets
    bob = torch.zeros((M_SLICES, ub.count), dtype=torch.uint8, device=dev)
    alice = torch.zeros_like(bob)
    iters = torch.zeros((M_SLICES, ub.F), dtype=torch.int32, device=dev)
    conv = torch.ones((M_SLICES, ub.F), dtype=torch.uint8, device=dev)
    yd, xd = torch.from_numpy(y).to(dev), torch.from_numpy(x).to(dev)
    for f in range(ub.F):
        a, b = off[f], off[f + 1]
        lo, hi = q.quantiser_range(ub.snrs[f])
        _, bits = q.qkdrec_quantise_slices(yd[a:b], M_SLICES, lo, hi, want_idx=False)
        bob[:, a:b] = bits
    for j in range(M_SLICES):
        llr = torch.empty(ub.count, dtype=torch.float32, device=dev)
        for f in range(ub.F):
            a, b = off[f], off[f + 1]
            lo, hi = q.quantiser_range(ub.snrs[f])
            lower = alice[:j, a:b].contiguous() if j else None
            q.qkdrec_slice_llr(xd[a:b], M_SLICES, j, lo, hi, ub.snrs[f] ** -0.5, lower, out=llr[a:b])
        for g in ub.groups[j]:
            nf, n = g["f1"] - g["f0"], g["code"].n
            s = q.qkdrec_syndrome(g["code"], bob[j, g["a"]:g["b"]].view(nf, n))
            out = q.qkdrec_decode_batch(g["code"], llr[g["a"]:g["b"]].view(nf, n), s, ub.group_opts or ub.opts)
            alice[j, g["a"]:g["b"]] = out["bits"].view(-1)
            iters[j, g["f0"]:g["f1"]] = out["iters"]
            conv[j, g["f0"]:g["f1"]] = out["converged"]
        for a, b in ub.disclosed[j]:
            alice[j, a:b] = bob[j, a:b]
    return bob, alice, iters, conv


@pytest.mark.parametrize("parts", [1, 2, 3])
def test_uneven_graph_equals_per_group_calls_and_replays(parts):
    """The batch in 1-3 parts on their own streams (a frame's slices all in one
    part): graph replays, and the same step run in order on one stream, equal
    the per-group calls."""
    n, snr, rates, codes, csr, x, y = make_batch(41, 48)
    ub = UnevenBatch(n, snr, rates, codes, M_SLICES, max_iter=40, parts=parts)
    assert len(set(ub.part_of.tolist())) == parts
    assert sum(len(g) for g in ub.groups) > M_SLICES           # several groups per slice
    assert any(ub.disclosed[j] for j in range(M_SLICES))       # some disclosed slices
    ub.x.copy_(torch.from_numpy(x))
    ub.y.copy_(torch.from_numpy(y))
    ub.capture()
    ub.replay()
    torch.cuda.synchronize()
    bob, alice, iters, conv = per_group_reference(ub, x, y)
    assert torch.equal(ub.bob, bob)
    assert torch.equal(ub.alice, alice)
    assert torch.equal(ub.iters, iters)
    assert torch.equal(ub.conv, conv)
    ok = ub.frame_ok().cpu().numpy()
    assert ok.mean() > 0.5
    assert 0 < ub.reconciled_bits() <= ub.decoded_bits()
    # replay on a second batch written in place
    x2, y2 = synth.gaussian_frames(42, n, snr)
    ub.x.copy_(torch.from_numpy(x2))
    ub.y.copy_(torch.from_numpy(y2))
    ub.replay()
    torch.cuda.synchronize()
    bob2, alice2, iters2, conv2 = per_group_reference(ub, x2, y2)
    assert torch.equal(ub.alice, alice2) and torch.equal(ub.iters, iters2) and torch.equal(ub.conv, conv2)
    ub.alice.zero_()
    ub.step(overlap=False)
    torch.cuda.synchronize()
    assert torch.equal(ub.alice, alice2) and torch.equal(ub.iters, iters2) and torch.equal(ub.conv, conv2)
    ub.destroy()


def test_uneven_plain_decoder_graph_equals_per_group_calls():
    """The same batch with the plain FP32 sum-product batch decoder on every group
    instead of the plan: graph replay equals the per-group calls."""
    n, snr, rates, codes, csr, x, y = make_batch(44, 40)
    ub = UnevenBatch(n, snr, rates, codes, M_SLICES, device="cuda",
                     decoder=q.DecodeOpts(algo="sp_flood", prec="f32", max_iter=40, early_stop=True))
    assert ub.plans == [] and ub.autotune() == [(None, 0.0)] * M_SLICES
    ub.x.copy_(torch.from_numpy(x))
    ub.y.copy_(torch.from_numpy(y))
    ub.replay()
    torch.cuda.synchronize()
    bob, alice, iters, conv = per_group_reference(ub, x, y)
    assert torch.equal(ub.bob, bob)
    assert torch.equal(ub.alice, alice)
    assert torch.equal(ub.iters, iters)
    assert torch.equal(ub.conv, conv)
    assert ub.frame_ok().cpu().numpy().mean() > 0.5
    ub.destroy()


def test_uneven_frames_vs_oracle_reconciliation():
    n, snr, rates, codes, csr, x, y = make_batch(43, 18, lengths=(1024, 2048), fraction=0.6)
    ub = UnevenBatch(n, snr, rates, codes, M_SLICES, max_iter=30)
    ub.x.copy_(torch.from_numpy(x))
    ub.y.copy_(torch.from_numpy(y))
    ub.step()
    torch.cuda.synchronize()
    alice = ub.alice.cpu().numpy()
    conv = ub.conv.cpu().numpy()
    agreed = 0
    for f in range(0, ub.F, 3):
        a, b = ub.offsets[f], ub.offsets[f + 1]
        lo, hi = oracle.quantiser_range(snr[f])
        _, bits = oracle.quantise(y[a:b], M_SLICES, lo, hi)
        assert np.array_equal(ub.bob[:, a:b].cpu().numpy(), bits)
        mine = np.zeros_like(bits)
        for j in range(M_SLICES):
            if rates[j, f] <= 0:
                mine[j] = bits[j]
                continue
            if not np.array_equal(alice[:j, a:b], mine[:j]):
                break      # one side failed a lower slice: its later LLRs differ
            rp, ci = csr[(int(n[f]), float(rates[j, f]))]
            s = oracle.syndrome(rp, ci, bits[j][None])
            llr = oracle.slice_llr(x[a:b].astype(np.float64), mine[:j] if j else None, j, M_SLICES, lo, hi,
                                   snr[f] ** -0.5)
            out = oracle.decode(rp, ci, llr[None], s, "oms_layered", max_iter=30, offset=0.5)
            mine[j] = out["bits"][0]
            if out["converged"][0] and conv[j, f]:
                agreed += 1
                assert np.array_equal(alice[j, a:b], mine[j]), (f, j)
    assert agreed >= 3


def test_backoff_rates_accept_only_rates_whose_trials_pass():
    from paper_2108_08418_b300.uneven import backoff_rates
    T = 16
    points = [(1024, 3.0, 2), (1024, 3.0, 3), (2048, 12.0, 4), (1024, 2.0, 0)]
    start = {}
    for p in points:
        lo, hi = q.quantiser_range(p[1])
        start[p] = min(int(np.floor(0.95 * q.qkdrec_slice_capacity(p[1], M_SLICES, p[2], lo, hi) * 64 + 0.5)), 60) / 64
    cache, csr = {}, {}

    def codes_for(keys):
        for i, (n, r) in enumerate(sorted(keys)):
            if (n, r) not in cache:
                rp, ci, _ = synth.make_regular_code(7000 + int(r * 64), n, synth.checks_for_rate(n, r))
                csr[(n, r)] = (rp, ci)
                cache[(n, r)] = q.Code(n, rp, ci)
        return cache

    def sample(p):
        return synth.gaussian_pair(8000 + p[0] // 1024 + int(p[1]), T * p[0], p[1])

    got = backoff_rates(points, start, codes_for, sample, trial_frames=T, max_fail=1)
    for p in points:
        rate, fails = got[p]
        assert rate <= start[p]
        assert rate == 0.0 or (rate >= 0.10 and fails <= 1)
        if rate > 0:
            # the accepted code decodes the trial frames with at most one frame error
            n, snr, j = p
            x, y = sample(p)
            lo, hi = q.quantiser_range(snr)
            _, bits = q.qkdrec_quantise_slices(torch.from_numpy(y).cuda(), M_SLICES, lo, hi, want_idx=False)
            llr = q.qkdrec_slice_llr(torch.from_numpy(x).cuda(), M_SLICES, j, lo, hi, snr ** -0.5,
                                     bits[:j] if j else None)
            c = cache[(n, rate)]
            bob = bits[j].reshape(T, n).contiguous()
            out = q.qkdrec_decode_batch(c, llr.view(T, n), q.qkdrec_syndrome(c, bob),
                                        q.DecodeOpts(algo="oms_layered", max_iter=50))
            assert int((out["bits"] != bob).any(dim=1).sum()) == fails
    assert got[(1024, 2.0, 0)][0] == 0.0          # the LSB at SNR 2 carries almost nothing: disclosed
