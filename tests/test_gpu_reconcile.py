"""The whole-block reconciliation call (qkdrec_reconcile) through the C ABI.

It must equal the same reconciliation done step by step with the single-step
calls (quantiser, byte syndromes, slice LLRs, batch decoder) bit for bit, with
its packed syndromes and packed outputs, for host and device buffers alike,
with its partitions decoded one after another or concurrently (also inside a
captured graph); and its reconciled slices must agree with the FP64 oracle's
reconciliation of the same block where both decoders converge.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402

M = 4
SNR = 3.0


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2108_08418_b300 import build
    build.build()
    assert torch.cuda.is_available()


def block(count, seed=900):
    x, y = synth.gaussian_pair(seed, count, SNR)
    return x, y


def codes_for(n, rates, seed0):
    out, host = [], []
    for j, r in enumerate(rates):
        if r <= 0:
            out.append(None)
            host.append(None)
            continue
        rp, ci, _ = synth.make_regular_code(seed0 + j, n, synth.checks_for_rate(n, r))
        out.append(q.Code(n, rp, ci))
        host.append((rp, ci))
    return out, host


def stepwise(x, y, n, codes, opts, lo, hi, sn):
    """The same reconciliation with the single-step calls (byte syndromes)."""
    count = x.numel()
    F = count // n
    _, bob = q.qkdrec_quantise_slices(y, M, lo, hi, want_idx=False)
    alice = torch.empty((M, count), dtype=torch.uint8, device="cuda")
    conv = torch.empty((M, F), dtype=torch.uint8, device="cuda")
    its = torch.empty((M, F), dtype=torch.int32, device="cuda")
    for j, c in enumerate(codes):
        if c is None:
            alice[j].copy_(bob[j])
            conv[j].fill_(1)
            its[j].zero_()
            continue
        s = q.qkdrec_syndrome(c, bob[j].view(F, n))
        llr = q.qkdrec_slice_llr(x, M, j, lo, hi, sn, alice[:j] if j else None)
        q.qkdrec_decode_batch(c, llr.view(F, n), s, opts,
                              out=dict(bits=alice[j].view(F, n), iters=its[j], converged=conv[j], post=None))
    return bob, alice, conv, its


def packbits(a):
    return np.packbits(a.astype(np.uint8), axis=-1, bitorder="little")


@pytest.mark.parametrize("opts", [q.DecodeOpts(algo="sp_flood", max_iter=30),
                                  q.DecodeOpts(algo="oms_flood", prec="i8", max_iter=30, fallback_f32="sp"),
                                  q.DecodeOpts(algo="oms_layered", prec="f16", max_iter=20, fallback_f32=True)])
def test_reconcile_equals_the_stepwise_calls(opts):
    count = 1 << 16
    xh, yh = block(count)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    lo, hi = q.qkdrec_quantiser_range(SNR)
    sn = SNR ** -0.5
    # two partitions of the block; the second's 16 frames fill half a 32-frame word
    parts = [(1024, [0.0, 0.0, 0.75, 0.5]), (4096, [0.0, 0.125, 0.75, 0.5])]
    pts, refs = [], []
    for i, (n, rates) in enumerate(parts):
        codes, _ = codes_for(n, rates, 1000 * (i + 1))
        F = count // n
        pts.append(dict(n=n, codes=codes, alice_packed=torch.zeros((M, count // 8), dtype=torch.uint8, device="cuda"),
                        converged=torch.zeros((M, F), dtype=torch.uint8, device="cuda"),
                        iters=torch.zeros((M, F), dtype=torch.int32, device="cuda")))
        refs.append(stepwise(x, y, n, codes, opts, lo, hi, sn))
    bobp = torch.zeros((M, count // 8), dtype=torch.uint8, device="cuda")
    q.qkdrec_reconcile(x, y, M, lo, hi, sn, opts, pts, bob_packed=bobp)
    torch.cuda.synchronize()
    for p, (bob, alice, conv, its) in zip(pts, refs):
        assert np.array_equal(bobp.cpu().numpy(), packbits(bob.cpu().numpy()))
        assert np.array_equal(p["alice_packed"].cpu().numpy(), packbits(alice.cpu().numpy()))
        assert torch.equal(p["converged"], conv) and torch.equal(p["iters"], its)


def test_reconcile_with_host_buffers_equals_device_buffers():
    count = 48 * 256                      # 48 frames of 256: one and a half 32-frame words
    xh, yh = block(count, seed=901)
    lo, hi = q.qkdrec_quantiser_range(SNR)
    n = 256
    codes, _ = codes_for(n, [0.0, 0.25, 0.75, 0.5], 3000)
    opts = q.DecodeOpts(algo="sp_flood", max_iter=25)
    F = count // n

    def outs(device, pin):
        mk = (lambda shape, dt: torch.zeros(shape, dtype=dt, device="cuda")) if device else \
            (lambda shape, dt: torch.zeros(shape, dtype=dt).pin_memory() if pin else torch.zeros(shape, dtype=dt))
        return dict(n=n, codes=codes, alice_packed=mk((M, count // 8), torch.uint8),
                    converged=mk((M, F), torch.uint8), iters=mk((M, F), torch.int32))

    res = []
    for device, pin in ((True, False), (False, True), (False, False)):
        p = outs(device, pin)
        if device:
            x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
        else:
            x, y = torch.from_numpy(xh), torch.from_numpy(yh)
            if pin:
                x, y = x.pin_memory(), y.pin_memory()
        ws = q.qkdrec_reconcile(x, y, M, lo, hi, SNR ** -0.5, opts, [p])
        torch.cuda.synchronize()
        res.append({k: p[k].cpu() for k in ("alice_packed", "converged", "iters")})
        del ws
    for r in res[1:]:
        for k in r:
            assert torch.equal(r[k], res[0][k]), k


def test_reconcile_partitions_in_flight_give_identical_results():
    """Three partitions decoded one after another, two at a time (a side stream
    takes the third after the first) and all at once, and the concurrent form
    captured in a CUDA graph and replayed: the same outputs bit for bit."""
    count = 1 << 15
    xh, yh = block(count, seed=905)
    x, y = torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda()
    lo, hi = q.qkdrec_quantiser_range(SNR)
    opts = q.DecodeOpts(algo="sp_flood", max_iter=30)
    parts = [(512, [0.0, 0.125, 0.75, 0.5]), (1024, [0.0, 0.0, 0.75, 0.5]), (2048, [0.0, 0.125, 0.75, 0.5])]
    codes = [codes_for(n, rates, 4000 + 100 * i)[0] for i, (n, rates) in enumerate(parts)]

    def points(host_last=False):
        out = []
        for i, (n, _) in enumerate(parts):
            F = count // n
            host = host_last and i == len(parts) - 1
            mk = (lambda shape, dt: torch.zeros(shape, dtype=dt).pin_memory()) if host else \
                (lambda shape, dt: torch.zeros(shape, dtype=dt, device="cuda"))
            out.append(dict(n=n, codes=codes[i], alice_packed=mk((M, count // 8), torch.uint8),
                            converged=mk((M, F), torch.uint8), iters=mk((M, F), torch.int32)))
        return out

    def grab(pts):
        return [{k: p[k].cpu().clone() for k in ("alice_packed", "converged", "iters")} for p in pts]

    res = []
    for k in (1, 2, 3):
        pts = points(host_last=(k == 2))
        ws = torch.empty(q.qkdrec_reconcile_workspace_size_limited(count, M, opts, pts, k), dtype=torch.uint8,
                         device="cuda")
        q.qkdrec_reconcile(x, y, M, lo, hi, SNR ** -0.5, opts, pts, workspace=ws)
        torch.cuda.synchronize()
        res.append(grab(pts))
    assert q.qkdrec_reconcile_workspace_size(count, M, opts, points()) == ws.numel()
    # the concurrent form inside a captured graph, replayed on a fresh output set
    pts = points()
    ws = torch.empty(q.qkdrec_reconcile_workspace_size(count, M, opts, pts), dtype=torch.uint8, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, capture_error_mode="relaxed"):
        q.qkdrec_reconcile(x, y, M, lo, hi, SNR ** -0.5, opts, pts, workspace=ws)
    for p in pts:
        for key in ("alice_packed", "converged", "iters"):
            p[key].zero_()
    g.replay()
    torch.cuda.synchronize()
    res.append(grab(pts))
    for r in res[1:]:
        for a, b in zip(r, res[0]):
            for key in a:
                assert torch.equal(a[key], b[key]), key


def test_reconcile_agrees_with_the_oracle():
    """Alice's reconciled slices against the FP64 oracle's reconciliation of the
    same block (its own quantiser, syndromes, LLRs from its own reconciled lower
    slices, sum-product decodes): identical sub-blocks wherever both decoders
    converge, and frame-error counts inside each other's Wilson intervals."""
    from _workloads import wilson
    count, n = 1 << 15, 1024
    xh, yh = block(count, seed=902)
    lo, hi = q.qkdrec_quantiser_range(SNR)
    sn = SNR ** -0.5
    rates = [0.0, 0.25, 0.6875, 0.375]       # 58 %, 78 %, 70 % of the slices' capacities
    codes, host = codes_for(n, rates, 4000)
    F = count // n
    opts = q.DecodeOpts(algo="sp_flood", max_iter=50)
    p = dict(n=n, codes=codes, alice_packed=torch.zeros((M, count // 8), dtype=torch.uint8, device="cuda"),
             converged=torch.zeros((M, F), dtype=torch.uint8, device="cuda"))
    q.qkdrec_reconcile(torch.from_numpy(xh).cuda(), torch.from_numpy(yh).cuda(), M, lo, hi, sn, opts, [p])
    got = np.unpackbits(p["alice_packed"].cpu().numpy(), axis=-1, bitorder="little")
    gconv = p["converged"].cpu().numpy().astype(bool)
    _, bob = oracle.quantise(yh, M, lo, hi)
    alice = np.zeros_like(bob)
    for j in range(M):
        if host[j] is None:
            alice[j] = bob[j]
            continue
        rp, ci = host[j]
        s = oracle.syndrome(rp, ci, bob[j].reshape(F, n))
        llr = oracle.slice_llr(xh, alice[:j] if j else None, j, M, lo, hi, sn)
        o = oracle.decode(rp, ci, llr.reshape(F, n), s, "sp_flood", max_iter=50)
        alice[j] = o["bits"].reshape(-1)
        both = gconv[j] & o["converged"].astype(bool)
        assert both.sum() > F // 2
        assert np.array_equal(got[j].reshape(F, n)[both], o["bits"][both])
        e_g = int(np.sum(np.any(got[j].reshape(F, n) != bob[j].reshape(F, n), axis=1)))
        e_o = int(np.sum(np.any(o["bits"] != bob[j].reshape(F, n), axis=1)))
        lo_, hi_ = wilson(e_o, F)
        assert lo_ <= e_g / F <= hi_, (j, e_g, e_o)


def test_pack_and_unpack_bits():
    g = np.random.default_rng(3)
    for count in (32, 4096, 32 * 1001):
        b = g.integers(0, 2, size=count).astype(np.uint8)
        d = torch.from_numpy(b).cuda()
        pk = q.qkdrec_pack_bits(d)
        assert np.array_equal(pk.cpu().numpy(), packbits(b))
        assert torch.equal(q.qkdrec_unpack_bits(pk, count), d)


def test_reconcile_rejects_bad_partitions_before_any_work():
    count = 4096
    x = torch.zeros(count, device="cuda")
    codes, _ = codes_for(512, [0.0, 0.0, 0.5, 0.5], 5000)
    opts = q.DecodeOpts()
    bad = [dict(n=1000, codes=codes, alice_packed=torch.zeros((M, count // 8), dtype=torch.uint8, device="cuda")),
           dict(n=1024, codes=codes, alice_packed=torch.zeros((M, count // 8), dtype=torch.uint8, device="cuda"))]
    for p in bad:
        with pytest.raises(q.QkdrecError) as e:
            q.qkdrec_reconcile(x, x, M, -1.0, 1.0, 0.5, opts, [p], workspace=torch.zeros(256, dtype=torch.uint8,
                                                                                           device="cuda"))
        assert e.value.status == q.ERR_ARG
