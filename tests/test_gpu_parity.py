"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer and index work must be bit-exact (quantiser, syndromes, layer
partition, integer min-sum); floating point within TOL = 1e-4 relative
(|gpu - oracle| <= 1e-4 max(|oracle|, 1)): FP32 arithmetic keeps ~1e-7 per
operation, and the tolerance leaves two orders of magnitude for the
accumulation through a few BP iterations.  Full decodes are compared per frame
where both sides converge (identical words) and by FER within each other's
Wilson 95% interval.
"""
import numpy as np
import pytest

import oracle
import synth
from _workloads import TOL, bpsk_frames, code, rel_ok, wilson

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


def host(t):
    return t.cpu().numpy()


# ------------------------------------------------------------------ quantiser
@pytest.mark.parametrize("m,label", [(4, "gray"), (5, "gray"), (5, "binary"), (8, "gray"), (1, "gray")])
def test_quantiser_bit_exact(m, label):
    snr = 3.0
    lo, hi = oracle.quantiser_range(snr)
    _, y = synth.gaussian_pair(21, 100_003, snr)
    t = oracle.thresholds(m, lo, hi).astype(np.float32)
    # thresholds themselves and their float neighbours, plus extremes
    edge = np.concatenate([t, np.nextafter(t, -np.inf), np.nextafter(t, np.inf),
                           np.array([-np.inf, np.inf, 0.0, -0.0, 1e30, -1e30], np.float32)]).astype(np.float32)
    y = np.concatenate([y, edge]).astype(np.float32)
    idx, bits = q.qkdrec_quantise_slices(dev(y), m, lo, hi, label)
    ridx, rbits = oracle.quantise(y, m, lo, hi, label)
    assert np.array_equal(host(idx), ridx)
    assert np.array_equal(host(bits), rbits)


def test_quantiser_empty_and_ragged():
    for count in (0, 1, 7, 4097):
        y = synth.gaussian_pair(5, count, 3.0)[1] if count else np.zeros(0, np.float32)
        if count == 0:
            idx, bits = q.qkdrec_quantise_slices(torch.zeros(0, device="cuda"), 4, -2.0, 2.0)
            assert idx.numel() == 0
            continue
        idx, bits = q.qkdrec_quantise_slices(dev(y), 4, -2.0, 2.0)
        ridx, rbits = oracle.quantise(y, 4, -2.0, 2.0)
        assert np.array_equal(host(idx), ridx) and np.array_equal(host(bits), rbits)


# ------------------------------------------------------------------ slice LLR
@pytest.mark.parametrize("snr,m,label", [(3.0, 4, "gray"), (15.0, 5, "gray"), (3.0, 5, "binary"),
                                         (2.0, 6, "gray"), (30.0, 8, "gray"), (8.0, 7, "binary")])
def test_slice_llr_vs_oracle(snr, m, label):
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    x, y = synth.gaussian_pair(31, 60_001, snr)
    _, bits = oracle.quantise(y, m, lo, hi, label)
    g = synth.philox(32)
    for j in range(m):
        for lower in ("bob", "random"):
            if j == 0 and lower == "random":
                continue
            lb = bits[:j] if lower == "bob" else g.integers(0, 2, size=(j, x.size)).astype(np.uint8)
            got = host(q.qkdrec_slice_llr(dev(x), m, j, lo, hi, sn, dev(lb) if j else None, label))
            ref = oracle.slice_llr(x, lb if j else None, j, m, lo, hi, sn, label)
            ok = rel_ok(got, ref)
            assert ok.all(), (j, lower, np.flatnonzero(~ok)[:5], got[~ok][:5], ref[~ok][:5])


def test_slice_llr_extreme_inputs():
    # far tails on both sides, exact thresholds, and candidate sets far from x
    snr, m = 15.0, 5
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    x = np.concatenate([np.linspace(-9, 9, 4001), oracle.thresholds(m, lo, hi)]).astype(np.float32)
    g = synth.philox(33)
    for j in range(m):
        lb = g.integers(0, 2, size=(j, x.size)).astype(np.uint8)
        got = host(q.qkdrec_slice_llr(dev(x), m, j, lo, hi, sn, dev(lb) if j else None))
        ref = oracle.slice_llr(x, lb if j else None, j, m, lo, hi, sn)
        assert rel_ok(got, ref).all(), j
        assert np.all(np.isfinite(got)) and np.all(np.abs(got) <= 30.0)


# ------------------------------------------------------------------ syndrome / layers
@pytest.mark.parametrize("n,rate,F", [(4096, 0.5, 16), (4096, 57 / 64, 3), (1024, 1 / 16, 33)])
def test_syndrome_bit_exact(n, rate, F):
    rp, ci, M = code(40 + F, n, rate)
    c = q.Code(n, rp, ci)
    b = synth.philox(41).integers(0, 2, size=(F, n)).astype(np.uint8)
    got = host(q.qkdrec_syndrome(c, dev(b)))
    assert np.array_equal(got, oracle.syndrome(rp, ci, b))


def test_layer_partition_identical():
    for n, rate in ((2048, 0.5), (4096, 57 / 64), (1024, 1 / 16)):
        rp, ci, M = code(50, n, rate)
        c = q.Code(n, rp, ci)
        layer_of, lptr, _ = oracle.greedy_layers(rp, ci, n)
        assert np.array_equal(c.layers(), layer_of)
        assert c.n_layers == len(lptr) - 1


# ------------------------------------------------------------------ decoders
FLOAT_ALGOS = ["sp_flood", "oms_flood", "oms_layered"]


def run_both(algo, prec, rp, ci, n, b, llr, max_iter, early_stop):
    c = q.Code(n, rp, ci)
    s_gpu = q.qkdrec_syndrome(c, dev(b))
    s_ref = oracle.syndrome(rp, ci, b)
    assert np.array_equal(host(s_gpu), s_ref)
    opts = q.DecodeOpts(algo=algo, prec=prec, max_iter=max_iter, early_stop=early_stop)
    out = q.qkdrec_decode_batch(c, dev(llr), s_gpu, opts, want_post=True)
    got = {k: host(v) for k, v in out.items()}
    oalgo = ("i" + algo) if prec == "i8" else algo
    ref = oracle.decode(rp, ci, llr.astype(np.float64), s_ref, oalgo, max_iter=max_iter,
                        early_stop=early_stop, offset=0.5, llr_step=0.5)
    return got, ref


@pytest.mark.parametrize("algo", FLOAT_ALGOS)
@pytest.mark.parametrize("iters", [0, 1, 2, 4])
def test_float_posteriors_after_fixed_iterations(algo, iters):
    n, F = 1024, 13                       # ragged: 13 frames -> 4 frame vectors, last one partial
    rp, ci, _ = code(60, n, 0.5)
    b, llr = bpsk_frames(61, F, n, 0.85)
    got, ref = run_both(algo, "f32", rp, ci, n, b, llr, iters, early_stop=False)
    ok = rel_ok(got["post"], ref["post"])
    assert ok.all(), (np.argwhere(~ok)[:5], got["post"][~ok][:5], ref["post"][~ok][:5])
    sure = np.abs(ref["post"]) > 1e-3
    assert np.array_equal(got["bits"][sure], ref["bits"][sure])
    assert np.array_equal(got["iters"], ref["iters"])
    assert np.array_equal(got["converged"], ref["converged"])


@pytest.mark.parametrize("algo", FLOAT_ALGOS)
@pytest.mark.parametrize("sigma", [0.8, 0.9])
def test_float_full_decode_matches_oracle(algo, sigma):
    n, F = 2048, 64
    rp, ci, _ = code(70, n, 0.5)
    b, llr = bpsk_frames(71, F, n, sigma)
    got, ref = run_both(algo, "f32", rp, ci, n, b, llr, 50, early_stop=True)
    both = (got["converged"] == 1) & (ref["converged"] == 1)
    assert np.array_equal(got["bits"][both], ref["bits"][both])
    # a converged output satisfies its syndrome
    s_ref = oracle.syndrome(rp, ci, b)
    for f in np.flatnonzero(got["converged"]):
        assert np.array_equal(oracle.syndrome(rp, ci, got["bits"][f:f + 1])[0], s_ref[f])
    ferr_g = int(np.sum(np.any(got["bits"] != b, axis=1)))
    ferr_r = int(np.sum(np.any(ref["bits"] != b, axis=1)))
    lo_g, hi_g = wilson(ferr_g, F)
    lo_r, hi_r = wilson(ferr_r, F)
    assert lo_g <= ferr_r / F <= hi_g and lo_r <= ferr_g / F <= hi_r
    # iteration counts agree on frames that converge in both (FP32 may shift one by a step)
    d = np.abs(got["iters"][both] - ref["iters"][both])
    assert np.mean(d == 0) > 0.9


@pytest.mark.parametrize("algo", ["oms_flood", "oms_layered"])
@pytest.mark.parametrize("early_stop", [False, True])
def test_integer_min_sum_bit_exact(algo, early_stop):
    n, F = 2048, 37
    rp, ci, _ = code(80, n, 0.5)
    b, llr = bpsk_frames(81, F, n, 0.8)
    got, ref = run_both(algo, "i8", rp, ci, n, b, llr, 30, early_stop)
    for k in ("bits", "iters", "converged", "post"):
        assert np.array_equal(got[k], ref[k]), k


@pytest.mark.parametrize("algo", FLOAT_ALGOS)
def test_high_rate_and_low_rate_codes(algo):
    for rate, sigma, seed in ((57 / 64, 0.45, 90), (1 / 16, 1.6, 92)):
        n, F = 4096, 8
        rp, ci, _ = code(seed, n, rate)
        b, llr = bpsk_frames(seed + 1, F, n, sigma)
        got, ref = run_both(algo, "f32", rp, ci, n, b, llr, 3, early_stop=False)
        assert rel_ok(got["post"], ref["post"]).all(), rate


def test_single_frame_and_tiny_code():
    n = 64
    rp, ci, _ = code(100, n, 0.5)
    for F in (1, 2, 5):
        b, llr = bpsk_frames(101 + F, F, n, 0.7)
        got, ref = run_both("sp_flood", "f32", rp, ci, n, b, llr, 3, early_stop=False)
        assert rel_ok(got["post"], ref["post"]).all()


def test_zero_frames_is_a_no_op():
    rp, ci, M = code(110, 256, 0.5)
    c = q.Code(256, rp, ci)
    out = q.qkdrec_decode_batch(c, torch.zeros((0, 256), device="cuda"),
                                torch.zeros((0, M), dtype=torch.uint8, device="cuda"))
    assert out["bits"].shape == (0, 256)


def test_consistent_channel_stops_at_zero():
    n, F = 1024, 9
    rp, ci, _ = code(120, n, 0.5)
    b, _ = bpsk_frames(121, F, n, 0.5)
    llr = (8.0 * (1.0 - 2.0 * b)).astype(np.float32)
    for algo in FLOAT_ALGOS:
        got, _ = run_both(algo, "f32", rp, ci, n, b, llr, 20, early_stop=True)
        assert np.all(got["iters"] == 0) and np.all(got["converged"] == 1)
        assert np.array_equal(got["bits"], b)


@pytest.mark.parametrize("algo", FLOAT_ALGOS)
def test_f16_messages_fer_matches_f32(algo):
    n, F = 2048, 96
    rp, ci, _ = code(130, n, 0.5)
    b, llr = bpsk_frames(131, F, n, 0.82)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    res = {}
    for prec in ("f32", "f16"):
        o = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec=prec, max_iter=50))
        res[prec] = int(np.sum(np.any(host(o["bits"]) != b, axis=1)))
    lo, hi = wilson(res["f32"], F)
    assert lo <= res["f16"] / F <= hi + 0.05


@pytest.mark.parametrize("early_stop", [False, True])
def test_f16_message_posteriors_track_f32(early_stop):
    """FP16 message storage changes each message by at most 2^-11 of itself, and
    offset min-sum passes such changes on without growth: after two flooding
    iterations the FP16-message posteriors stay within 1e-2 (relative) of the
    FP32 ones and make the same hard decisions wherever |L| > 0.1 (a frame or
    variable mixed up anywhere would be off by O(1))."""
    n, F = 1024, 200                      # two 128-frame blocks, the second partial
    rp, ci, _ = code(170, n, 0.5)
    b, llr = bpsk_frames(171, F, n, 0.8)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    out = {p: q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="oms_flood", prec=p, max_iter=2,
                                                                   early_stop=early_stop), want_post=True)
           for p in ("f16", "f32")}
    p16, p32 = host(out["f16"]["post"]), host(out["f32"]["post"])
    same = host(out["f16"]["iters"]) == host(out["f32"]["iters"])
    assert same.sum() > F // 2
    assert np.all(np.abs(p16[same] - p32[same]) <= 1e-2 * np.maximum(np.abs(p32[same]), 1.0))
    sure = same[:, None] & (np.abs(p32) > 0.1)
    assert np.array_equal(host(out["f16"]["bits"])[sure], host(out["f32"]["bits"])[sure])


@pytest.mark.parametrize("prec", ["i8", "f16"])
def test_fp32_redecode_of_failed_frames(prec):
    n, F = 2048, 64
    rp, ci, _ = code(140, n, 0.5)
    b, llr = bpsk_frames(141, F, n, 0.86)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    lowp = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="oms_flood", prec=prec, max_iter=30))
    f32 = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="oms_flood", prec="f32", max_iter=30))
    fb = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="oms_flood", prec=prec, max_iter=30,
                                                            fallback_f32=True))
    lc, fc = host(lowp["converged"]).astype(bool), host(fb["converged"]).astype(bool)
    # frames the low-precision pass solved are untouched; the others equal a plain FP32 decode
    assert np.array_equal(host(fb["bits"])[lc], host(lowp["bits"])[lc])
    assert np.array_equal(host(fb["iters"])[lc], host(lowp["iters"])[lc])
    redo = ~lc
    assert np.array_equal(host(fb["bits"])[redo], host(f32["bits"])[redo])
    assert np.array_equal(host(fb["converged"])[redo], host(f32["converged"])[redo])
    assert np.array_equal(host(fb["iters"])[redo], host(lowp["iters"])[redo] + host(f32["iters"])[redo])
    assert fc.sum() >= lc.sum()


@pytest.mark.parametrize("algo,prec", [("oms_flood", "f16"), ("oms_flood", "i8"), ("oms_layered", "i8")])
def test_sum_product_redecode_of_failed_frames(algo, prec):
    """Fallback 2: frames the low-precision min-sum pass leaves unsatisfied are
    decoded again by the plain form (FP32 sum-product flooding)."""
    n, F = 2048, 64
    rp, ci, _ = code(150, n, 0.5)
    b, llr = bpsk_frames(151, F, n, 0.88)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    lowp = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec=prec, max_iter=30))
    sp = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="sp_flood", prec="f32", max_iter=30))
    fb = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec=prec, max_iter=30, fallback_f32="sp"))
    lc = host(lowp["converged"]).astype(bool)
    assert (~lc).any() and lc.any()
    assert np.array_equal(host(fb["bits"])[lc], host(lowp["bits"])[lc])
    redo = ~lc
    assert np.array_equal(host(fb["bits"])[redo], host(sp["bits"])[redo])
    assert np.array_equal(host(fb["converged"])[redo], host(sp["converged"])[redo])
    assert np.array_equal(host(fb["iters"])[redo], host(lowp["iters"])[redo] + host(sp["iters"])[redo])
    # the combined form fails no frame the plain form decodes
    assert not np.any(host(sp["converged"]).astype(bool) & ~host(fb["converged"]).astype(bool))


@pytest.mark.parametrize("algo,prec,fallback", [("oms_flood", "i8", "sp"), ("oms_flood", "f16", True),
                                                ("oms_layered", "i8", True)])
def test_redecode_compaction_many_failures_across_blocks(algo, prec, fallback):
    """The re-decode packs the failed frames to the front; with failures spread
    over many frame blocks and a ragged frame count, every re-decoded frame
    (bits, flags, iterations, posteriors) equals a plain FP32 decode of it, and
    every other frame keeps the first pass's outputs."""
    n, F = 1024, 301
    rp, ci, _ = code(160, n, 0.5)
    # half the frames easy, half hard, mixed at random over the frame blocks
    b1, llr1 = bpsk_frames(161, F, n, 0.7)
    b2, llr2 = bpsk_frames(162, F, n, 1.0)
    hard = synth.philox(163).random(F) < 0.5
    b = np.where(hard[:, None], b2, b1)
    llr = np.where(hard[:, None], llr2, llr1)
    c = q.Code(n, rp, ci)
    s = q.qkdrec_syndrome(c, dev(b))
    lowp = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec=prec, max_iter=12), want_post=True)
    o2 = "sp_flood" if fallback == "sp" else algo
    ref = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=o2, prec="f32", max_iter=12), want_post=True)
    fb = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo=algo, prec=prec, max_iter=12, fallback_f32=fallback),
                               want_post=True)
    lc = host(lowp["converged"]).astype(bool)
    redo = ~lc
    blocks = np.unique(np.flatnonzero(redo) // 32)
    assert redo.sum() > 40 and blocks.size > 4 and lc.any()
    for k in ("bits", "post", "iters", "converged"):
        assert np.array_equal(host(fb[k])[lc], host(lowp[k])[lc]), k
    assert np.array_equal(host(fb["bits"])[redo], host(ref["bits"])[redo])
    assert np.array_equal(host(fb["post"])[redo], host(ref["post"])[redo])
    assert np.array_equal(host(fb["converged"])[redo], host(ref["converged"])[redo])
    assert np.array_equal(host(fb["iters"])[redo], host(lowp["iters"])[redo] + host(ref["iters"])[redo])


@pytest.mark.parametrize("algo,prec", [("sp_flood", "f32"), ("oms_flood", "i8"), ("oms_layered", "f32")])
def test_corrupted_syndromes_are_detected(algo, prec):
    """Failure detection without a device fault: one syndrome bit flipped on the
    host in half the frames (a message corrupted in transit).  The decode ends
    with every frame accounted for: intact frames decode Bob's word; a corrupted
    frame either reports no convergence after all its iterations (its word may
    still be Bob's: the flag carries the failure), or converges to a word that
    satisfies the corrupted syndrome, which cannot be Bob's -- so the flag and
    the comparison with Bob's bits (the protocol's check) together flag every
    corrupted frame."""
    n, F, T = 1024, 64, 30
    rp, ci, M = code(180, n, 0.5)
    b, llr = bpsk_frames(181, F, n, 0.6)
    synd = oracle.syndrome(rp, ci, b)
    g = synth.philox(182)
    bad = g.random(F) < 0.5
    flip = g.integers(0, M, size=F)
    s2 = synd.copy()
    s2[bad, flip[bad]] ^= 1
    c = q.Code(n, rp, ci)
    out = q.qkdrec_decode_batch(c, dev(llr), dev(s2), q.DecodeOpts(algo=algo, prec=prec, max_iter=T))
    bits, conv, iters = host(out["bits"]), host(out["converged"]).astype(bool), host(out["iters"])
    good = ~bad
    assert bad.sum() > 10 and good.sum() > 10
    assert np.array_equal(bits[good], b[good]) and conv[good].all()
    wrong = (bits != b).any(axis=1)
    assert np.all(~conv[bad] | wrong[bad])
    assert not np.any(conv[bad] & ~wrong[bad])
    assert np.all(iters[bad & ~conv] == T)
    got = oracle.syndrome(rp, ci, bits)
    assert np.array_equal(got[conv], s2[conv])


# ------------------------------------------------------------------ full pipeline
def test_config1_pipeline_vs_oracle():
    """x, y at SNR 3, 16 frames x 4096, 4 Gray slices, codes at 0.95 x capacity, SP flooding,
    50 iterations: every stage of the GPU pipeline against the oracle's own pipeline."""
    snr, m, n, F = 3.0, 4, 4096, 16
    lo, hi = oracle.quantiser_range(snr)
    sn = snr ** -0.5
    x, y = synth.gaussian_pair(1, F * n, snr)
    idx_g, bits_g = q.qkdrec_quantise_slices(dev(y), m, lo, hi)
    _, bits_r = oracle.quantise(y, m, lo, hi)
    assert np.array_equal(host(bits_g), bits_r)
    dec_g = torch.zeros((m, F * n), dtype=torch.uint8, device="cuda")
    dec_r = np.zeros((m, F * n), dtype=np.uint8)
    for j in range(m):
        r = oracle.code_rate(oracle.slice_capacity(snr, m, j))
        if r <= 0:
            dec_g[j] = bits_g[j]
            dec_r[j] = bits_r[j]
            continue
        rp, ci, M = code(1000 + j, n, r)
        c = q.Code(n, rp, ci)
        llr_g = q.qkdrec_slice_llr(dev(x), m, j, lo, hi, sn, dec_g[:j] if j else None)
        llr_r = oracle.slice_llr(x, dec_r[:j] if j else None, j, m, lo, hi, sn)
        s_g = q.qkdrec_syndrome(c, bits_g[j].reshape(F, n).contiguous())
        s_r = oracle.syndrome(rp, ci, bits_r[j].reshape(F, n))
        assert np.array_equal(host(s_g), s_r)
        out = q.qkdrec_decode_batch(c, llr_g.reshape(F, n), s_g, q.DecodeOpts(max_iter=50))
        ref = oracle.decode(rp, ci, llr_r.reshape(F, n), s_r, "sp_flood", max_iter=50)
        both = (host(out["converged"]) == 1) & (ref["converged"] == 1)
        assert np.array_equal(host(out["bits"])[both], ref["bits"][both])
        fe_g = int(np.sum(np.any(host(out["bits"]) != bits_r[j].reshape(F, n), axis=1)))
        fe_r = int(np.sum(np.any(ref["bits"] != bits_r[j].reshape(F, n), axis=1)))
        lo_g, hi_g = wilson(fe_g, F)
        assert lo_g <= fe_r / F <= hi_g, (j, fe_g, fe_r)
        dec_g[j] = out["bits"].reshape(-1)
        dec_r[j] = ref["bits"].reshape(-1)


# ------------------------------------------------------------------ full size, sampled
def test_full_size_sampled_frames():
    """n = 2^16 sub-blocks of a 2^27-sample block (F = 2048), the sizes and launch
    configuration of the block-size sweep: two sampled frames after two SP
    iterations against the oracle, and the syndrome invariant on every frame
    of a full early-stopped decode."""
    n, F = 1 << 16, 2048
    rp, ci, M = code(2000 + 100 * 16 + 3, n, 0.84375)
    c = q.Code(n, rp, ci)
    b, llr = bpsk_frames(2001, F, n, 0.52)
    s = q.qkdrec_syndrome(c, dev(b))
    out = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(max_iter=2, early_stop=False), want_post=True)
    post = out["post"]
    s_ref = oracle.syndrome(rp, ci, b[[7, 1999]])
    assert np.array_equal(host(s[[7, 1999]]), s_ref)
    ref = oracle.decode(rp, ci, llr[[7, 1999]].astype(np.float64), s_ref, "sp_flood", max_iter=2,
                        early_stop=False)
    assert rel_ok(host(post[[7, 1999]]), ref["post"]).all()
    full = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(max_iter=100))
    conv = host(full["converged"]).astype(bool)
    synd_out = host(q.qkdrec_syndrome(c, full["bits"]))
    assert np.array_equal(synd_out[conv], host(s)[conv])
    assert np.all(np.any(synd_out[~conv] != host(s)[~conv], axis=1))


@pytest.mark.parametrize("logn,F", [(20, 128), (12, 32768)])
def test_sweep_extreme_sizes_sampled_frames(logn, F):
    """The largest and the smallest sub-blocks of the sweep in its launch
    configuration (2^27 samples per slice): sampled frames after two SP
    iterations against the oracle."""
    n = 1 << logn
    rp, ci, M = code(2000 + 100 * logn + 2, n, 0.5)
    c = q.Code(n, rp, ci)
    b, llr = bpsk_frames(2100 + logn, F, n, 0.8)
    s = q.qkdrec_syndrome(c, dev(b))
    out = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(max_iter=2, early_stop=False), want_post=True)
    pick = [0, F // 2 + 3, F - 1]
    s_ref = oracle.syndrome(rp, ci, b[pick])
    assert np.array_equal(host(s[pick]), s_ref)
    ref = oracle.decode(rp, ci, llr[pick].astype(np.float64), s_ref, "sp_flood", max_iter=2, early_stop=False)
    assert rel_ok(host(out["post"][pick]), ref["post"]).all()


def test_maximum_frame_count_of_one_launch():
    """F = 65535 x 32 frames (the most one decode accepts) of a 64-variable code:
    first, middle and last frames against the oracle; one frame more is refused."""
    n, F = 64, 65535 * 32
    rp, ci, M = code(2200, n, 0.5)
    c = q.Code(n, rp, ci)
    g = synth.philox(2201)
    b = g.integers(0, 2, size=(F, n)).astype(np.uint8)
    llr = ((2 / 0.8 ** 2) * ((1.0 - 2.0 * b) + 0.8 * g.standard_normal((F, n), dtype=np.float32))).astype(np.float32)
    s = q.qkdrec_syndrome(c, dev(b))
    out = q.qkdrec_decode_batch(c, dev(llr), s, q.DecodeOpts(algo="oms_flood", max_iter=3, early_stop=False),
                                want_post=True)
    pick = [0, 1048577, F - 1]
    ref = oracle.decode(rp, ci, llr[pick].astype(np.float64), oracle.syndrome(rp, ci, b[pick]), "oms_flood",
                        max_iter=3, early_stop=False, offset=0.5)
    assert rel_ok(host(out["post"][pick]), ref["post"]).all()
    del out
    torch.cuda.empty_cache()
    with pytest.raises(RuntimeError):
        q.qkdrec_decode_batch(c, torch.zeros((F + 1, n), device="cuda"), torch.zeros((F + 1, M), dtype=torch.uint8,
                                                                                        device="cuda"),
                              q.DecodeOpts(algo="oms_flood", max_iter=1))


def test_full_block_quantiser_and_llr_sampled():
    """2^27 samples (one SNR point of the sweep) through the quantiser and the
    slice-3 LLR with random lower bits: sampled positions against the oracle."""
    snr, m, N = 15.0, 5, 1 << 27
    lo, hi = oracle.quantiser_range(snr)
    x, y = synth.gaussian_pair(3, N, snr)
    idx, bits = q.qkdrec_quantise_slices(dev(y), m, lo, hi)
    g = synth.philox(2300)
    pos = np.sort(g.integers(0, N, size=20000))
    ridx, rbits = oracle.quantise(y[pos], m, lo, hi)
    assert np.array_equal(host(idx)[pos], ridx) and np.array_equal(host(bits)[:, pos], rbits)
    lower = g.integers(0, 2, size=(3, N)).astype(np.uint8)
    llr = q.qkdrec_slice_llr(dev(x), m, 3, lo, hi, snr ** -0.5, dev(lower))
    ref = oracle.slice_llr(x[pos].astype(np.float64), lower[:, pos], 3, m, lo, hi, snr ** -0.5)
    assert rel_ok(host(llr)[pos], ref).all()
