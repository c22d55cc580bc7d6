"""Pins of the oracle's forward error bounds of the FP16- and FP32-message
decoder forms (oracle/bound.c).

The bound is checked against an independent emulation of those forms written
here with numpy's IEEE binary32 arithmetic and binary16 storage: every
emulated posterior must lie within the bound's radius of the FP64 posterior,
and a coarser storage (8-bit significand) must leave it somewhere, so the
radius is neither wrong nor vacuous.  The midpoints must be bp.c's FP64
results exactly.
"""
import numpy as np
import pytest

import oracle
from _workloads import bpsk_frames, code

F32 = np.float32


def phi64(x):
    return np.log1p(2.0 / np.expm1(x))


def bf16ish(x):
    """Round float32 values to an 8-bit significand (nearest, ties to even)."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def store_as(kind):
    if kind == "f16":
        return lambda x: x.astype(np.float16).astype(F32)
    if kind == "f32":
        return lambda x: x.astype(F32)
    return bf16ish


def emulate(rp, ci, llr, synd, algo, T, kind="f16", beta=0.5, layers=None):
    """The decoder rules in binary32 with messages stored by `kind`, all frames at once."""
    st = store_as(kind)
    Fn, n = llr.shape
    M = len(rp) - 1
    E = rp[-1]
    llr = llr.astype(F32)
    L = llr.copy()
    m = np.zeros((Fn, E), F32)
    sgn_s = np.where(synd & 1, F32(-1), F32(1))
    order = [list(range(M))] if algo != "oms_layered" else \
        [list(layers[2][layers[1][l]:layers[1][l + 1]]) for l in range(len(layers[1]) - 1)]
    for _ in range(T):
        mnew = m.copy()
        for group in order:
            for c in group:
                e = np.arange(rp[c], rp[c + 1])
                q = (L[:, ci[e]] - m[:, e]).astype(F32)
                neg = q < 0
                for i in range(len(e)):
                    other = np.ones(len(e), bool)
                    other[i] = False
                    sign = sgn_s[:, c] * np.where(np.sum(neg[:, other], axis=1) & 1, F32(-1), F32(1))
                    if algo == "sp_flood":
                        a = np.clip(np.abs(q[:, other]).astype(np.float64), 1e-30, 30.0)
                        f = phi64(a).astype(F32)
                        s = F32(0)
                        for k in range(f.shape[1]):
                            s = (s + f[:, k]).astype(F32)
                        mag = phi64(np.clip(s.astype(np.float64), 1e-30, 30.0)).astype(F32)
                    else:
                        mn = np.min(np.abs(q[:, other]), axis=1)
                        mag = np.maximum((mn - F32(beta)).astype(F32), F32(0))
                    mnew[:, e[i]] = st((sign * mag).astype(F32))
                if algo == "oms_layered":
                    m[:, e] = mnew[:, e]
                    L[:, ci[e]] = (q + m[:, e]).astype(F32)
        if algo != "oms_layered":
            m = mnew
            L = llr.copy()
            for e in range(E):
                L[:, ci[e]] = (L[:, ci[e]] + m[:, e]).astype(F32)
    return L.astype(np.float64)


CASES = [("oms_flood", 4), ("sp_flood", 4), ("oms_layered", 3)]


@pytest.fixture(scope="module")
def frames():
    n = 256
    rp, ci, _ = code(401, n, 0.5)
    b, llr = bpsk_frames(402, 6, n, 0.8)
    rp2, ci2, _ = code(403, n, 0.75)                     # check degree 12
    b2, llr2 = bpsk_frames(404, 6, n, 0.55)
    return [(rp, ci, b, llr, n), (rp2, ci2, b2, llr2, n)]


@pytest.mark.parametrize("algo,T", CASES)
def test_midpoint_is_the_fp64_decoder(frames, algo, T):
    for rp, ci, b, llr, n in frames:
        s = oracle.syndrome(rp, ci, b)
        for t in range(T + 1):
            post, rad = oracle.decode_bound(rp, ci, llr, s, algo, t)
            ref = oracle.decode(rp, ci, llr, s, algo, max_iter=t, early_stop=False)["post"]
            assert np.array_equal(post, ref)
            assert np.all(rad >= 0) and (t > 0 or np.all(rad == 0))


@pytest.mark.parametrize("kind", ["f16", "f32"])
@pytest.mark.parametrize("algo,T", CASES)
def test_emulated_low_precision_decoder_stays_inside_the_bound(frames, algo, T, kind):
    for rp, ci, b, llr, n in frames:
        s = oracle.syndrome(rp, ci, b)
        layers = oracle.greedy_layers(rp, ci, n)
        for t in range(1, T + 1):
            post, rad = oracle.decode_bound(rp, ci, llr, s, algo, t, f16=(kind == "f16"), layers=layers)
            emu = emulate(rp, ci, llr, s, algo, t, kind, layers=layers)
            gap = np.abs(emu - post)
            assert np.all(gap <= rad), (t, float(np.max(gap - rad)))
            # and the radius is informative: most posteriors keep their sign for certain
            assert np.mean(np.abs(post) > rad) > 0.95


@pytest.mark.parametrize("algo,T", CASES)
def test_coarser_storage_leaves_the_fp16_bound(frames, algo, T):
    """Messages stored with an 8-bit significand (2^-9 relative rounding, 4x the
    binary16 unit roundoff) break the binary16 radius somewhere: a bound loose
    enough to hide that would not pin the FP16 form."""
    rp, ci, b, llr, n = frames[0]
    s = oracle.syndrome(rp, ci, b)
    layers = oracle.greedy_layers(rp, ci, n)
    broke = False
    for t in range(1, T + 1):
        post, rad = oracle.decode_bound(rp, ci, llr, s, algo, t, layers=layers)
        emu = emulate(rp, ci, llr, s, algo, t, "bf16ish", layers=layers)
        broke |= bool(np.any(np.abs(emu - post) > rad))
    assert broke


def test_storage_radius_of_one_check_by_hand():
    """One check of degree 3, offset min-sum, one flooding iteration, syndrome 0:
    q = llr = (2, -3, 5), so v0 <- -(3 - 0.5) = -2.5, v1 <- +1.5, v2 <- -1.5 and
    the posteriors are -0.5, -1.5, 3.5.  Radii by the rules: r_q = u32 |q| (the
    subtraction L - 0 is charged one rounding); the minimum over the other edges
    moves by at most u32 x that minimum; max(x - 0.5, 0) adds u32 |x - 0.5|;
    binary16 storage adds u16 (|m| + r) + 2^-25; the one-message variable sum adds
    u32 (1 + u32) (|llr| + |m| + r_m)."""
    rp = np.array([0, 3], np.int32)
    ci = np.array([0, 1, 2], np.int32)
    llr = np.array([[2.0, -3.0, 5.0]])
    post, rad = oracle.decode_bound(rp, ci, llr, np.zeros((1, 1), np.uint8), "oms_flood", 1)
    assert np.array_equal(post[0], [-0.5, -1.5, 3.5])
    u32, u16, sub = 2.0 ** -24, 2.0 ** -11, 2.0 ** -25
    mn = np.array([3.0, 2.0, 2.0])                      # min |q| over the other edges
    mag = mn - 0.5
    rmag = u32 * mn + u32 * (mag + u32 * mn)
    rs = rmag + u16 * (mag + rmag) + sub
    expect = rs + u32 * (1 + u32) * (np.abs(llr[0]) + mag + rs)
    assert np.allclose(rad[0], expect, rtol=1e-12, atol=0)
