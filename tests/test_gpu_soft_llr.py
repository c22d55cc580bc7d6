"""GPU soft-conditioned slice LLR against the FP64 oracle.

Lower slices known softly (finite LLRs of any size and sign, including values
that contradict the interval x lies in), infinite lower LLRs against the
hard-conditioned LLR, the no-information case, and a short soft-chained
reconciliation against the oracle's own soft chain.
"""
import numpy as np
import pytest

import oracle
import synth
from _workloads import TOL, rel_ok

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


@pytest.mark.parametrize("snr,m,label", [(3.0, 5, "gray"), (15.0, 5, "gray"), (2.0, 4, "binary"), (3.0, 6, "gray")])
def test_soft_llr_vs_oracle(snr, m, label):
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    x, y = synth.gaussian_pair(300, 20_000, snr)
    x = np.concatenate([x, np.array([-6.0, 6.0, 0.0, 4.9, -5.5], np.float32)]).astype(np.float32)
    g = np.random.default_rng(301)
    for j in range(m):
        post = (g.normal(size=(j, x.size)) * g.choice([0.3, 3.0, 12.0, 40.0], size=(j, 1))).astype(np.float32)
        got = q.qkdrec_slice_llr_soft(dev(x), m, j, lo, hi, s, dev(post) if j else None, label).cpu().numpy()
        ref = oracle.slice_llr_soft(x.astype(np.float64), post.astype(np.float64), j, m, lo, hi, s, label)
        ok = rel_ok(got, ref)
        assert ok.all(), (j, np.argwhere(~ok)[:5].ravel(), got[~ok][:5], ref[~ok][:5])


@pytest.mark.parametrize("j", [1, 2, 4])
def test_infinite_lower_llrs_match_hard_conditioning(j):
    snr, m = 3.0, 5
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    x, y = synth.gaussian_pair(310, 30_000, snr)
    _, bits = q.qkdrec_quantise_slices(dev(y), m, lo, hi, want_idx=False)
    post = torch.stack([q.qkdrec_bits_to_llr(bits[l].contiguous()) for l in range(j)])
    b = bits[:j].cpu().numpy()
    pl = post.cpu().numpy()
    assert np.all(np.isinf(pl)) and np.array_equal(pl < 0, b == 1)
    soft = q.qkdrec_slice_llr_soft(dev(x), m, j, lo, hi, s, post).cpu().numpy()
    hard = q.qkdrec_slice_llr(dev(x), m, j, lo, hi, s, bits[:j].contiguous()).cpu().numpy()
    ref = oracle.slice_llr(x.astype(np.float64), b, j, m, lo, hi, s)
    assert rel_ok(soft, ref).all() and rel_ok(hard, ref).all()


def test_no_lower_information_msb_is_sign_of_y():
    from scipy.special import log_ndtr
    snr, m = 3.0, 5
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    x = np.linspace(-3, 3, 4001).astype(np.float32)
    got = q.qkdrec_slice_llr_soft(dev(x), m, m - 1, lo, hi, s, dev(np.zeros((m - 1, x.size), np.float32)))
    ref = np.clip(log_ndtr(-x.astype(np.float64) / s) - log_ndtr(x.astype(np.float64) / s), -30, 30)
    assert rel_ok(got.cpu().numpy(), ref).all()


def test_soft_chained_reconciliation_vs_oracle():
    """Slices 0..4 of 6 frames (n = 1024, SNR 3): each slice's LLRs from the lower
    slices' decoder posteriors (disclosed slices as known bits), SP flooding;
    decoded words equal the oracle's soft chain wherever both converge."""
    snr, m, n, F = 3.0, 5, 1024, 6
    lo, hi = oracle.quantiser_range(snr)
    s = snr ** -0.5
    rates = [0.0, 0.0, 0.25, 0.75, 0.3125]
    x, y = synth.gaussian_pair(320, F * n, snr)
    _, bits = oracle.quantise(y, m, lo, hi)
    post_g = torch.zeros((m, F * n), dtype=torch.float32, device="cuda")
    post_r = np.zeros((m, F * n))
    agreed = 0
    for j in range(m):
        if rates[j] == 0:
            q.qkdrec_bits_to_llr(dev(bits[j]), out=post_g[j])
            post_r[j] = np.where(bits[j] == 0, np.inf, -np.inf)
            continue
        rp, ci, _ = synth.make_regular_code(330 + j, n, synth.checks_for_rate(n, rates[j]))
        c = q.Code(n, rp, ci)
        synd = oracle.syndrome(rp, ci, bits[j].reshape(F, n))
        lg = q.qkdrec_slice_llr_soft(dev(x), m, j, lo, hi, s, post_g[:j] if j else None)
        lr = oracle.slice_llr_soft(x.astype(np.float64), post_r[:j], j, m, lo, hi, s)
        out = q.qkdrec_decode_batch(c, lg.view(F, n), dev(synd), q.DecodeOpts(max_iter=50), want_post=True)
        ref = oracle.decode(rp, ci, lr.reshape(F, n), synd, "sp_flood", max_iter=50)
        post_g[j] = out["post"].reshape(-1)
        post_r[j] = ref["post"].reshape(-1)
        both = (out["converged"].cpu().numpy() == 1) & (ref["converged"] == 1)
        assert np.array_equal(out["bits"].cpu().numpy()[both], ref["bits"][both])
        agreed += int(both.sum())
    assert agreed > 0
