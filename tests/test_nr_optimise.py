"""The analytic optimum sub-block length (Sec. III-B/C, IV, appendix).

Oracle (oracle/nropt.py) pinned by mathematics, since the paper's printed
optimum does not follow from its printed formulas under any reading (see the
readings in oracle/nropt.py): closed forms of the Holevo quantity for a
noiseless and a pure-loss channel, the inverse Q-function against erfc, the
finite-length capacity's limit, and the returned N_R being a stationary
maximum by finite differences.  The library's implementation (a separate C
restatement) must agree with the oracle and its second derivative with
finite differences.
"""
import math

import numpy as np
import pytest

import paper_2108_08418_b300 as q
from oracle import nropt

STANDARD = dict(N=1e9, m=5, eps_ec=2.5e-10, eps_s=1.25e-10, eps_pa=2.5e-10, eps_pe=2.5e-10, va=5.0, T=0.9,
                xi_ch=0.0186, xi_d=0.0133, eta=1.0, c_h=3.2e-9)
GREEN = dict(N=1e10, m=5, eps_ec=2.5e-7, eps_s=1.25e-7, eps_pa=2.5e-7, eps_pe=2.5e-7, va=4.0, T=0.92,
             xi_ch=0.0180, xi_d=0.0128, eta=1.0, c_h=3.2e-9)


def to_c(kw):
    """Keyword names of the library binding for an oracle parameter set."""
    ren = dict(N="n_signals", m="m_slices", T="transmissivity", eta="eta_d", n_e="n_estimation")
    out = {ren.get(k, k): v for k, v in kw.items() if k not in ("g", "d_iters", "form")}
    out["dispersion_form"] = 1 if kw.get("form") == "printed" else 0
    return out


def test_holevo_closed_forms():
    # a lossless noiseless channel leaves Eve nothing
    chi, (p1, p2, t1, t2) = nropt.holevo_be(5.0, 1.0, 0.0, 1.0, 0.0)
    assert abs(chi) < 1e-12 and abs(p1 - 1) < 1e-9 and abs(p2 - 1) < 1e-9
    # pure loss: Eve holds the other beam-splitter output, symplectic eigenvalues
    # (1 - T) V + T and 1, so chi_E = g((1 - T) V_A / 2)
    for va, T in ((5.0, 0.5), (3.0, 0.9), (10.0, 0.1)):
        chi, (p1, p2, t1, t2) = nropt.holevo_be(va, T, 0.0, 1.0, 0.0)
        assert abs(p1 - ((1 - T) * (va + 1) + T)) < 1e-9 and abs(p2 - 1.0) < 1e-9
        assert 0.0 < chi < nropt.g_entropy((1 - T) * va / 2)
    # more excess noise can only help Eve
    a = nropt.holevo_be(5.0, 0.9, 0.01, 1.0, 0.01)[0]
    b = nropt.holevo_be(5.0, 0.9, 0.05, 1.0, 0.01)[0]
    assert b > a > 0


def test_inverse_q_and_capacity_limit():
    for p in (0.4, 1e-3, 2.5e-10, 1e-15):
        z = nropt.qinv(p)
        assert abs(0.5 * math.erfc(z / math.sqrt(2)) / p - 1) < 1e-10
    c = nropt.setup(**STANDARD)
    assert abs(nropt.c_finite(1e30, c["i_ab"], c["A"], c["q"]) - c["i_ab"]) < 1e-12
    assert nropt.c_finite(1e6, c["i_ab"], c["A"], c["q"]) < nropt.c_finite(1e8, c["i_ab"], c["A"], c["q"])


@pytest.mark.parametrize("kw", [dict(STANDARD, form="printed", d_iters=[20] * 5),
                                dict(GREEN, form="printed", d_iters=[15] * 5),
                                dict(STANDARD, form="printed", d_iters=[8, 14, 20, 14, 9])])
def test_oracle_optimum_is_a_stationary_maximum(kw):
    r = nropt.optimise(**kw)
    assert r["stationary"] is not None and not r["boundary"]
    x = r["nr_opt"]
    c = {k: r[k] for k in ("N", "i_ab", "A", "q", "b1", "b2")}
    k0 = nropt.key_rate(c, x)
    for d in (1e-3, 1e-2, 1e-1):
        assert k0 >= nropt.key_rate(c, x * (1 + d)) and k0 >= nropt.key_rate(c, x * (1 - d))
    # the derivative vanishes there (central differences, relative to its scale)
    h = x * 1e-4
    dk = (nropt.key_rate(c, x + h) - nropt.key_rate(c, x - h)) / (2 * h)
    assert abs(dk) * x < 1e-5 * abs(k0)


def test_oracle_optimum_at_the_floor_when_the_rate_only_falls():
    # with the AWGN dispersion the stationary point lies below 1e5: the optimum is
    # the lower end of the range, where K' is falling
    r = nropt.optimise(**STANDARD, d_iters=[20] * 5)
    assert r["boundary"] and r["nr_opt"] == 1e5
    c = {k: r[k] for k in ("N", "i_ab", "A", "q", "b1", "b2")}
    assert nropt.key_rate(c, 1e5) > nropt.key_rate(c, 1.1e5) > nropt.key_rate(c, 1e9)


@pytest.mark.parametrize("kw", [dict(STANDARD, d_iters=[20] * 5), dict(STANDARD, form="printed", d_iters=[20] * 5),
                                dict(GREEN, form="printed", d_iters=[15] * 5),
                                dict(STANDARD, form="printed", g=[0, 0, 3, 3, 3], d_iters=[0, 0, 21, 14, 15]),
                                dict(STANDARD, va=2.0, T=0.5, xi_ch=0.01, form="printed", d_iters=[10] * 5)])
def test_library_matches_the_oracle(kw):
    g = kw.get("g", [3.0] * kw["m"])
    d = kw["d_iters"]
    ref = nropt.optimise(**kw)
    got = q.qkdrec_nr_optimise(g, d, **to_c(kw))
    for k_c, k_o in (("snr", "snr"), ("i_ab", "i_ab"), ("dispersion", "A"), ("qinv_ec", "q"),
                     ("delta_aep", "delta_aep"), ("s_be", "s_be"), ("t_low", "t_low"), ("xi_up", "xi_up"),
                     ("b1", "b1"), ("b2", "b2"), ("nr_opt", "nr_opt"), ("key_rate_opt", "k_opt")):
        assert got[k_c] == pytest.approx(ref[k_o], rel=1e-9, abs=1e-12), k_c
    assert bool(got["at_boundary"]) == bool(ref["boundary"])
    # the library's second derivative against its own key rate by central differences
    x = got["nr_opt"]
    h = x * 1e-3
    kr = lambda t: q.qkdrec_nr_key_rate(t, g, d, **to_c(kw))
    fd2 = (kr(x + h) - 2 * kr(x) + kr(x - h)) / h ** 2
    assert got["d2_key_rate"] == pytest.approx(fd2, rel=1e-3)
    c = nropt.setup(**kw)
    if not got["at_boundary"]:
        assert got["d2_key_rate"] < 0
    assert kr(got["nr_opt"]) == pytest.approx(nropt.key_rate(c, got["nr_opt"]), rel=1e-12)


def test_library_rejects_bad_parameters():
    with pytest.raises(q.QkdrecError):
        q.qkdrec_nr_optimise([3.0] * 5, [20.0] * 5, eps_ec=0.7)
    with pytest.raises(q.QkdrecError):
        q.qkdrec_nr_optimise([0.0] * 5, [20.0] * 5)
    with pytest.raises(ValueError):
        q.qkdrec_nr_optimise([3.0] * 4, [20.0] * 5)
