"""Analytic optimum of the sub-block length N_R -- oracle.

TEST INFRASTRUCTURE ONLY (imported by tests/ and bench.py's reference legs;
never by the library).  Plain FP64 numpy/scipy, written from the paper's
finite-length analysis in the order it is stated:

* Eq. SNR:   gamma = (V_A T / 2) / (1 + xi / 2),  xi = xi_ch + xi_d;
  I_AB = C(gamma) = 1/2 log2(1 + gamma).
* Eq. R_Finite (normal approximation of the finite-length AWGN capacity):
  C_Finite(N_R) = C(gamma) - (sqrt(N_R A) Q^-1(eps_EC) + 1/2 log2 N_R) / N_R,
  A the channel dispersion.
* Eq. AEP:  Delta_AEP = (m+1)^2 + 4 (m+1) sqrt(log2(2/eps_s^2))
                        + 2 log2(2/(eps^2 eps_s)) + 4 eps_s m / (eps sqrt N),
  eps = eps_EC + 2 eps_s + eps_PA + eps_PE.
* Appendix: S_BE = chi_BE at the worst-case estimates T^L and xi_ch^U of
  parameter estimation on N_e signals (t^ = sqrt(eta_d T),
  sigma^2 = T eta_d xi_ch + 1 + xi_d, tau = Q^-1(eps_PE / 2)).
* Eq. FiniteK, BPSRate, simplifiedOpt: with B_1 = N S_BE + sqrt(N) Delta_AEP
  + 2 log2(1/(2 eps_PA)) and B_2 = sum_j 7 (G_j / N_R) D_j c_h (Eq. EP and
  DeltaT: 7 operations per edge and iteration, G_j / N_R edges per sample of
  slice j's code, D_j iterations), the key rate in bits per second is
  K'(N_R) = (N C_Finite(N_R) - B_1) / (B_2 N_R), maximised over
  10^5 <= N_R <= N at the root of dK'/dN_R (Eq. diff_eq2) or at a boundary.

Readings where the printed formulas are garbled or silent (the same in the
library's implementation, which shares no code with this one):
  - A = gamma (gamma + 2) / (2 (gamma + 1)^2) (log2 e)^2, the AWGN dispersion
    in bits^2 of the cited finite-length analysis (the paper prints
    (log eps_EC)^2 in place of (log2 e)^2; dispersion="printed" takes that,
    with log2);
  - logarithms of information quantities in base 2 throughout, so the
    derivative of 1/2 log2 N_R / N_R carries 1/ln 2;
  - the symplectic eigenvalues with the squares the appendix drops restored
    (Psi_1's last bracket, Psi_2, Theta_1's denominator), Psi_2 with
    chi_ch in place of xi_ch, and the heterodyne detector term
    chi_het = (2 - eta_d + 2 xi_d) / eta_d (the appendix's chi_d refers to
    itself; xi_d is the detector noise);
  - N_e = N / 2 signals for parameter estimation unless given.
D_j (mean decoding iterations) and c_h are inputs: the library's decoder
measures both on B300.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.optimize import brentq
from scipy.special import ndtri

LN2 = math.log(2.0)


def qinv(p: float) -> float:
    """Q^-1(p): z with P(N(0,1) > z) = p."""
    return float(-ndtri(p))


def snr(va: float, T: float, xi: float) -> float:
    return 0.5 * va * T / (1.0 + 0.5 * xi)


def capacity(g: float) -> float:
    return 0.5 * math.log2(1.0 + g)


def dispersion(g: float, eps_ec: float, form: str = "awgn") -> float:
    if form == "awgn":
        return g * (g + 2.0) / (2.0 * (g + 1.0) ** 2) * math.log2(math.e) ** 2
    return 0.5 * g * (g + 2.0) / (g + 1.0) ** 2 * math.log2(eps_ec) ** 2


def c_finite(nr: float, i_ab: float, A: float, q: float) -> float:
    return i_ab - (math.sqrt(nr * A) * q + 0.5 * math.log2(nr)) / nr


def delta_aep(m: int, eps: float, eps_s: float, N: float) -> float:
    return ((m + 1) ** 2 + 4 * (m + 1) * math.sqrt(math.log2(2.0 / eps_s ** 2))
            + 2.0 * math.log2(2.0 / (eps ** 2 * eps_s)) + 4.0 * eps_s * m / (eps * math.sqrt(N)))


def g_entropy(x: float) -> float:
    """(x+1) log2(x+1) - x log2 x, the entropy of a thermal state of mean photon number x."""
    if x <= 0.0:
        return 0.0
    return (x + 1.0) * math.log2(x + 1.0) - x * math.log2(x)


def symplectic_pair(a: float, b: float):
    r = math.sqrt(max(a * a - 4.0 * b, 0.0))
    return math.sqrt((a + r) / 2.0), math.sqrt(max((a - r) / 2.0, 0.0))


def holevo_be(va: float, T: float, xi_ch: float, eta: float, xi_d: float):
    """chi_BE = chi_E - chi_E|B for reverse reconciliation with heterodyne detection
    (appendix, squares restored): returns (chi_BE, (psi1, psi2, theta1, theta2))."""
    V = va + 1.0
    chi_ch = (1.0 - T) / T + xi_ch
    Psi1 = V ** 2 * (1.0 - 2.0 * T) + 2.0 * T + T ** 2 * (V + chi_ch) ** 2
    Psi2 = T ** 2 * (V * chi_ch + 1.0) ** 2
    psi1, psi2 = symplectic_pair(Psi1, Psi2)
    chi_het = (2.0 - eta + 2.0 * xi_d) / eta
    chi_tot = chi_ch + chi_het / T
    Theta1 = (Psi1 * chi_het ** 2 + Psi2 + 1.0 + 2.0 * chi_het * (T * (V + chi_ch) + V * math.sqrt(Psi2))
              + 2.0 * T * (va ** 2 + 2.0 * va)) / (T ** 2 * (V + chi_tot) ** 2)
    Theta2 = ((V + chi_het * math.sqrt(Psi2)) / (T * (V + chi_tot))) ** 2
    th1, th2 = symplectic_pair(Theta1, Theta2)
    chi_e = g_entropy((psi1 - 1.0) / 2.0) + g_entropy((psi2 - 1.0) / 2.0)
    chi_eb = g_entropy((th1 - 1.0) / 2.0) + g_entropy((th2 - 1.0) / 2.0)
    return chi_e - chi_eb, (psi1, psi2, th1, th2)


def s_be(va, T, xi_ch, xi_d, eta, eps_pe, n_e):
    """S_BE^eps_PE: chi_BE at the confidence-interval ends T^L, xi_ch^U (appendix)."""
    t_hat = math.sqrt(eta * T)
    sig2 = T * eta * xi_ch + 1.0 + xi_d
    tau = qinv(eps_pe / 2.0)
    t_low = (t_hat - tau * math.sqrt(sig2 / (n_e * va))) ** 2
    xi_up = (sig2 + tau * sig2 * math.sqrt(2.0) / math.sqrt(n_e) - 1.0 - xi_d) / t_hat ** 2
    chi, _ = holevo_be(va, t_low, xi_up, eta, xi_d)
    return chi, t_low, xi_up


def setup(N=1e9, m=5, eps_ec=2.5e-10, eps_s=1.25e-10, eps_pa=2.5e-10, eps_pe=2.5e-10, va=5.0, T=0.9,
          xi_ch=0.0186, xi_d=0.0133, eta=1.0, n_e=None, c_h=3.2e-9, g=None, d_iters=None, form="awgn"):
    """The constants of K'(N_R) for a parameter set (defaults: the paper's standard
    CV-QKD settings of Sec. IV-B).  g[j]: edges per sample of slice j's code (0 for
    a disclosed slice), d_iters[j]: its decoding iterations."""
    if n_e is None:
        n_e = N / 2.0
    g = [3.0] * m if g is None else list(g)
    d_iters = [1.0] * m if d_iters is None else list(d_iters)
    gam = snr(va, T, xi_ch + xi_d)
    i_ab = capacity(gam)
    A = dispersion(gam, eps_ec, form)
    q = qinv(eps_ec)
    eps = eps_ec + 2.0 * eps_s + eps_pa + eps_pe
    daep = delta_aep(m, eps, eps_s, N)
    sbe, t_low, xi_up = s_be(va, T, xi_ch, xi_d, eta, eps_pe, n_e)
    b1 = N * sbe + math.sqrt(N) * daep + 2.0 * math.log2(1.0 / (2.0 * eps_pa))
    b2 = sum(7.0 * gj * dj * c_h for gj, dj in zip(g, d_iters))
    return dict(N=N, snr=gam, i_ab=i_ab, A=A, q=q, delta_aep=daep, s_be=sbe, t_low=t_low, xi_up=xi_up,
                b1=b1, b2=b2)


def key_rate(c, nr):
    """K'_Finite(N_R) in bits per second (Eq. BPSRate)."""
    return (c["N"] * c_finite(nr, c["i_ab"], c["A"], c["q"]) - c["b1"]) / (c["b2"] * nr)


def dkey_rate(c, nr):
    """dK'/dN_R times B_2 N_R^2 / N (the bracket of Eq. diff_eq2, base-2 logarithms)."""
    return (1.5 * math.sqrt(c["A"]) * c["q"] / math.sqrt(nr) + (math.log2(nr) - 0.5 / LN2) / nr - c["i_ab"]
            + c["b1"] / c["N"])


def optimise(nr_min=1e5, **kw):
    """Maximise K'(N_R) over nr_min <= N_R <= N: dict(nr_opt, k_opt, stationary, boundary, ...)."""
    c = setup(**kw)
    lo, hi = nr_min, c["N"]
    stationary = None
    f_lo, f_hi = dkey_rate(c, lo), dkey_rate(c, hi)
    if f_lo > 0 > f_hi:
        stationary = brentq(lambda t: dkey_rate(c, math.exp(t)), math.log(lo), math.log(hi), xtol=1e-14, rtol=1e-14)
        stationary = math.exp(stationary)
    cands = [lo, hi] + ([stationary] if stationary else [])
    best = max(cands, key=lambda x: key_rate(c, x))
    return dict(c, nr_opt=best, k_opt=key_rate(c, best), stationary=stationary, boundary=best != stationary)
