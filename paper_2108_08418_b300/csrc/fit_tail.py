"""Coefficients of the Gaussian upper tail used by the slice LLR kernel.

Q(z) = P(N(0,1) > z) = e^{-z^2/2} M(z) / sqrt(2 pi), with M the Mills ratio.
For z in [0, ZMAX] the kernel evaluates

    Q(z) = e^{-z^2/2} r p(s),   r = 1 / (z + KAPPA),  s = z r  in [0, ZMAX / (ZMAX + KAPPA)],

where p is a degree-DEG polynomial fitted here to (z + KAPPA) M(z) / sqrt(2 pi)
with minimal maximum relative error (Lawson's iteratively reweighted least
squares on Chebyshev points, values from mpmath at 40 digits).  Beyond ZMAX the
tail is below 1e-44, under the smallest normal float, and the kernel returns 0.

Run:  python paper_2108_08418_b300/csrc/fit_tail.py   (prints the coefficients,
highest degree first, in the order q_tail_fit2 in quant_llr.cu applies them)
"""
import mpmath as mp
import numpy as np

KAPPA = 4.0
ZMAX = 14.0
DEG = 8
mp.mp.dps = 40


def target(z):
    z = mp.mpf(z)
    return float((z + KAPPA) * mp.erfc(z / mp.sqrt(2)) / 2 * mp.exp(z * z / 2))


def fit(npts=400, iters=300):
    smax = ZMAX / (ZMAX + KAPPA)
    s = (1 - np.cos(np.pi * np.arange(npts) / (npts - 1))) / 2 * smax
    z = KAPPA * s / (1 - s)
    f = np.array([target(v) for v in z])
    V = np.vander(s, DEG + 1, increasing=True)
    w = np.full(npts, 1.0 / npts)
    for _ in range(iters):
        sw = np.sqrt(w) / f
        c, *_ = np.linalg.lstsq(V * sw[:, None], f * sw, rcond=None)
        e = np.abs(V @ c / f - 1)
        w = w * e
        w /= w.sum()
    return c, e.max()


if __name__ == "__main__":
    c, err = fit()
    print(f"// degree {DEG}, kappa {KAPPA}, z in [0, {ZMAX}]: max relative error {err:.2e} in exact arithmetic")
    for i in range(DEG, -1, -1):
        print("  c[%d] = %.9ef" % (i, c[i]))
