"""FP64 oracle for the slice-reconciliation hot path.

TEST INFRASTRUCTURE ONLY.  Only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` may import this package.
The CUDA library never calls it, and it imports nothing from the library: the
two share only the seeded input generators in `synth/`.

Everything here is plain FP64 numpy/scipy (plus plain C for the iterative
decoders in bp.c), written from the paper's definitions:

* quantiser + labelling: constant-step quantiser M(.) with 2^m bins centred on
  zero (Sec. III-B, text after Eq. beta), m-bit labels with LSB l_0
  (Sec. III-B, step 1 and footnote), Gray labelling (Sec. II, Step 4);
* slices S_j = bit plane j (Sec. III-B, step 2);
* slice LLRs from Alice's quadratures and the already reconciled lower slices
  (Sec. III-B, steps 4-5; multi-stage hard decoding, Sec. II footnote);
* conditional slice capacities and the code rate rule (Sec. II Step 5,
  Sec. III-B "closest to the capacity"); chain rule and Slepian-Wolf bound
  (Eqs. beta2, SWB);
* syndrome s_j = H_j S_j (Sec. II Step 5, Sec. III-B step 2);
* BP decoders (Sec. III-C) -- see bp.c; forward error radii of the FP16- and
  FP32-message forms around them -- see bound.c.

Readings where the paper is silent are listed in the module constants and in
the function docstrings (quantiser range +-4 sigma_y, tie rule, LLR clip, SP
saturation constants, layer partition, integer min-sum widths).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np
from scipy import integrate
from scipy.special import log_ndtr, ndtr

LLR_CLIP = 30.0          # channel LLRs are clipped to +-30 nats (reading; paper silent)
SP_A_MIN = 1e-30         # sum-product saturation: |q| and the phi-sum clamp to [A_MIN, A_MAX]
SP_A_MAX = 30.0
INT_QMAX = 31            # 6-bit integer min-sum: messages in [-31, 31]
INT_PMAX = 32767         # int16 saturating posterior

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


# --------------------------------------------------------------------------- C part
def _lib():
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        srcs = [os.path.join(_HERE, "bp.c"), os.path.join(_HERE, "bound.c")]
        so = os.path.join(_BUILD, "liboracle_bp.so")
        if not os.path.exists(so) or os.path.getmtime(so) < max(os.path.getmtime(f) for f in srcs):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", *srcs, "-o", tmp, "-lm"])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        P = ctypes.c_void_p
        I = ctypes.c_int
        D = ctypes.c_double
        lib.oracle_sp_flood.argtypes = [I, I, P, P, P, P, I, I, I, P, P, P, P]
        lib.oracle_oms_flood.argtypes = [I, I, P, P, P, P, I, I, D, I, P, P, P, P]
        lib.oracle_oms_layered.argtypes = [I, I, P, P, I, P, P, P, P, I, I, D, I, P, P, P, P]
        lib.oracle_ioms.argtypes = [I, I, I, P, P, I, P, P, P, P, I, I, D, I, P, P, P, P]
        lib.oracle_woms.argtypes = [I, I, P, P, P, P, P, I, I, P, P, P, P, P, P]
        lib.oracle_woms.restype = I
        lib.oracle_lowp_bound.argtypes = [I, I, I, I, P, P, I, P, P, P, P, I, I, D, D, P, P]
        lib.oracle_lowp_bound.restype = I
        for f in (lib.oracle_sp_flood, lib.oracle_oms_flood, lib.oracle_oms_layered, lib.oracle_ioms):
            f.restype = I
        _LIB = lib
        return lib


def build() -> None:
    """Compile the C part of the oracle (building the checker is not using it)."""
    _lib()


# ----------------------------------------------------------------- quantiser (a1)
def quantiser_range(snr: float, va: float = 1.0):
    """[lo, hi] = [-4 sigma_y, 4 sigma_y], sigma_y^2 = V_A + 1/SNR (model value).

    Reading: the paper fixes a constant step on 2^m bins centred on zero whose
    size depends on the SNR (Sec. III-B, after Eq. beta) but prints no range.
    """
    sy = np.sqrt(va + 1.0 / snr)
    return -4.0 * sy, 4.0 * sy


def thresholds(m: int, lo: float, hi: float) -> np.ndarray:
    """Interior thresholds t_k = lo + k (hi - lo) / 2^m, k = 1 .. 2^m - 1 (FP64)."""
    K = 1 << m
    delta = (hi - lo) / K
    return lo + delta * np.arange(1, K, dtype=np.float64)


def labels(m: int, label: str = "gray") -> np.ndarray:
    """m-bit label of each interval index k: Gray k ^ (k >> 1), or binary k."""
    k = np.arange(1 << m, dtype=np.int64)
    if label == "gray":
        return k ^ (k >> 1)
    if label == "binary":
        return k
    raise ValueError(label)


def quantise(y, m: int, lo: float, hi: float, label: str = "gray"):
    """Interval index and bit planes of Bob's samples.

    Interval k = number of interior thresholds t <= y, so a sample exactly on
    t_k goes to interval k (the upper one), below t_1 to 0, from t_{2^m-1} on
    to 2^m - 1.  Bit plane j = bit j of the label, j = 0 the LSB l_0.
    Returns (idx uint8 [count], bits uint8 [m][count]).
    """
    y = np.asarray(y, dtype=np.float64).ravel()
    t = thresholds(m, lo, hi)
    k = np.searchsorted(t, y, side="right")
    lab = labels(m, label)[k]
    bits = np.stack([((lab >> j) & 1).astype(np.uint8) for j in range(m)]) if m > 0 else None
    return k.astype(np.uint8), bits


# ------------------------------------------------- interval probabilities (a3)
def _log_interval_prob(a, b):
    """log(Phi(b) - Phi(a)) for a < b (standardised bounds), stable in both tails."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    out = np.empty(np.broadcast(a, b).shape)
    a, b = np.broadcast_arrays(a, b)
    right = a >= 0.0          # whole interval above the mean: Q(a) - Q(b)
    left = b <= 0.0           # whole interval below the mean: Phi(b) - Phi(a)
    mid = ~(right | left)
    with np.errstate(divide="ignore", invalid="ignore"):
        la, lb = log_ndtr(-a[right]), log_ndtr(-b[right])
        out[right] = la + np.log1p(-np.exp(lb - la))
        la, lb = log_ndtr(a[left]), log_ndtr(b[left])
        out[left] = lb + np.log1p(-np.exp(la - lb))
        out[mid] = np.log1p(-(ndtr(a[mid]) + ndtr(-b[mid])))
    return out


def interval_logprob(x, m: int, lo: float, hi: float, sigma_n: float) -> np.ndarray:
    """log P(k | x) for every interval k: y = x + n, n ~ N(0, sigma_n^2).

    P(k|x) = Phi((t_{k+1} - x)/sigma_n) - Phi((t_k - x)/sigma_n) with
    t_0 = -inf, t_{2^m} = +inf.  Shape [count, 2^m].
    """
    x = np.asarray(x, dtype=np.float64).ravel()
    t = np.concatenate([[-np.inf], thresholds(m, lo, hi), [np.inf]])
    a = (t[None, :-1] - x[:, None]) / sigma_n
    b = (t[None, 1:] - x[:, None]) / sigma_n
    return _log_interval_prob(a, b)


def _logsumexp_masked(lp, mask):
    """Row-wise log sum_{k in mask} exp(lp[k]); -inf for an empty mask."""
    v = np.where(mask, lp, -np.inf)
    mx = v.max(axis=1)
    fin = np.isfinite(mx)
    out = np.full(lp.shape[0], -np.inf)
    out[fin] = mx[fin] + np.log(np.exp(v[fin] - mx[fin, None]).sum(axis=1))
    return out


def slice_llr(x, lower_bits, j: int, m: int, lo: float, hi: float, sigma_n: float,
              label: str = "gray", clip: float = LLR_CLIP) -> np.ndarray:
    """Channel LLR of slice j for Alice (Sec. III-B steps 4-5, multi-stage hard decoding).

    L_j(i) = ln sum_{k in K0(i)} P(k|x_i) - ln sum_{k in K1(i)} P(k|x_i),
    K_b(i) = { k : bit j of label(k) = b, bits 0..j-1 of label(k) = the
    reconciled lower bits of sample i }.  lower_bits: uint8 [j][count] (None
    for j = 0).  Clipped to [-clip, clip] (reading: paper silent).
    """
    x = np.asarray(x, dtype=np.float64).ravel()
    lp = interval_logprob(x, m, lo, hi, sigma_n)
    lab = labels(m, label)
    low = np.zeros(x.shape[0], dtype=np.int64)
    for i in range(j):
        low |= np.asarray(lower_bits[i], dtype=np.int64).ravel() << i
    lowmask = (1 << j) - 1
    match = (lab[None, :] & lowmask) == low[:, None]
    bj = (lab >> j) & 1
    l0 = _logsumexp_masked(lp, match & (bj[None, :] == 0))
    l1 = _logsumexp_masked(lp, match & (bj[None, :] == 1))
    with np.errstate(invalid="ignore"):
        llr = l0 - l1
    llr = np.where(np.isnan(llr), 0.0, llr)
    return np.clip(llr, -clip, clip)


def slice_llr_soft(x, lower_post, j: int, m: int, lo: float, hi: float, sigma_n: float,
                   label: str = "gray", clip: float = LLR_CLIP) -> np.ndarray:
    """Channel LLR of slice j with the lower slices known only softly (Sec. III-B
    step 4 and its footnote: the soft decoding output of the lower slices gives
    a-priori reliabilities).

    L_j(i) = ln sum_{k: b_j(k)=0} P(k|x_i) w_k(i) - ln sum_{k: b_j(k)=1} P(k|x_i) w_k(i),
    w_k(i) = prod_{l<j} P(b_l = bit l of label(k) | L_l(i)),
    P(b = 0 | L) = 1 / (1 + e^-L), P(b = 1 | L) = 1 / (1 + e^L).
    lower_post: float [j][count] LLRs of the lower slices (+-inf = known bit).
    With every |L_l| infinite this is `slice_llr` with those bits.
    """
    x = np.asarray(x, dtype=np.float64).ravel()
    lp = interval_logprob(x, m, lo, hi, sigma_n)
    lab = labels(m, label)
    logw = np.zeros_like(lp)
    for l in range(j):
        L = np.asarray(lower_post[l], dtype=np.float64).ravel()[:, None]
        bit = ((lab >> l) & 1)[None, :]
        # log P(b_l = bit | L) = -log(1 + e^{-L}) for bit 0, -log(1 + e^{L}) for bit 1
        z = np.where(bit == 0, L, -L)
        with np.errstate(invalid="ignore"):
            logw += -np.logaddexp(0.0, -z)
    lw = lp + logw
    bj = (lab >> j) & 1
    l0 = _logsumexp_masked(lw, np.broadcast_to(bj[None, :] == 0, lw.shape))
    l1 = _logsumexp_masked(lw, np.broadcast_to(bj[None, :] == 1, lw.shape))
    with np.errstate(invalid="ignore"):
        llr = l0 - l1
    llr = np.where(np.isnan(llr), 0.0, llr)
    return np.clip(llr, -clip, clip)


# --------------------------------------------------- capacities and code rates
def _cond_entropy_integrand(x, m, lo, hi, sigma_n, lab, j):
    """sum_low P(low|x) h2(P(b_j = 1 | x, low)) in bits, vectorised over x."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    P = np.exp(interval_logprob(x, m, lo, hi, sigma_n))
    lowmask = (1 << j) - 1
    bj = (lab >> j) & 1
    H = np.zeros(x.shape[0])
    for low in range(1 << j):
        sel = (lab & lowmask) == low
        P0 = P[:, sel & (bj == 0)].sum(axis=1)
        P1 = P[:, sel & (bj == 1)].sum(axis=1)
        S = P0 + P1
        with np.errstate(divide="ignore", invalid="ignore"):
            t0 = np.where(P0 > 0, -P0 * np.log2(P0 / S), 0.0)
            t1 = np.where(P1 > 0, -P1 * np.log2(P1 / S), 0.0)
        H += np.nan_to_num(t0) + np.nan_to_num(t1)
    return H


def _gauss(x, va):
    return np.exp(-x * x / (2.0 * va)) / np.sqrt(2.0 * np.pi * va)


def slice_cond_entropy(snr: float, m: int, j: int, label: str = "gray", va: float = 1.0,
                       method: str = "simpson") -> float:
    """H(B_j | X, B_0..B_{j-1}) in bits, x ~ N(0, V_A), by numerical integration.

    method "simpson": composite Simpson's rule, 20001 points on [-12, 12] sigma_x;
    method "quad": scipy adaptive Gauss-Kronrod on the same interval.
    """
    lo, hi = quantiser_range(snr, va)
    sn = 1.0 / np.sqrt(snr)
    lab = labels(m, label)
    L = 12.0 * np.sqrt(va)
    if method == "simpson":
        xs = np.linspace(-L, L, 20001)
        f = _gauss(xs, va) * _cond_entropy_integrand(xs, m, lo, hi, sn, lab, j)
        return float(integrate.simpson(f, x=xs))
    if method == "quad":
        g = lambda s: float(_gauss(s, va) * _cond_entropy_integrand(s, m, lo, hi, sn, lab, j)[0])
        v, _ = integrate.quad(g, -L, L, limit=400, epsabs=1e-13, epsrel=1e-12,
                              points=list(np.concatenate([[lo], thresholds(m, lo, hi), [hi]])))
        return float(v)
    raise ValueError(method)


def slice_capacity(snr: float, m: int, j: int, label: str = "gray", va: float = 1.0,
                   method: str = "simpson") -> float:
    """Conditional capacity C_j = 1 - H(B_j | X, B_{<j}) of slice j (bits per sample)."""
    return 1.0 - slice_cond_entropy(snr, m, j, label, va, method)


def total_cond_entropy(snr: float, m: int, va: float = 1.0) -> float:
    """H(K | X) in bits computed directly from the interval distribution (no slicing)."""
    lo, hi = quantiser_range(snr, va)
    sn = 1.0 / np.sqrt(snr)
    xs = np.linspace(-12.0 * np.sqrt(va), 12.0 * np.sqrt(va), 20001)
    P = np.exp(interval_logprob(xs, m, lo, hi, sn))
    with np.errstate(divide="ignore", invalid="ignore"):
        h = np.where(P > 0, -P * np.log2(P), 0.0).sum(axis=1)
    return float(integrate.simpson(_gauss(xs, va) * h, x=xs))


def label_entropy(snr: float, m: int, va: float = 1.0) -> float:
    """H(K) = Pi(M(Y)) per sample: entropy of Bob's quantised value, y ~ N(0, V_A + 1/SNR)."""
    lo, hi = quantiser_range(snr, va)
    sy = np.sqrt(va + 1.0 / snr)
    t = np.concatenate([[-np.inf], thresholds(m, lo, hi), [np.inf]])
    P = ndtr(t[1:] / sy) - ndtr(t[:-1] / sy)
    P = P[P > 0]
    return float(-(P * np.log2(P)).sum())


def code_rate(capacity: float, fraction: float = 0.95, denom: int = 64) -> float:
    """Rate rule: r = fraction * C rounded to the nearest 1/denom (ties up), capped at
    (denom-1)/denom; r <= 0 means the slice is disclosed (returned as 0.0)."""
    k = int(np.floor(fraction * capacity * denom + 0.5))
    k = min(k, denom - 1)
    return max(k, 0) / denom


# ------------------------------------------------------------- syndrome (a2)
def syndrome(row_ptr, col_idx, bits) -> np.ndarray:
    """s_c = XOR of the bits on check c, per frame.  bits uint8 [F][n] -> uint8 [F][M]."""
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    b = np.asarray(bits, dtype=np.uint8)
    M = rp.shape[0] - 1
    out = np.zeros((b.shape[0], M), dtype=np.uint8)
    for c in range(M):
        cols = ci[rp[c]:rp[c + 1]]
        out[:, c] = np.bitwise_xor.reduce(b[:, cols], axis=1) if cols.size else 0
    return out


# ------------------------------------------------------------ layer partition
def greedy_layers(row_ptr, col_idx, n: int):
    """Greedy first-fit colouring of checks in index order.

    Check c joins the lowest layer that holds none of its variables.  Returns
    (layer_of_check int32 [M], layer_ptr int32 [L+1], layer_checks int32 [M]),
    layer_checks listing each layer's checks in increasing index order.
    """
    rp = np.asarray(row_ptr, dtype=np.int64)
    ci = np.asarray(col_idx, dtype=np.int64)
    M = rp.shape[0] - 1
    used = [set() for _ in range(n)]
    layer_of = np.zeros(M, dtype=np.int32)
    for c in range(M):
        vs = ci[rp[c]:rp[c + 1]]
        taken = set()
        for v in vs:
            taken |= used[v]
        lay = 0
        while lay in taken:
            lay += 1
        layer_of[c] = lay
        for v in vs:
            used[v].add(lay)
    n_layers = int(layer_of.max()) + 1 if M else 0
    order = np.argsort(layer_of, kind="stable").astype(np.int32)
    counts = np.bincount(layer_of, minlength=n_layers)
    layer_ptr = np.zeros(n_layers + 1, dtype=np.int32)
    np.cumsum(counts, out=layer_ptr[1:])
    return layer_of, layer_ptr, order


# --------------------------------------------------------------- decoders (a4-a5)
def _prep(row_ptr, col_idx, llr, synd):
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    llr = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    synd = np.ascontiguousarray(np.atleast_2d(synd), dtype=np.uint8)
    F, n = llr.shape
    M = rp.shape[0] - 1
    if synd.shape != (F, M):
        raise ValueError("syndrome shape")
    bits = np.zeros((F, n), dtype=np.uint8)
    iters = np.zeros(F, dtype=np.int32)
    conv = np.zeros(F, dtype=np.uint8)
    post = np.zeros((F, n), dtype=np.float64)
    return rp, ci, llr, synd, F, n, M, bits, iters, conv, post


def decode(row_ptr, col_idx, llr, synd, algo: str = "sp_flood", max_iter: int = 50,
           early_stop: bool = True, offset: float = 0.5, llr_step: float = 0.5,
           layers=None):
    """Decode F frames sharing one parity-check matrix.

    algo: "sp_flood" | "oms_flood" | "oms_layered" | "ioms_flood" | "ioms_layered".
    Returns dict(bits uint8 [F][n], iters int32 [F], converged uint8 [F],
    post float64 [F][n]).  For the integer decoders post = integer posterior * llr_step.
    """
    rp, ci, llr, synd, F, n, M, bits, iters, conv, post = _prep(row_ptr, col_idx, llr, synd)
    lib = _lib()
    es = 1 if early_stop else 0
    if F == 0:
        return dict(bits=bits, iters=iters, converged=conv, post=post)
    P = lambda a: a.ctypes.data
    if algo in ("oms_layered", "ioms_layered"):
        if layers is None:
            layers = greedy_layers(rp, ci, n)
        _, lptr, lchk = layers
        lptr = np.ascontiguousarray(lptr, dtype=np.int32)
        lchk = np.ascontiguousarray(lchk, dtype=np.int32)
    if algo == "sp_flood":
        rc = lib.oracle_sp_flood(n, M, P(rp), P(ci), P(llr), P(synd), F, max_iter, es,
                                 P(bits), P(iters), P(conv), P(post))
    elif algo == "oms_flood":
        rc = lib.oracle_oms_flood(n, M, P(rp), P(ci), P(llr), P(synd), F, max_iter, float(offset),
                                  es, P(bits), P(iters), P(conv), P(post))
    elif algo == "oms_layered":
        rc = lib.oracle_oms_layered(n, M, P(rp), P(ci), lptr.shape[0] - 1, P(lptr), P(lchk),
                                    P(llr), P(synd), F, max_iter, float(offset), es,
                                    P(bits), P(iters), P(conv), P(post))
    elif algo in ("ioms_flood", "ioms_layered"):
        lay = algo == "ioms_layered"
        nl = lptr.shape[0] - 1 if lay else 0
        lp_ = P(lptr) if lay else None
        lc_ = P(lchk) if lay else None
        rc = lib.oracle_ioms(1 if lay else 0, n, M, P(rp), P(ci), nl, lp_, lc_, P(llr), P(synd), F,
                             max_iter, float(llr_step), es, P(bits), P(iters), P(conv), P(post))
    else:
        raise ValueError(algo)
    if rc != 0:
        raise MemoryError("oracle decoder allocation")
    return dict(bits=bits, iters=iters, converged=conv, post=post)


def decode_bound(row_ptr, col_idx, llr, synd, algo: str, iters: int, f16: bool = True, offset: float = 0.5,
                 phi_rel: float = 4e-6, layers=None):
    """Posteriors after exactly `iters` iterations (no stopping test) with a forward
    error radius per posterior (bound.c): (post float64 [F][n], radius float64 [F][n]).

    post is the FP64 result of decode(..., max_iter=iters, early_stop=False); radius
    bounds |L~ - L| for a decoder that runs the same rules in FP32 with the edge
    messages stored in binary16 (f16=True) or binary32 (f16=False) and, for
    sum-product, evaluates phi to a relative error of at most phi_rel.
    algo: "sp_flood" | "oms_flood" | "oms_layered"."""
    rp, ci, llr, synd, F, n, M, _, _, _, post = _prep(row_ptr, col_idx, llr, synd)
    rad = np.zeros_like(post)
    a = {"sp_flood": 0, "oms_flood": 1, "oms_layered": 2}[algo]
    lptr = lchk = None
    nl = 0
    if a == 2:
        if layers is None:
            layers = greedy_layers(rp, ci, n)
        _, lptr, lchk = layers
        lptr = np.ascontiguousarray(lptr, dtype=np.int32)
        lchk = np.ascontiguousarray(lchk, dtype=np.int32)
        nl = lptr.shape[0] - 1
    if F == 0:
        return post, rad
    P = lambda x: x.ctypes.data if x is not None else None
    rc = _lib().oracle_lowp_bound(a, 1 if f16 else 0, n, M, P(rp), P(ci), nl, P(lptr), P(lchk), P(llr),
                                  P(synd), F, int(iters), float(offset), float(phi_rel), P(post), P(rad))
    if rc != 0:
        raise MemoryError("oracle bound allocation")
    return post, rad


# ------------------------------------------------ weighted min-sum and gradient (a7)
def woms(row_ptr, col_idx, llr, synd, target, alpha, beta, want_post: bool = False):
    """Unrolled weighted offset min-sum (flooding, T = len(alpha) iterations) and the
    reverse-mode gradient of the mean binary cross-entropy loss -- see bp.c.

    alpha, beta: [T][2] (degree class 0 = the code's smallest check degree).
    Returns dict(loss float, galpha [T][2], gbeta [T][2], post [F][n] or None).
    """
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    llr = np.ascontiguousarray(np.atleast_2d(llr), dtype=np.float64)
    synd = np.ascontiguousarray(np.atleast_2d(synd), dtype=np.uint8)
    tgt = np.ascontiguousarray(np.atleast_2d(target), dtype=np.uint8)
    a = np.ascontiguousarray(alpha, dtype=np.float64).reshape(-1, 2)
    b = np.ascontiguousarray(beta, dtype=np.float64).reshape(-1, 2)
    T = a.shape[0]
    F, n = llr.shape
    M = rp.shape[0] - 1
    ga = np.zeros((T, 2))
    gb = np.zeros((T, 2))
    post = np.zeros((F, n)) if want_post else None
    loss = ctypes.c_double()
    P = lambda x: x.ctypes.data if x is not None else None
    rc = _lib().oracle_woms(n, M, P(rp), P(ci), P(llr), P(synd), P(tgt), F, T, P(a), P(b),
                            ctypes.byref(loss), P(ga), P(gb), P(post))
    if rc != 0:
        raise MemoryError("oracle woms allocation")
    return dict(loss=loss.value, galpha=ga, gbeta=gb, post=post)
