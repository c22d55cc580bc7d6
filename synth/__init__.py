"""Seeded synthetic inputs for CV-QKD slice reconciliation.

This module only MAKES INPUTS; it holds none of the reconciliation arithmetic
(no quantiser, no likelihoods, no decoding).  Both the FP64 oracle and the
CUDA library consume what it returns, so it is the one piece they share.

* Quadratures (Sec. V, "Decoding Error and Time" set-up): Alice's
  x_i ~ N(0, V_A) with V_A = 1, Bob's y_i = x_i + n_i, n_i ~ N(0, sigma_n^2),
  sigma_n^2 = 1/SNR.  Normal draws come from numpy's Philox-4x32-10
  counter-based generator (Salmon et al., SC'11), x from key (seed, 0) and the
  noise from key (seed, 1).  Both arrays are returned as float32 (y is rounded
  once, after the FP64 addition).
* Parity-check matrices: random left-regular LDPC codes (variable degree dv,
  check degrees floor/ceil of dv*n/M), placed by a Philox-drawn socket
  permutation, with double edges and 4-cycles broken by seeded socket swaps
  (C helper in _codegen.c).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = None
_LOCK = threading.Lock()


def _lib():
    """Compile (once, with gcc) and load the socket-swap helper."""
    global _LIB
    with _LOCK:
        if _LIB is not None:
            return _LIB
        src = os.path.join(_HERE, "_codegen.c")
        so = os.path.join(_BUILD, "libsynth_codegen.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            os.makedirs(_BUILD, exist_ok=True)
            tmp = so + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", src, "-o", tmp])
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        lib.synth_break_short_cycles.restype = ctypes.c_int64
        lib.synth_break_short_cycles.argtypes = [
            ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
            ctypes.c_uint64, ctypes.c_int32]
        lib.synth_philox_permutation.restype = None
        lib.synth_philox_permutation.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p]
        lib.synth_make_regular_code.restype = ctypes.c_int64
        lib.synth_make_regular_code.argtypes = [
            ctypes.c_uint64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
            ctypes.c_void_p, ctypes.c_void_p]
        _LIB = lib
        return lib


def build() -> None:
    _lib()


def philox(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(key=int(seed)))


def gaussian_pair(seed: int, count: int, snr: float, va: float = 1.0):
    """(x, y) float32 arrays of length `count`: x ~ N(0, va), y = x + N(0, 1/snr).

    x and the noise come from two Philox streams (keys (seed, 0) and (seed, 1)),
    so the first k samples do not depend on `count`: any prefix of a long
    block can be regenerated on its own.
    """
    gx = np.random.Generator(np.random.Philox(key=[int(seed), 0]))
    gn = np.random.Generator(np.random.Philox(key=[int(seed), 1]))
    x = gx.standard_normal(count) * np.sqrt(va)
    noise = gn.standard_normal(count) * np.sqrt(1.0 / snr)
    y = x + noise
    return x.astype(np.float32), y.astype(np.float32)


def uneven_frames(seed: int, count: int, lengths=(4096, 16384, 65536), snr_range=(2.0, 15.0),
                  snr_step: float | None = None):
    """Frame lengths drawn uniformly from `lengths` and SNRs uniformly from
    `snr_range` (Philox key (seed, 2)); with `snr_step` the SNR is drawn uniformly
    from the grid lo, lo + step, ..., hi instead.  Returns (n int64 [count],
    snr float64 [count])."""
    g = np.random.Generator(np.random.Philox(key=[int(seed), 2]))
    n = np.asarray(lengths, dtype=np.int64)[g.integers(0, len(lengths), size=count)]
    if snr_step:
        k = int(round((snr_range[1] - snr_range[0]) / snr_step))
        snr = snr_range[0] + snr_step * g.integers(0, k + 1, size=count)
    else:
        snr = g.uniform(snr_range[0], snr_range[1], size=count)
    return n, snr


def gaussian_frames(seed: int, lengths, snrs, va: float = 1.0):
    """Concatenated (x, y) float32 of frames with their own SNR: x ~ N(0, va) from key
    (seed, 0), noise N(0, 1/snr_f) from key (seed, 1) scaled per frame."""
    lengths = np.asarray(lengths, dtype=np.int64)
    total = int(lengths.sum())
    gx = np.random.Generator(np.random.Philox(key=[int(seed), 0]))
    gn = np.random.Generator(np.random.Philox(key=[int(seed), 1]))
    x = gx.standard_normal(total) * np.sqrt(va)
    scale = np.repeat(1.0 / np.sqrt(np.asarray(snrs, dtype=np.float64)), lengths)
    y = x + gn.standard_normal(total) * scale
    return x.astype(np.float32), y.astype(np.float32)


def checks_for_rate(n: int, rate: float) -> int:
    """Number of parity checks M = n (1 - r) of a rate-r code of length n."""
    m = int(round(n * (1.0 - rate)))
    if m <= 0 or m > n:
        raise ValueError(f"rate {rate} gives {m} checks for n={n}")
    return m


def make_regular_code(seed: int, n: int, m_checks: int, dv: int = 3, max_passes: int = 100):
    """Left-regular parity-check matrix in CSR form.

    Returns (row_ptr int32[M+1], col_idx int32[E], residual) where E = dv*n and
    `residual` counts the 4-cycle / double-edge detections left after the swap
    passes (0 means girth >= 6).  Deterministic in `seed`.
    """
    n, M = int(n), int(m_checks)
    E = dv * n
    if M <= 0 or M > E:
        raise ValueError("bad check count")
    d_lo = E // M
    n_hi = E - M * d_lo
    deg = np.full(M, d_lo, dtype=np.int64)
    deg[:n_hi] += 1
    row_ptr = np.zeros(M + 1, dtype=np.int32)
    np.cumsum(deg, out=row_ptr[1:])
    sockets = np.repeat(np.arange(n, dtype=np.int32), dv)
    perm = philox(seed).permutation(E)
    col_idx = np.ascontiguousarray(sockets[perm], dtype=np.int32)
    residual = _lib().synth_break_short_cycles(
        n, M, row_ptr.ctypes.data, col_idx.ctypes.data,
        ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(max_passes))
    if residual < 0:
        raise MemoryError("code construction")
    return row_ptr, col_idx, int(residual)


def philox_permutation_c(seed: int, count: int) -> np.ndarray:
    """The C helper's Philox-4x64-10 permutation of 0..count-1 (the same draws as
    numpy's Generator(Philox(key=seed)).permutation(count))."""
    out = np.empty(int(count), dtype=np.int32)
    _lib().synth_philox_permutation(ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), int(count), out.ctypes.data)
    return out


def make_regular_code_c(seed: int, n: int, m_checks: int, dv: int = 3, max_passes: int = 100):
    """make_regular_code done entirely by the C helper (permutation included)."""
    n, M = int(n), int(m_checks)
    row_ptr = np.zeros(M + 1, dtype=np.int32)
    col_idx = np.zeros(dv * n, dtype=np.int32)
    residual = _lib().synth_make_regular_code(ctypes.c_uint64(int(seed) & 0xFFFFFFFFFFFFFFFF), n, M, int(dv),
                                              int(max_passes), row_ptr.ctypes.data, col_idx.ctypes.data)
    if residual < 0:
        raise ValueError("code construction failed (sizes or memory)")
    return row_ptr, col_idx, int(residual)


def make_qc_code(seed: int, Z: int, nb: int, mb: int = 3, max_tries: int = 10000):
    """Quasi-cyclic parity-check matrix: an mb x nb base matrix with every entry
    a Z x Z circulant permutation P^s (shift s drawn from Philox key (seed, 3)),
    so every variable has degree mb and every check degree nb; n = nb Z,
    M = mb Z.  Shifts are redrawn until no 4-cycle remains
    (s_ij - s_ik + s_lk - s_lj != 0 mod Z for all row pairs i, l and column
    pairs j, k), at most `max_tries` redraws.
    Check c = i Z + z (base row i) has its edges in base-column order: edge
    k goes to variable k Z + (z + s_ik) mod Z.
    Returns (row_ptr int32[M+1], col_idx int32[E], shifts int32[mb][nb], residual
    4-cycle count)."""
    g = np.random.Generator(np.random.Philox(key=[int(seed), 3]))
    S = g.integers(0, Z, size=(mb, nb)).astype(np.int64)

    def cycles(S):
        bad = []
        for i in range(mb):
            for l in range(i + 1, mb):
                d = (S[i] - S[l]) % Z                 # s_ij - s_lj per column j
                for j in range(nb):
                    for k in range(j + 1, nb):
                        if d[j] == d[k]:
                            bad.append((i, j))
        return bad

    for _ in range(max_tries):
        bad = cycles(S)
        if not bad:
            break
        i, j = bad[int(g.integers(0, len(bad)))]
        S[i, j] = g.integers(0, Z)
    residual = len(cycles(S))
    M, E = mb * Z, mb * Z * nb
    row_ptr = (np.arange(M + 1, dtype=np.int64) * nb).astype(np.int32)
    z = np.arange(Z, dtype=np.int64)
    col = np.empty((mb, Z, nb), dtype=np.int64)
    for i in range(mb):
        for k in range(nb):
            col[i, :, k] = k * Z + (z + S[i, k]) % Z
    return row_ptr, col.reshape(E).astype(np.int32), S.astype(np.int32), residual


def degrees(row_ptr, col_idx, n):
    """(column degrees, row degrees) of a CSR parity-check matrix."""
    cols = np.bincount(col_idx, minlength=n)
    rows = np.diff(row_ptr)
    return cols, rows
