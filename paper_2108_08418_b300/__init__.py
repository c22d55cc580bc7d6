"""Python binding of libqkdrec (CV-QKD slice reconciliation hot path on B300).

Thin layer over the C ABI in include/qkdrec.h: every function below has the
name of the C entry point it calls, checks and marshals its torch arguments,
allocates outputs (and the decoder workspace) through torch, and passes
torch's current CUDA stream.  All arithmetic of the path runs in the CUDA
kernels of libqkdrec.so; there is no CPU fallback -- if the library cannot be
loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libqkdrec.so")

# C enums (include/qkdrec.h)
OK, ERR_ARG, ERR_CSR, ERR_CUDA, ERR_NOMEM, ERR_TIMEOUT, ERR_UNSUPPORTED = range(7)
SP_FLOOD, OMS_FLOOD, OMS_LAYERED = 0, 1, 2
F32, F16MSG, I8SAT = 0, 1, 2
LABEL_GRAY, LABEL_BINARY = 0, 1
_LABELS = {"gray": LABEL_GRAY, "binary": LABEL_BINARY}
_ALGOS = {"sp_flood": SP_FLOOD, "oms_flood": OMS_FLOOD, "oms_layered": OMS_LAYERED}
_PRECS = {"f32": F32, "f16": F16MSG, "i8": I8SAT}

EXPORTED = [
    "qkdrec_code_create", "qkdrec_code_destroy", "qkdrec_code_info", "qkdrec_code_layers",
    "qkdrec_quantise_slices", "qkdrec_slice_llr", "qkdrec_syndrome",
    "qkdrec_decode_opts_default", "qkdrec_decode_workspace_size", "qkdrec_decode_batch",
    "qkdrec_slice_capacity", "qkdrec_last_error", "qkdrec_version",
    "qkdrec_profile_begin", "qkdrec_profile_end",
    "qkdrec_decode_static_capacity", "qkdrec_decode_batch_static",
    "qkdrec_woms_workspace_size", "qkdrec_woms_forward", "qkdrec_woms_backward",
    "qkdrec_quantise_slices_frames", "qkdrec_slice_llr_frames", "qkdrec_tuning_default",
    "qkdrec_plan_create", "qkdrec_plan_destroy", "qkdrec_plan_workspace_size", "qkdrec_plan_launch",
    "qkdrec_plan_get_tuning", "qkdrec_plan_autotune", "qkdrec_slice_llr_soft", "qkdrec_bits_to_llr",
    "qkdrec_code_set_qc", "qkdrec_qc_timeouts",
    "qkdrec_make_regular_code", "qkdrec_free", "qkdrec_code_rate", "qkdrec_checks_for_rate",
    "qkdrec_quantiser_range", "qkdrec_reconcile", "qkdrec_reconcile_workspace_size",
    "qkdrec_reconcile_workspace_size_limited", "qkdrec_pack_bits",
    "qkdrec_unpack_bits", "qkdrec_reconciliation_efficiency", "qkdrec_nr_optimise", "qkdrec_nr_key_rate",
]
SELFTEST = ["qkdrec_selftest_phi", "qkdrec_selftest_phi_pair", "qkdrec_selftest_gauss_tail"]


class QkdrecError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qkdrec status {status}: {msg}")
        self.status = status


class KernelStatC(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("ms", ctypes.c_double),
                ("units", ctypes.c_double), ("bytes", ctypes.c_double)]


class GroupC(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("frames", ctypes.c_int32), ("llr", ctypes.c_void_p),
                ("synd", ctypes.c_void_p), ("bits_out", ctypes.c_void_p), ("iters_out", ctypes.c_void_p),
                ("conv_out", ctypes.c_void_p)]


class TuningC(ctypes.Structure):
    _fields_ = [("frames_per_tile", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("stage_depth", ctypes.c_int32), ("ctas_per_tile", ctypes.c_int32),
                ("tiles_per_item", ctypes.c_int32), ("frames_per_lane", ctypes.c_int32),
                ("sparse_frames", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class PointC(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("codes", ctypes.c_void_p), ("alice_packed", ctypes.c_void_p),
                ("converged", ctypes.c_void_p), ("iters", ctypes.c_void_p)]


class NrParamsC(ctypes.Structure):
    _fields_ = [("n_signals", ctypes.c_double), ("m_slices", ctypes.c_int32), ("eps_ec", ctypes.c_double),
                ("eps_s", ctypes.c_double), ("eps_pa", ctypes.c_double), ("eps_pe", ctypes.c_double),
                ("va", ctypes.c_double), ("transmissivity", ctypes.c_double), ("xi_ch", ctypes.c_double),
                ("xi_d", ctypes.c_double), ("eta_d", ctypes.c_double), ("n_estimation", ctypes.c_double),
                ("c_h", ctypes.c_double), ("edges_per_sample", ctypes.c_void_p), ("iterations", ctypes.c_void_p),
                ("dispersion_form", ctypes.c_int32), ("nr_min", ctypes.c_double)]


class NrResultC(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("snr", "i_ab", "dispersion", "qinv_ec", "delta_aep", "s_be", "t_low",
                                               "xi_up", "b1", "b2", "nr_stationary", "nr_opt", "key_rate_opt",
                                               "d2_key_rate")] + [("at_boundary", ctypes.c_int32)]


class DecodeOptsC(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("prec", ctypes.c_int32), ("max_iter", ctypes.c_int32),
                ("offset", ctypes.c_float), ("llr_step", ctypes.c_float), ("early_stop", ctypes.c_int32),
                ("fallback_f32", ctypes.c_int32)]


_LIB = None


def lib():
    """Load libqkdrec.so (built by paper_2108_08418_b300.build); raises if absent."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libqkdrec.so not built ({LIB_PATH}); run python -m paper_2108_08418_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U64, D, U = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                              ctypes.c_double, ctypes.c_int)
    sig = {
        "qkdrec_code_create": (U, [I32, I32, P, P, U64, P]),
        "qkdrec_code_destroy": (None, [P]),
        "qkdrec_code_info": (U, [P, P, P, P, P, P]),
        "qkdrec_code_layers": (U, [P, P]),
        "qkdrec_quantise_slices": (U, [P, I64, I32, D, D, U, P, P, P]),
        "qkdrec_slice_llr": (U, [P, I64, I32, I32, D, D, D, U, P, P, P]),
        "qkdrec_slice_llr_soft": (U, [P, I64, I32, I32, D, D, D, U, P, P, P]),
        "qkdrec_bits_to_llr": (U, [P, I64, P, P]),
        "qkdrec_code_set_qc": (U, [P, I32, I32, I32, P, I32]),
        "qkdrec_qc_timeouts": (U, [P]),
        "qkdrec_syndrome": (U, [P, P, I32, P, P]),
        "qkdrec_decode_opts_default": (None, [P]),
        "qkdrec_decode_workspace_size": (U, [P, I32, P, P]),
        "qkdrec_decode_batch": (U, [P, P, P, I32, P, P, P, P, P, P, ctypes.c_size_t, P]),
        "qkdrec_slice_capacity": (U, [D, I32, I32, D, D, U, D, P]),
        "qkdrec_make_regular_code": (U, [U64, I32, I32, I32, P, P, P]),
        "qkdrec_free": (None, [P]),
        "qkdrec_reconcile_workspace_size": (U, [I64, I32, P, P, I32, P]),
        "qkdrec_reconcile_workspace_size_limited": (U, [I64, I32, P, P, I32, I32, P]),
        "qkdrec_reconcile": (U, [P, P, I64, I32, D, D, D, U, P, P, I32, P, P, ctypes.c_size_t, P]),
        "qkdrec_pack_bits": (U, [P, I64, P, P]),
        "qkdrec_unpack_bits": (U, [P, I64, P, P]),
        "qkdrec_code_rate": (U, [D, D, I32, P]),
        "qkdrec_checks_for_rate": (U, [I32, D, P]),
        "qkdrec_quantiser_range": (U, [D, D, P, P]),
        "qkdrec_reconciliation_efficiency": (U, [D, I32, D, D, D, P, P, P]),
        "qkdrec_nr_optimise": (U, [P, P]),
        "qkdrec_nr_key_rate": (U, [P, D, P]),
        "qkdrec_decode_static_capacity": (ctypes.c_size_t, []),
        "qkdrec_decode_batch_static": (U, [P, P, P, I32, P, P, P, P, P, P]),
        "qkdrec_woms_workspace_size": (U, [P, I32, I32, I32, P]),
        "qkdrec_woms_forward": (U, [P, P, P, P, I32, I32, P, P, I32, P, P, P, ctypes.c_size_t, P]),
        "qkdrec_woms_backward": (U, [P, P, P, P, I32, I32, P, P, I32, P, P, P, ctypes.c_size_t, P]),
        "qkdrec_quantise_slices_frames": (U, [P, I64, P, P, I32, I32, U, P, P, P]),
        "qkdrec_slice_llr_frames": (U, [P, I64, P, P, I32, I32, I32, U, P, P, P]),
        "qkdrec_tuning_default": (None, [P]),
        "qkdrec_plan_create": (U, [P, I32, P, P, P]),
        "qkdrec_plan_destroy": (None, [P]),
        "qkdrec_plan_workspace_size": (U, [P, P]),
        "qkdrec_plan_launch": (U, [P, P, ctypes.c_size_t, P]),
        "qkdrec_plan_get_tuning": (U, [P, P]),
        "qkdrec_plan_autotune": (U, [P, P, ctypes.c_size_t, I32, P, P, P]),
        "qkdrec_profile_begin": (U, []),
        "qkdrec_selftest_phi": (U, [P, I64, P, P]),
        "qkdrec_selftest_phi_pair": (U, [P, I64, P, P]),
        "qkdrec_selftest_gauss_tail": (U, [P, I64, P, P]),
        "qkdrec_profile_end": (U, [P, I32, P]),
        "qkdrec_last_error": (ctypes.c_char_p, []),
        "qkdrec_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def _check(status):
    if status != OK:
        raise QkdrecError(status, lib().qkdrec_last_error().decode())


def version() -> str:
    return lib().qkdrec_version().decode()


def _torch():
    import torch
    return torch


def _stream(t):
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream(t.device).cuda_stream)


def _dev(t, dtype, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------- codes
class Code:
    """Parity-check matrix H (M x n) in CSR form with its device copies."""

    def __init__(self, n: int, row_ptr, col_idx, seed: int = 0, device=None):
        torch = _torch()
        rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(col_idx, dtype=np.int32)
        self._h = ctypes.c_void_p()
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        with torch.cuda.device(dev):
            _check(lib().qkdrec_code_create(int(n), rp.shape[0] - 1, rp.ctypes.data, ci.ctypes.data,
                                            ctypes.c_uint64(int(seed) & (2**64 - 1)), ctypes.byref(self._h)))
        self.device = dev
        n_, m_, e_, l_, d_ = (ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int32(),
                              ctypes.c_int32())
        _check(lib().qkdrec_code_info(self._h, ctypes.byref(n_), ctypes.byref(m_), ctypes.byref(e_),
                                      ctypes.byref(l_), ctypes.byref(d_)))
        self.n, self.M, self.E, self.n_layers, self.dc_max = n_.value, m_.value, e_.value, l_.value, d_.value

    @property
    def handle(self):
        return self._h

    def set_qc(self, Z: int, mb: int, nb: int, shifts, tma: bool = True):
        """Declare the code quasi-cyclic (shifts int [mb][nb]); with `tma` the layered
        FP32 decoder stages posteriors and messages with TMA tile copies."""
        sh = np.ascontiguousarray(shifts, dtype=np.int32).reshape(mb, nb)
        _check(lib().qkdrec_code_set_qc(self._h, int(Z), int(mb), int(nb), sh.ctypes.data, int(bool(tma))))
        self.qc = (int(Z), int(mb), int(nb))

    def layers(self) -> np.ndarray:
        out = np.zeros(self.M, dtype=np.int32)
        _check(lib().qkdrec_code_layers(self._h, out.ctypes.data))
        return out

    def destroy(self):
        if self._h:
            lib().qkdrec_code_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


def qkdrec_qc_timeouts() -> int:
    """Tile-copy waits the quasi-cyclic layer kernel gave up on (0 in normal operation)."""
    c = ctypes.c_int32()
    _check(lib().qkdrec_qc_timeouts(ctypes.byref(c)))
    return c.value


def qkdrec_code_create(n, row_ptr, col_idx, seed=0, device=None) -> Code:
    return Code(n, row_ptr, col_idx, seed, device)


# --------------------------------------------------------------- quantiser
def qkdrec_quantise_slices(y, m_slices: int, lo: float, hi: float, label: str = "gray",
                           want_idx: bool = True, want_bits: bool = True):
    """Interval index uint8 [count] and bit planes uint8 [m][count] of Bob's y (float32 CUDA)."""
    torch = _torch()
    count = y.numel()
    yp = _dev(y, torch.float32, "y")
    idx = torch.empty(count, dtype=torch.uint8, device=y.device) if want_idx else None
    bits = torch.empty((m_slices, count), dtype=torch.uint8, device=y.device) if want_bits else None
    _check(lib().qkdrec_quantise_slices(yp, count, int(m_slices), float(lo), float(hi), _LABELS[label],
                                        ctypes.c_void_p(idx.data_ptr()) if idx is not None else None,
                                        ctypes.c_void_p(bits.data_ptr()) if bits is not None else None,
                                        _stream(y)))
    return idx, bits


def qkdrec_slice_llr(x, m_slices: int, j: int, lo: float, hi: float, sigma_n: float, lower_bits=None,
                     label: str = "gray", out=None):
    """Channel LLR float32 [count] of slice j from Alice's x and reconciled lower bits uint8 [j][count]."""
    torch = _torch()
    count = x.numel()
    xp = _dev(x, torch.float32, "x")
    lb = None
    if j > 0:
        if lower_bits is None or lower_bits.shape[0] < j or lower_bits[0].numel() != count:
            raise ValueError("lower_bits must be uint8 [>= j][count]")
        lb = _dev(lower_bits, torch.uint8, "lower_bits")
    if out is None:
        out = torch.empty(count, dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, "out")
    _check(lib().qkdrec_slice_llr(xp, count, int(m_slices), int(j), float(lo), float(hi), float(sigma_n),
                                  _LABELS[label], lb, op, _stream(x)))
    return out


def qkdrec_slice_llr_soft(x, m_slices: int, j: int, lo: float, hi: float, sigma_n: float, lower_post=None,
                          label: str = "gray", out=None):
    """Channel LLR float32 [count] of slice j with the lower slices known softly:
    lower_post float32 [j][count] LLRs of slices 0..j-1 (+-inf = known bit)."""
    torch = _torch()
    count = x.numel()
    xp = _dev(x, torch.float32, "x")
    lp = None
    if j > 0:
        if lower_post is None or lower_post.shape[0] < j or lower_post[0].numel() != count:
            raise ValueError("lower_post must be float32 [>= j][count]")
        lp = _dev(lower_post, torch.float32, "lower_post")
    if out is None:
        out = torch.empty(count, dtype=torch.float32, device=x.device)
    op = _dev(out, torch.float32, "out")
    _check(lib().qkdrec_slice_llr_soft(xp, count, int(m_slices), int(j), float(lo), float(hi), float(sigma_n),
                                       _LABELS[label], lp, op, _stream(x)))
    return out


def qkdrec_bits_to_llr(bits, out=None):
    """Known bits uint8 [count] as certain LLRs float32 [count] (0 -> +inf, 1 -> -inf)."""
    torch = _torch()
    count = bits.numel()
    bp = _dev(bits, torch.uint8, "bits")
    if out is None:
        out = torch.empty(count, dtype=torch.float32, device=bits.device)
    _check(lib().qkdrec_bits_to_llr(bp, count, _dev(out, torch.float32, "out"), _stream(bits)))
    return out


# ---------------------------------------------------------------- syndrome
def qkdrec_syndrome(code: Code, bits, out=None):
    """Syndromes uint8 [F][M] of bits uint8 [F][n] (into `out` if given)."""
    torch = _torch()
    bits2 = bits.reshape(-1, code.n)
    F = bits2.shape[0]
    bp = _dev(bits2, torch.uint8, "bits")
    if out is None:
        out = torch.empty((F, code.M), dtype=torch.uint8, device=bits.device)
    elif out.numel() != F * code.M:
        raise ValueError("out must be uint8 [F][M]")
    op = _dev(out, torch.uint8, "out")
    _check(lib().qkdrec_syndrome(code.handle, bp, F, op, _stream(bits)))
    return out


# ----------------------------------------------------------------- decoder
@dataclass
class DecodeOpts:
    algo: str = "sp_flood"        # sp_flood | oms_flood | oms_layered
    prec: str = "f32"             # f32 | f16 | i8
    max_iter: int = 50
    offset: float = 0.5
    llr_step: float = 0.5
    early_stop: bool = True
    fallback_f32: bool | str = False    # True / "same": FP32 with the same algorithm; "sp": FP32 sum-product

    def c(self) -> DecodeOptsC:
        return DecodeOptsC(_ALGOS[self.algo], _PRECS[self.prec], int(self.max_iter), float(self.offset),
                           float(self.llr_step), int(bool(self.early_stop)),
                           2 if self.fallback_f32 == "sp" else int(bool(self.fallback_f32)))


def qkdrec_decode_workspace_size(code: Code, F: int, opts: DecodeOpts) -> int:
    o = opts.c()
    b = ctypes.c_size_t()
    _check(lib().qkdrec_decode_workspace_size(code.handle, int(F), ctypes.byref(o), ctypes.byref(b)))
    return b.value


def workspace_for(code: Code, F: int, opts: DecodeOpts, device):
    torch = _torch()
    nbytes = qkdrec_decode_workspace_size(code, F, opts)
    # torch's caching allocator hands out 512-byte aligned blocks
    return torch.empty(max(nbytes, 256), dtype=torch.uint8, device=device)


def qkdrec_decode_batch(code: Code, llr, synd, opts: DecodeOpts | None = None, want_post: bool = False,
                        workspace=None, out=None):
    """Decode F frames: llr float32 [F][n], synd uint8 [F][M] -> dict(bits, iters, converged, post)."""
    torch = _torch()
    opts = opts or DecodeOpts()
    llr2 = llr.reshape(-1, code.n)
    F = llr2.shape[0]
    if synd.numel() != F * code.M:
        raise ValueError("synd must be uint8 [F][M]")
    lp = _dev(llr2, torch.float32, "llr")
    sp = _dev(synd, torch.uint8, "synd")
    dev = llr.device
    if out is None:
        out = dict(bits=torch.empty((F, code.n), dtype=torch.uint8, device=dev),
                   iters=torch.empty(F, dtype=torch.int32, device=dev),
                   converged=torch.empty(F, dtype=torch.uint8, device=dev),
                   post=torch.empty((F, code.n), dtype=torch.float32, device=dev) if want_post else None)
    if workspace is None:
        workspace = workspace_for(code, F, opts, dev)
    o = opts.c()
    post = out.get("post")
    _check(lib().qkdrec_decode_batch(code.handle, lp, sp, F, ctypes.byref(o),
                                     ctypes.c_void_p(out["bits"].data_ptr()),
                                     ctypes.c_void_p(out["iters"].data_ptr()),
                                     ctypes.c_void_p(out["converged"].data_ptr()),
                                     ctypes.c_void_p(post.data_ptr()) if post is not None else None,
                                     ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(llr)))
    return out


def qkdrec_decode_static_capacity() -> int:
    """Bytes of the decoder workspace compiled into the library."""
    return lib().qkdrec_decode_static_capacity()


def qkdrec_decode_batch_static(code: Code, llr, synd, opts: DecodeOpts | None = None, want_post: bool = False,
                               out=None):
    """qkdrec_decode_batch on the library's built-in device workspace (no device
    allocation by the library; outputs are allocated here unless given)."""
    torch = _torch()
    opts = opts or DecodeOpts()
    llr2 = llr.reshape(-1, code.n)
    F = llr2.shape[0]
    if synd.numel() != F * code.M:
        raise ValueError("synd must be uint8 [F][M]")
    lp = _dev(llr2, torch.float32, "llr")
    sp = _dev(synd, torch.uint8, "synd")
    dev = llr.device
    if out is None:
        out = dict(bits=torch.empty((F, code.n), dtype=torch.uint8, device=dev),
                   iters=torch.empty(F, dtype=torch.int32, device=dev),
                   converged=torch.empty(F, dtype=torch.uint8, device=dev),
                   post=torch.empty((F, code.n), dtype=torch.float32, device=dev) if want_post else None)
    o = opts.c()
    post = out.get("post")
    _check(lib().qkdrec_decode_batch_static(code.handle, lp, sp, F, ctypes.byref(o),
                                            ctypes.c_void_p(out["bits"].data_ptr()),
                                            ctypes.c_void_p(out["iters"].data_ptr()),
                                            ctypes.c_void_p(out["converged"].data_ptr()),
                                            ctypes.c_void_p(post.data_ptr()) if post is not None else None,
                                            _stream(llr)))
    return out


# ------------------------------------------------- whole reconciliation of a block
def _ptr(t, dtype, name):
    """Address of a contiguous tensor on the host or a CUDA device (the C side tells them apart)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    return ctypes.c_void_p(t.data_ptr())


class _Points:
    """qkdrec_point array for a list of dicts(n, codes, alice_packed, converged=None, iters=None)."""

    def __init__(self, points, m_slices):
        torch = _torch()
        self.keep = []
        self.arr = (PointC * len(points))()
        for i, p in enumerate(points):
            if len(p["codes"]) != m_slices:
                raise ValueError("one code (or None) per slice")
            codes = (ctypes.c_void_p * m_slices)(*[c.handle.value if c is not None else None for c in p["codes"]])
            self.keep.append(codes)
            conv, its = p.get("converged"), p.get("iters")
            self.arr[i] = PointC(int(p["n"]), ctypes.cast(codes, ctypes.c_void_p).value,
                                 _ptr(p["alice_packed"], torch.uint8, "alice_packed").value,
                                 _ptr(conv, torch.uint8, "converged").value if conv is not None else None,
                                 _ptr(its, torch.int32, "iters").value if its is not None else None)


def qkdrec_reconcile_workspace_size(count: int, m_slices: int, opts: DecodeOpts, points) -> int:
    o = opts.c()
    pts = _Points(points, m_slices)
    b = ctypes.c_size_t()
    _check(lib().qkdrec_reconcile_workspace_size(int(count), int(m_slices), ctypes.byref(o), pts.arr, len(points),
                                                 ctypes.byref(b)))
    return b.value


def qkdrec_reconcile_workspace_size_limited(count: int, m_slices: int, opts: DecodeOpts, points,
                                            max_in_flight: int) -> int:
    """Workspace bytes for at most max_in_flight partitions decoding at once (1: in order)."""
    o = opts.c()
    pts = _Points(points, m_slices)
    b = ctypes.c_size_t()
    _check(lib().qkdrec_reconcile_workspace_size_limited(int(count), int(m_slices), ctypes.byref(o), pts.arr,
                                                         len(points), int(max_in_flight), ctypes.byref(b)))
    return b.value


def qkdrec_reconcile(x, y, m_slices: int, lo: float, hi: float, sigma_n: float, opts: DecodeOpts, points,
                     bob_packed=None, label: str = "gray", workspace=None, device=None):
    """Reverse slice reconciliation of one block (see include/qkdrec.h).  x, y: float32
    [count] on the host (pinned for overlap) or the device; points: dicts with n, codes
    (Code or None per slice), alice_packed uint8 [m][count/8], optional converged uint8
    [m][count/n] and iters int32 [m][count/n], each on the host or the device.  Runs on
    torch's current stream of `device` (default: the current CUDA device)."""
    torch = _torch()
    count = x.numel()
    if y.numel() != count:
        raise ValueError("x and y must have the same length")
    dev = torch.device(device) if device is not None else (x.device if x.is_cuda else
                                                           torch.device("cuda", torch.cuda.current_device()))
    o = opts.c()
    pts = _Points(points, m_slices)
    if workspace is None:
        workspace = torch.empty(max(qkdrec_reconcile_workspace_size(count, m_slices, opts, points), 256),
                                dtype=torch.uint8, device=dev)
    st = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    with torch.cuda.device(dev):
        _check(lib().qkdrec_reconcile(_ptr(x, torch.float32, "x"), _ptr(y, torch.float32, "y"), count,
                                      int(m_slices), float(lo), float(hi), float(sigma_n), _LABELS[label],
                                      ctypes.byref(o), pts.arr, len(points),
                                      _ptr(bob_packed, torch.uint8, "bob_packed") if bob_packed is not None else None,
                                      ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), st))
    return workspace


def qkdrec_pack_bits(bits, out=None):
    """0/1 bytes (CUDA uint8 [count], count % 32 == 0) -> packed uint8 [count/8], bit i%8 of byte i/8."""
    torch = _torch()
    count = bits.numel()
    if out is None:
        out = torch.empty(count // 8, dtype=torch.uint8, device=bits.device)
    _check(lib().qkdrec_pack_bits(_dev(bits, torch.uint8, "bits"), count, _dev(out, torch.uint8, "out"),
                                  _stream(bits)))
    return out


def qkdrec_unpack_bits(packed, count=None, out=None):
    """Inverse of qkdrec_pack_bits."""
    torch = _torch()
    count = packed.numel() * 8 if count is None else int(count)
    if out is None:
        out = torch.empty(count, dtype=torch.uint8, device=packed.device)
    _check(lib().qkdrec_unpack_bits(_dev(packed, torch.uint8, "packed"), count, _dev(out, torch.uint8, "out"),
                                    _stream(packed)))
    return out


# ------------------------------------------------------------ uneven batches
def qkdrec_quantise_slices_frames(y, frame_offsets, frame_ranges, m_slices: int, label: str = "gray",
                                  want_idx: bool = True, bits_out=None):
    """Quantiser with a range per frame: frame_offsets int64 [F+1], frame_ranges float64 [F][2]."""
    torch = _torch()
    count = y.numel()
    F = frame_offsets.numel() - 1
    idx = torch.empty(count, dtype=torch.uint8, device=y.device) if want_idx else None
    bits = bits_out if bits_out is not None else torch.empty((m_slices, count), dtype=torch.uint8, device=y.device)
    if bits.numel() != m_slices * count:
        raise ValueError("bits_out must be uint8 [m][count]")
    _dev(bits, torch.uint8, "bits_out")
    _check(lib().qkdrec_quantise_slices_frames(_dev(y, torch.float32, "y"), count,
                                               _dev(frame_offsets, torch.int64, "frame_offsets"),
                                               _dev(frame_ranges, torch.float64, "frame_ranges"), F,
                                               int(m_slices), _LABELS[label],
                                               ctypes.c_void_p(idx.data_ptr()) if idx is not None else None,
                                               ctypes.c_void_p(bits.data_ptr()), _stream(y)))
    return idx, bits


def qkdrec_slice_llr_frames(x, frame_offsets, frame_params, m_slices: int, j: int, lower_bits=None,
                            label: str = "gray", out=None):
    """Slice LLRs with (lo, hi, sigma_n) per frame: frame_params float64 [F][3]."""
    torch = _torch()
    count = x.numel()
    F = frame_offsets.numel() - 1
    if out is None:
        out = torch.empty(count, dtype=torch.float32, device=x.device)
    lb = _dev(lower_bits, torch.uint8, "lower_bits") if j > 0 else None
    _check(lib().qkdrec_slice_llr_frames(_dev(x, torch.float32, "x"), count,
                                         _dev(frame_offsets, torch.int64, "frame_offsets"),
                                         _dev(frame_params, torch.float64, "frame_params"), F, int(m_slices),
                                         int(j), _LABELS[label], lb, _dev(out, torch.float32, "out"), _stream(x)))
    return out


class Plan:
    """One-launch decode of an uneven batch (groups of frames with their own codes).

    groups: list of dicts with keys code (Code), llr float32 [F][n], synd uint8 [F][M],
    bits uint8 [F][n], iters int32 [F], conv uint8 [F] -- CUDA tensors the plan binds
    (kept alive here; refill them in place between launches)."""

    def __init__(self, groups, opts: DecodeOpts, tuning: dict | None = None):
        torch = _torch()
        self._keep = groups
        arr = (GroupC * max(len(groups), 1))()
        for i, g in enumerate(groups):
            c = g["code"]
            F = g["llr"].numel() // c.n
            arr[i] = GroupC(c.handle.value, F, _dev(g["llr"], torch.float32, "llr").value,
                            _dev(g["synd"], torch.uint8, "synd").value, _dev(g["bits"], torch.uint8, "bits").value,
                            _dev(g["iters"], torch.int32, "iters").value, _dev(g["conv"], torch.uint8, "conv").value)
        o = opts.c()
        t = None
        if tuning is not None:
            d = TuningC()
            lib().qkdrec_tuning_default(ctypes.byref(d))
            t = TuningC(**{**d.as_dict(), **tuning})
        self._h = ctypes.c_void_p()
        _check(lib().qkdrec_plan_create(arr, len(groups), ctypes.byref(o), ctypes.byref(t) if t else None,
                                        ctypes.byref(self._h)))

    def workspace_size(self) -> int:
        b = ctypes.c_size_t()
        _check(lib().qkdrec_plan_workspace_size(self._h, ctypes.byref(b)))
        return b.value

    def workspace(self, device="cuda"):
        return _torch().empty(self.workspace_size(), dtype=_torch().uint8, device=device)

    def launch(self, workspace, stream=None):
        torch = _torch()
        st = stream if stream is not None else torch.cuda.current_stream(workspace.device)
        _check(lib().qkdrec_plan_launch(self._h, ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                        ctypes.c_void_p(st.cuda_stream)))

    def tuning(self) -> dict:
        t = TuningC()
        _check(lib().qkdrec_plan_get_tuning(self._h, ctypes.byref(t)))
        return t.as_dict()

    def autotune(self, workspace, max_iter: int = 10):
        torch = _torch()
        t = TuningC()
        ms = ctypes.c_float()
        _check(lib().qkdrec_plan_autotune(self._h, ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                          int(max_iter), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(t), ctypes.byref(ms)))
        return t.as_dict(), ms.value

    def destroy(self):
        if self._h:
            lib().qkdrec_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------ differentiable weighted min-sum
def qkdrec_woms_workspace_size(code: Code, F: int, T: int, ckpt_every: int) -> int:
    b = ctypes.c_size_t()
    _check(lib().qkdrec_woms_workspace_size(code.handle, int(F), int(T), int(ckpt_every), ctypes.byref(b)))
    return b.value


def _woms_ptrs(code, llr, synd, target, alpha, beta):
    torch = _torch()
    llr2 = llr.reshape(-1, code.n)
    F = llr2.shape[0]
    if synd.numel() != F * code.M or target.numel() != F * code.n:
        raise ValueError("synd must be uint8 [F][M] and target uint8 [F][n]")
    if alpha.shape != beta.shape or alpha.dim() != 2 or alpha.shape[1] != 2:
        raise ValueError("alpha and beta must be float32 [T][2]")
    return (F, alpha.shape[0], _dev(llr2, torch.float32, "llr"), _dev(synd, torch.uint8, "synd"),
            _dev(target, torch.uint8, "target"), _dev(alpha, torch.float32, "alpha"),
            _dev(beta, torch.float32, "beta"))


def qkdrec_woms_forward(code: Code, llr, synd, target, alpha, beta, ckpt_every: int, workspace,
                        want_post: bool = False):
    """Loss (float32 [1]) of the unrolled weighted min-sum; `workspace` keeps the checkpoints."""
    torch = _torch()
    F, T, lp, sp, tp, ap, bp = _woms_ptrs(code, llr, synd, target, alpha, beta)
    loss = torch.empty(1, dtype=torch.float32, device=llr.device)
    post = torch.empty((F, code.n), dtype=torch.float32, device=llr.device) if want_post else None
    _check(lib().qkdrec_woms_forward(code.handle, lp, sp, tp, F, T, ap, bp, int(ckpt_every),
                                     ctypes.c_void_p(loss.data_ptr()),
                                     ctypes.c_void_p(post.data_ptr()) if post is not None else None,
                                     ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(llr)))
    return loss, post


def qkdrec_woms_backward(code: Code, llr, synd, target, alpha, beta, ckpt_every: int, workspace):
    """(d loss / d alpha, d loss / d beta), float32 [T][2] each."""
    torch = _torch()
    F, T, lp, sp, tp, ap, bp = _woms_ptrs(code, llr, synd, target, alpha, beta)
    ga = torch.empty_like(alpha)
    gb = torch.empty_like(beta)
    _check(lib().qkdrec_woms_backward(code.handle, lp, sp, tp, F, T, ap, bp, int(ckpt_every),
                                      ctypes.c_void_p(ga.data_ptr()), ctypes.c_void_p(gb.data_ptr()),
                                      ctypes.c_void_p(workspace.data_ptr()), workspace.numel(), _stream(llr)))
    return ga, gb


# ------------------------------------------------------------ host helpers
def qkdrec_slice_capacity(snr: float, m_slices: int, j: int, lo: float, hi: float, label: str = "gray",
                          va: float = 1.0) -> float:
    c = ctypes.c_double()
    _check(lib().qkdrec_slice_capacity(float(snr), int(m_slices), int(j), float(lo), float(hi), _LABELS[label],
                                       float(va), ctypes.byref(c)))
    return c.value


def qkdrec_quantiser_range(snr: float, va: float = 1.0):
    """[-4 sigma_y, 4 sigma_y], sigma_y^2 = V_A + 1/SNR: the quantiser range the workloads use."""
    lo, hi = ctypes.c_double(), ctypes.c_double()
    _check(lib().qkdrec_quantiser_range(float(snr), float(va), ctypes.byref(lo), ctypes.byref(hi)))
    return lo.value, hi.value


quantiser_range = qkdrec_quantiser_range


def qkdrec_code_rate(capacity: float, fraction: float = 0.95, denom: int = 64) -> float:
    """Rate rule: fraction * capacity rounded to the nearest 1/denom (ties up), at most
    (denom-1)/denom; 0.0 means the slice is disclosed."""
    r = ctypes.c_double()
    _check(lib().qkdrec_code_rate(float(capacity), float(fraction), int(denom), ctypes.byref(r)))
    return r.value


code_rate = qkdrec_code_rate


def qkdrec_reconciliation_efficiency(snr: float, m_slices: int, lo: float, hi: float, rates, va: float = 1.0):
    """(beta, Pi(M(Y))): Eq. beta for slice code rates `rates` (0 = disclosed)."""
    r = np.ascontiguousarray(rates, dtype=np.float64)
    if r.shape != (m_slices,):
        raise ValueError("one rate per slice")
    b, h = ctypes.c_double(), ctypes.c_double()
    _check(lib().qkdrec_reconciliation_efficiency(float(snr), int(m_slices), float(lo), float(hi), float(va),
                                                  r.ctypes.data, ctypes.byref(b), ctypes.byref(h)))
    return b.value, h.value


# the paper's standard CV-QKD settings (Sec. IV-B)
NR_STANDARD = dict(n_signals=1e9, m_slices=5, eps_ec=2.5e-10, eps_s=1.25e-10, eps_pa=2.5e-10, eps_pe=2.5e-10,
                   va=5.0, transmissivity=0.9, xi_ch=0.0186, xi_d=0.0133, eta_d=1.0, n_estimation=0.0,
                   c_h=3.2e-9, dispersion_form=0, nr_min=1e5)


def _nr_params(edges_per_sample, iterations, **kw):
    p = {**NR_STANDARD, **kw}
    g = np.ascontiguousarray(edges_per_sample, dtype=np.float64)
    d = np.ascontiguousarray(iterations, dtype=np.float64)
    if g.shape != (p["m_slices"],) or d.shape != (p["m_slices"],):
        raise ValueError("one edges-per-sample and one iteration count per slice")
    c = NrParamsC(**{k: v for k, v in p.items()}, edges_per_sample=g.ctypes.data, iterations=d.ctypes.data)
    return c, (g, d)


def qkdrec_nr_optimise(edges_per_sample, iterations, **kw) -> dict:
    """Optimum sub-block length (include/qkdrec.h); keyword overrides of NR_STANDARD."""
    c, keep = _nr_params(edges_per_sample, iterations, **kw)
    r = NrResultC()
    _check(lib().qkdrec_nr_optimise(ctypes.byref(c), ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in r._fields_}


def qkdrec_nr_key_rate(nr: float, edges_per_sample, iterations, **kw) -> float:
    c, keep = _nr_params(edges_per_sample, iterations, **kw)
    v = ctypes.c_double()
    _check(lib().qkdrec_nr_key_rate(ctypes.byref(c), float(nr), ctypes.byref(v)))
    return v.value


def qkdrec_checks_for_rate(n: int, rate: float) -> int:
    """Number of checks M = n (1 - rate) of a rate-r code of length n."""
    m = ctypes.c_int32()
    _check(lib().qkdrec_checks_for_rate(int(n), float(rate), ctypes.byref(m)))
    return m.value


def qkdrec_make_regular_code(seed: int, n: int, m_checks: int, dv: int = 3):
    """Seeded left-regular parity-check matrix from the library: (row_ptr int32 [M+1],
    col_idx int32 [dv n], residual 4-cycle detections)."""
    rp, ci, left = ctypes.POINTER(ctypes.c_int32)(), ctypes.POINTER(ctypes.c_int32)(), ctypes.c_int32()
    _check(lib().qkdrec_make_regular_code(ctypes.c_uint64(int(seed) & (2**64 - 1)), int(n), int(m_checks),
                                          int(dv), ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(left)))
    try:
        row_ptr = np.ctypeslib.as_array(rp, shape=(int(m_checks) + 1,)).copy()
        col_idx = np.ctypeslib.as_array(ci, shape=(int(dv) * int(n),)).copy()
    finally:
        lib().qkdrec_free(ctypes.cast(rp, ctypes.c_void_p))
        lib().qkdrec_free(ctypes.cast(ci, ctypes.c_void_p))
    return row_ptr, col_idx, left.value


# ------------------------------------------------------------- measurement
def qkdrec_profile_begin():
    """Start per-kernel-class event timing and work counters (see include/qkdrec.h)."""
    _check(lib().qkdrec_profile_begin())


def qkdrec_profile_end():
    """Stop recording; returns {kernel class: dict(launches, ms, units, bytes)}."""
    arr = (KernelStatC * 64)()
    n = ctypes.c_int32()
    _check(lib().qkdrec_profile_end(arr, 64, ctypes.byref(n)))
    return {arr[i].name.decode(): dict(launches=arr[i].launches, ms=arr[i].ms, units=arr[i].units,
                                       bytes=arr[i].bytes) for i in range(n.value)}


# ---------------------------------------------------------------- self-test
def qkdrec_selftest_phi(x):
    """phi(clamp(x)) evaluated by the sum-product kernels' device function."""
    torch = _torch()
    xp = _dev(x, torch.float32, "x")
    out = torch.empty_like(x)
    _check(lib().qkdrec_selftest_phi(xp, x.numel(), ctypes.c_void_p(out.data_ptr()), _stream(x)))
    return out


def qkdrec_selftest_phi_pair(x):
    """phi(clamp(|x|)) evaluated by the two-frames-per-lane sum-product kernel's function
    (x: float32 CUDA tensor of even length)."""
    torch = _torch()
    xp = _dev(x, torch.float32, "x")
    out = torch.empty_like(x)
    _check(lib().qkdrec_selftest_phi_pair(xp, x.numel(), ctypes.c_void_p(out.data_ptr()), _stream(x)))
    return out


def qkdrec_selftest_gauss_tail(z):
    """Q(|z|) = P(N(0,1) > |z|) as the slice LLR kernel evaluates it (z: float32 CUDA
    tensor of even length)."""
    torch = _torch()
    zp = _dev(z, torch.float32, "z")
    out = torch.empty_like(z)
    _check(lib().qkdrec_selftest_gauss_tail(zp, z.numel(), ctypes.c_void_p(out.data_ptr()), _stream(z)))
    return out
