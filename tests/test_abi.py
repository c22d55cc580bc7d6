"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates arguments before touching the device, and its host
helpers agree with the oracle."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_2108_08418_b300 as q
from paper_2108_08418_b300 import build as qbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    qbuild.build()
    return q.lib()


def declared_symbols(header="qkdrec.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qkdrec_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 13
    for n in names:
        assert hasattr(L, n), n
    assert sorted(q.EXPORTED) == names
    for header in sorted(os.listdir(os.path.join(ROOT, "include"))):
        for n in declared_symbols(header):
            assert hasattr(L, n), (header, n)
    assert sorted(q.SELFTEST) == declared_symbols("qkdrec_selftest.h")


def test_version(L):
    assert "sm_103a" in q.version()


def test_code_create_rejects_bad_csr_before_device_work(L):
    h = ctypes.c_void_p()
    rp = np.array([0, 2, 4], dtype=np.int32)
    ci = np.array([0, 1, 1, 5], dtype=np.int32)         # 5 out of range for n = 4
    st = L.qkdrec_code_create(4, 2, rp.ctypes.data, ci.ctypes.data, 0, ctypes.byref(h))
    assert st == q.ERR_CSR and b"outside" in L.qkdrec_last_error()
    ci = np.array([0, 0, 1, 2], dtype=np.int32)         # repeated variable in one check
    assert L.qkdrec_code_create(4, 2, rp.ctypes.data, ci.ctypes.data, 0, ctypes.byref(h)) == q.ERR_CSR
    rp1 = np.array([0, 1, 4], dtype=np.int32)           # degree-1 check
    ci1 = np.array([0, 1, 2, 3], dtype=np.int32)
    assert L.qkdrec_code_create(4, 2, rp1.ctypes.data, ci1.ctypes.data, 0, ctypes.byref(h)) == q.ERR_CSR
    rpb = np.array([1, 2, 4], dtype=np.int32)           # row_ptr[0] != 0
    assert L.qkdrec_code_create(4, 2, rpb.ctypes.data, ci1.ctypes.data, 0, ctypes.byref(h)) == q.ERR_CSR
    assert L.qkdrec_code_create(0, 2, rp.ctypes.data, ci.ctypes.data, 0, ctypes.byref(h)) == q.ERR_ARG
    assert L.qkdrec_code_create(4, 2, None, ci.ctypes.data, 0, ctypes.byref(h)) == q.ERR_ARG
    assert L.qkdrec_code_create(4, 2, rp.ctypes.data, ci.ctypes.data, 0, None) == q.ERR_ARG


def test_argument_errors_are_synchronous(L):
    assert L.qkdrec_quantise_slices(None, -1, 4, -1.0, 1.0, 0, None, None, None) == q.ERR_ARG
    assert L.qkdrec_quantise_slices(None, 10, 9, -1.0, 1.0, 0, None, None, None) == q.ERR_ARG
    assert L.qkdrec_quantise_slices(None, 10, 4, 1.0, 1.0, 0, None, None, None) == q.ERR_ARG
    assert L.qkdrec_quantise_slices(None, 0, 4, -1.0, 1.0, 0, None, None, None) == q.OK   # empty is valid
    assert L.qkdrec_slice_llr(None, 10, 4, 4, -1.0, 1.0, 0.5, 0, None, None, None) == q.ERR_ARG  # j >= m
    assert L.qkdrec_slice_llr(None, 10, 4, 1, -1.0, 1.0, 0.5, 0, None, None, None) == q.ERR_ARG  # NULLs
    assert L.qkdrec_slice_llr(None, 10, 4, 0, -1.0, 1.0, 0.0, 0, None, None, None) == q.ERR_ARG  # sigma
    assert L.qkdrec_syndrome(None, None, 1, None, None) == q.ERR_ARG
    o = q.DecodeOptsC()
    L.qkdrec_decode_opts_default(ctypes.byref(o))
    assert (o.algo, o.prec, o.max_iter, o.early_stop, o.fallback_f32) == (q.SP_FLOOD, q.F32, 50, 1, 0)
    assert abs(o.offset - 0.5) < 1e-7 and abs(o.llr_step - 0.5) < 1e-7
    assert L.qkdrec_decode_batch(None, None, None, 1, ctypes.byref(o), None, None, None, None, None, 0,
                                 None) == q.ERR_ARG


def test_host_capacity_matches_oracle(L):
    for snr, m in ((3.0, 4), (15.0, 5)):
        lo, hi = oracle.quantiser_range(snr)
        for j in range(m):
            for lab in ("gray", "binary"):
                c = q.qkdrec_slice_capacity(snr, m, j, lo, hi, lab)
                ref = 1.0 - oracle.slice_cond_entropy(snr, m, j, lab)
                assert abs(c - ref) < 1e-9, (snr, m, j, lab)


def test_rate_rule_matches_oracle():
    for c in np.linspace(-0.1, 1.2, 1301):
        assert q.code_rate(c) == oracle.code_rate(c)
