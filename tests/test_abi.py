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


def test_rate_rule_matches_oracle(L):
    for c in np.linspace(-0.1, 1.2, 1301):
        assert q.qkdrec_code_rate(c) == oracle.code_rate(c)
    # the nearest multiple of 1/64, ties up, capped at 63/64; 0 = disclosed
    assert q.qkdrec_code_rate(0.5 / 0.95) == 0.5
    assert q.qkdrec_code_rate((10.5 / 64) / 0.95) == 11 / 64
    assert q.qkdrec_code_rate(2.0) == 63 / 64 and q.qkdrec_code_rate(-1.0) == 0.0
    assert q.qkdrec_code_rate(0.3, fraction=0.9, denom=128) == oracle.code_rate(0.3, 0.9, 128)
    r = ctypes.c_double()
    assert L.qkdrec_code_rate(0.5, 0.95, 1, ctypes.byref(r)) == q.ERR_ARG
    assert L.qkdrec_code_rate(float("nan"), 0.95, 64, ctypes.byref(r)) == q.ERR_ARG
    assert L.qkdrec_code_rate(0.5, 0.95, 64, None) == q.ERR_ARG


def test_quantiser_range_and_check_count_match_the_workload_helpers(L):
    for snr in (2.0, 3.0, 7.3, 15.0):
        for va in (1.0, 2.5):
            lo, hi = q.qkdrec_quantiser_range(snr, va)
            rlo, rhi = oracle.quantiser_range(snr, va)
            assert lo == rlo and hi == rhi
    lo, hi = ctypes.c_double(), ctypes.c_double()
    assert L.qkdrec_quantiser_range(0.0, 1.0, ctypes.byref(lo), ctypes.byref(hi)) == q.ERR_ARG
    import synth
    for n in (64, 4096, 1 << 20):
        for k in range(1, 64):
            assert q.qkdrec_checks_for_rate(n, k / 64) == synth.checks_for_rate(n, k / 64)
    m = ctypes.c_int32()
    assert L.qkdrec_checks_for_rate(64, 1.0, ctypes.byref(m)) == q.ERR_ARG


@pytest.mark.parametrize("seed,n,rate,dv", [(2012, 4096, 0.75, 3), (2000 + 100 * 14 + 3, 1 << 14, 54 / 64, 3),
                                            (11, 1024, 0.5, 4), (5000, 16384, 0.5, 3), (7, 256, 60 / 64, 3)])
def test_make_regular_code_through_the_abi_equals_the_input_generator(L, seed, n, rate, dv):
    """The library builds the same seeded slice code as the generator the tests and
    the bench construct their inputs with (numpy Philox permutation + C swaps)."""
    import synth
    M = synth.checks_for_rate(n, rate)
    rp, ci, left = q.qkdrec_make_regular_code(seed, n, M, dv)
    rp_ref, ci_ref, left_ref = synth.make_regular_code(seed, n, M, dv)
    assert np.array_equal(rp, rp_ref) and np.array_equal(ci, ci_ref) and left == left_ref
    cols, rows = synth.degrees(rp, ci, n)
    assert np.all(cols == dv) and rows.max() - rows.min() <= 1 and rp[-1] == dv * n
    # a set of (check, variable) pairs: what qkdrec_code_create accepts
    for c in range(0, M, max(1, M // 50)):
        row = ci[rp[c]:rp[c + 1]]
        assert len(np.unique(row)) == len(row)


def test_make_regular_code_argument_errors(L):
    P = ctypes.POINTER(ctypes.c_int32)
    rp, ci, left = P(), P(), ctypes.c_int32()
    assert L.qkdrec_make_regular_code(1, 0, 10, 3, ctypes.byref(rp), ctypes.byref(ci), None) == q.ERR_ARG
    assert L.qkdrec_make_regular_code(1, 64, 0, 3, ctypes.byref(rp), ctypes.byref(ci), None) == q.ERR_ARG
    assert L.qkdrec_make_regular_code(1, 64, 193, 3, ctypes.byref(rp), ctypes.byref(ci), None) == q.ERR_ARG
    assert L.qkdrec_make_regular_code(1, 4, 1, 3, ctypes.byref(rp), ctypes.byref(ci), None) == q.ERR_ARG  # degree 12 > n
    assert L.qkdrec_make_regular_code(1, 64, 32, 3, None, ctypes.byref(ci), None) == q.ERR_ARG
    assert L.qkdrec_make_regular_code(1, 64, 32, 3, ctypes.byref(rp), ctypes.byref(ci), ctypes.byref(left)) == q.OK
    L.qkdrec_free(ctypes.cast(rp, ctypes.c_void_p))
    L.qkdrec_free(ctypes.cast(ci, ctypes.c_void_p))
    L.qkdrec_free(None)


def test_reconciliation_efficiency_matches_the_oracle(L):
    """Eq. beta from the library against the oracle's quantiser entropy: with the
    rates at the slice capacities the numerator is I(M(Y); X) (Eq. beta2 with the
    Slepian-Wolf bound tight), so beta < 1; with every slice disclosed it is
    (Pi(M(Y)) - m) / I_AB."""
    import math
    for snr, m in ((3.0, 5), (15.0, 5), (3.0, 4)):
        lo, hi = oracle.quantiser_range(snr)
        caps = [oracle.slice_capacity(snr, m, j) for j in range(m)]
        beta, H = q.qkdrec_reconciliation_efficiency(snr, m, lo, hi, caps)
        assert abs(H - oracle.label_entropy(snr, m)) < 1e-10
        iab = 0.5 * math.log2(1 + snr)
        assert abs(beta - (oracle.label_entropy(snr, m) - m + sum(caps)) / iab) < 1e-9
        assert 0.9 < beta < 1.0
        b0, _ = q.qkdrec_reconciliation_efficiency(snr, m, lo, hi, [0.0] * m)
        assert abs(b0 - (H - m) / iab) < 1e-12
    with pytest.raises(q.QkdrecError):
        q.qkdrec_reconciliation_efficiency(3.0, 2, -1.0, 1.0, [0.5, 1.0])


def test_reconcile_workspace_grows_by_one_slot_per_partition_in_flight(L):
    """Host-side sizing of the whole-block call (no device work: every slice of
    these partitions is disclosed, so no code is needed): a shared part plus one
    equal slot per partition in flight, capped at the number of partitions;
    max_in_flight < 1 is refused."""
    torch = pytest.importorskip("torch")
    count, m = 1 << 12, 3
    opts = q.DecodeOpts()
    pts = [dict(n=n, codes=[None] * m, alice_packed=torch.zeros((m, count // 8), dtype=torch.uint8))
           for n in (256, 512, 1024)]
    s = [q.qkdrec_reconcile_workspace_size_limited(count, m, opts, pts, k) for k in (1, 2, 3, 10)]
    slot = s[1] - s[0]
    assert slot > 0 and s[2] - s[1] == slot and s[3] == s[2]
    assert q.qkdrec_reconcile_workspace_size(count, m, opts, pts) == s[2]
    assert s[0] - slot >= count * 8        # the shared part holds x and y staging
    with pytest.raises(q.QkdrecError) as e:
        q.qkdrec_reconcile_workspace_size_limited(count, m, opts, pts, 0)
    assert e.value.status == q.ERR_ARG
