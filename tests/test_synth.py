"""Input generators: determinism, degree structure, girth, and sample statistics."""
import numpy as np
import pytest

import synth


@pytest.mark.parametrize("n,rate", [(4096, 0.5), (4096, 57 / 64), (4096, 1 / 16), (16384, 0.40625)])
def test_regular_code_structure(n, rate):
    M = synth.checks_for_rate(n, rate)
    rp, ci, res = synth.make_regular_code(77, n, M)
    cols, rows = synth.degrees(rp, ci, n)
    assert np.all(cols == 3)
    assert rows.max() - rows.min() <= 1
    assert rows.sum() == 3 * n and len(rows) == M
    assert res == 0
    # no repeated variable inside a check, no 4-cycle (two checks sharing two variables)
    sets = [frozenset(ci[rp[c]:rp[c + 1]].tolist()) for c in range(M)]
    assert all(len(s) == rp[c + 1] - rp[c] for c, s in enumerate(sets))
    pairs = {}
    for c, s in enumerate(sets):
        vs = sorted(s)
        for i in range(len(vs)):
            for j in range(i + 1, len(vs)):
                key = (vs[i], vs[j])
                assert key not in pairs, "4-cycle"
                pairs[key] = c


def test_code_is_deterministic():
    a = synth.make_regular_code(5, 2048, 1024)
    b = synth.make_regular_code(5, 2048, 1024)
    c = synth.make_regular_code(6, 2048, 1024)
    assert np.array_equal(a[1], b[1]) and not np.array_equal(a[1], c[1])


def test_gaussian_pair_statistics():
    x, y = synth.gaussian_pair(3, 1_000_000, 3.0)
    assert x.dtype == np.float32 and y.dtype == np.float32
    n = (y.astype(np.float64) - x)
    assert abs(x.mean()) < 5e-3 and abs(x.var() - 1) < 5e-3
    assert abs(n.var() - 1 / 3) < 3e-3
    assert abs(np.corrcoef(x, n)[0, 1]) < 5e-3
    x2, y2 = synth.gaussian_pair(3, 1000, 3.0)
    assert np.array_equal(x2, synth.gaussian_pair(3, 1000, 3.0)[0])


def test_gaussian_pair_prefix_consistent():
    x1, y1 = synth.gaussian_pair(9, 5000, 15.0)
    x2, y2 = synth.gaussian_pair(9, 123, 15.0)
    assert np.array_equal(x1[:123], x2) and np.array_equal(y1[:123], y2)


@pytest.mark.parametrize("n,rate", [(512, 60 / 64), (4096, 60 / 64), (2048, 0.9)])
def test_dense_codes_have_no_repeated_pairs(n, rate):
    """Dense high-rate codes keep 4-cycles, but H stays a set of distinct
    (check, variable) pairs with every column of degree 3."""
    M = synth.checks_for_rate(n, rate)
    rp, ci, res = synth.make_regular_code(17, n, M)
    rows = np.repeat(np.arange(M), np.diff(rp))
    assert np.unique(rows.astype(np.int64) * n + ci).size == ci.size
    assert np.all(np.bincount(ci, minlength=n) == 3)


def test_uneven_frames_and_gaussian_frames():
    n, snr = synth.uneven_frames(3, 500, (4096, 16384), (2.0, 15.0), snr_step=0.1)
    assert set(n.tolist()) <= {4096, 16384} and snr.min() >= 2.0 - 1e-12 and snr.max() <= 15.0 + 1e-12
    assert np.allclose(np.round((snr - 2.0) / 0.1), (snr - 2.0) / 0.1)
    lengths = np.array([5, 0, 7])
    x, y = synth.gaussian_frames(4, lengths, np.array([3.0, 5.0, 1e6]))
    assert x.size == y.size == 12 and x.dtype == np.float32
    assert np.allclose(x[5:], y[5:], atol=1e-2)          # SNR 1e6: y ~ x


@pytest.mark.parametrize("Z,nb", [(64, 6), (256, 24), (1024, 8)])
def test_quasi_cyclic_code_structure(Z, nb):
    rp, ci, S, res = synth.make_qc_code(11, Z, nb)
    n, M = nb * Z, 3 * Z
    assert res == 0 and rp.size == M + 1 and ci.size == 3 * n
    cols, rows = synth.degrees(rp, ci, n)
    assert np.all(cols == 3) and np.all(rows == nb)
    # check i Z + z, edge k -> variable k Z + (z + S[i, k]) mod Z
    for c in (0, Z - 1, Z, 2 * Z + 5):
        i, z = divmod(c, Z)
        assert np.array_equal(ci[rp[c]:rp[c + 1]], np.arange(nb) * Z + (z + S[i]) % Z)
    # no 4-cycle: two checks share at most one variable
    from scipy.sparse import csr_matrix
    H = csr_matrix((np.ones(ci.size, dtype=np.int32), ci, rp), shape=(M, n))
    overlap = (H @ H.T).tocoo()
    assert overlap.data[overlap.row != overlap.col].max(initial=0) <= 1


def test_c_philox_permutation_matches_numpy():
    """The C generator's Philox-4x64-10 stream and Fisher-Yates shuffle draw the
    permutation numpy's Generator(Philox(seed)) draws (so the library's code
    construction and the generator's agree)."""
    for seed, count in ((0, 1), (7, 10), (2003, 3 * 4096), (2**40 + 5, 99991), (2**64 - 1, 777)):
        assert np.array_equal(synth.philox_permutation_c(seed, count), synth.philox(seed).permutation(count))


def test_c_construction_equals_numpy_construction():
    for seed, n, rate in ((2012, 4096, 0.75), (9, 2048, 40 / 64), (31337, 8192, 0.25)):
        M = synth.checks_for_rate(n, rate)
        a = synth.make_regular_code(seed, n, M)
        b = synth.make_regular_code_c(seed, n, M)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2]
