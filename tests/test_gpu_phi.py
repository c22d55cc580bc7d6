"""The sum-product check function phi(x) = -ln tanh(x/2) as the kernels evaluate it
(series and identities on MUFU ex2/rcp/lg2), against FP64 truth over the whole
clamped range [1e-30, 30], and its involution phi(phi(x)) = x."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402


def phi64(x):
    x = np.clip(np.asarray(x, dtype=np.float64), 1e-30, 30.0)
    return np.log1p(2.0 / np.expm1(x))


def test_phi_relative_error():
    from paper_2108_08418_b300 import build
    build.build()
    x = np.concatenate([np.logspace(-30, np.log10(30.0), 200_001),
                        np.linspace(0.0, 4.0, 100_001),
                        np.array([0.0, 1e-38, 0.5, 2.0, 30.0, 31.0, 1e30])]).astype(np.float32)
    got = q.qkdrec_selftest_phi(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = phi64(x.astype(np.float64))
    rel = np.abs(got - ref) / ref
    print("max relative error of phi:", rel.max())
    assert rel.max() < 4e-6


def test_phi_pair_relative_error():
    """The packed two-value form used by the two-frames-per-lane kernel: same bound."""
    from paper_2108_08418_b300 import build
    build.build()
    x = np.concatenate([np.logspace(-30, np.log10(30.0), 200_000),
                        np.linspace(0.0, 4.0, 100_000), np.linspace(0.09, 0.11, 10_000),
                        np.array([0.0, 1e-38, 0.1, 2.0, 30.0, 31.0, 1e30, -2.5])]).astype(np.float32)
    got = q.qkdrec_selftest_phi_pair(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    ref = phi64(np.abs(x.astype(np.float64)))
    rel = np.abs(got - ref) / ref
    print("max relative error of the pair phi:", rel.max())
    assert rel.max() < 4e-6


def test_phi_is_an_involution():
    x = np.logspace(-6, np.log10(25.0), 10_001).astype(np.float32)
    d = torch.from_numpy(x).cuda()
    back = q.qkdrec_selftest_phi(q.qkdrec_selftest_phi(d)).cpu().numpy()
    assert np.all(np.abs(back - x) <= 1e-4 * np.maximum(x, 1.0))
