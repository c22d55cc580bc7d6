"""The Gaussian upper tail Q(z) = P(N(0,1) > z) as the slice LLR kernel evaluates it
(a fitted Mills-ratio polynomial times e^{-z^2/2} on the MUFU approximations, two
values per packed FP32x2 operation), against FP64 truth from scipy: relative error
below 2e-6 while Q is a normal float, absolute error below the smallest normal float
beyond, exactly 0 from z = 14 (and at infinity)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2108_08418_b300 as q  # noqa: E402

FLT_MIN = float(np.finfo(np.float32).tiny)


def test_gauss_tail_error():
    from scipy.special import ndtr
    from paper_2108_08418_b300 import build
    build.build()
    z = np.concatenate([np.linspace(0.0, 16.0, 400_000), np.linspace(0.0, 1e-3, 1000),
                        -np.linspace(0.0, 10.0, 1000),
                        np.array([0.0, 1e-38, 1.0, 12.9, 14.0, 30.0, 1e30, np.inf, -np.inf, 7.5])]).astype(np.float32)
    got = q.qkdrec_selftest_gauss_tail(torch.from_numpy(z).cuda()).cpu().numpy().astype(np.float64)
    ref = ndtr(-np.abs(z.astype(np.float64)))
    normal = ref >= FLT_MIN
    rel = np.abs(got[normal] - ref[normal]) / ref[normal]
    print("max relative error of Q where Q is normal:", rel.max())
    assert rel.max() < 2e-6
    assert np.all(np.abs(got[~normal] - ref[~normal]) < FLT_MIN)
    assert np.all(got[np.abs(z) >= 14.0] == 0.0)
    assert np.all(got >= 0.0) and np.all(np.isfinite(got))


def test_gauss_tail_argument_errors():
    from paper_2108_08418_b300 import build
    build.build()
    with pytest.raises(q.QkdrecError):
        q.qkdrec_selftest_gauss_tail(torch.zeros(3, device="cuda"))
