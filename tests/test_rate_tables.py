"""The committed back-off rate tables (Sec. V-B: start from the capacity rule,
lower the rate by a fixed step while too many trial frames fail, disclose the
slice below 0.10) are complete and follow their own procedure:

* one entry per point of the workload (sweep: SNR x length x slice; uneven
  batch: length x SNR bin x slice);
* the start rate is the capacity rule recomputed here by the FP64 oracle's
  integral (0.95 x C_j on the 1/64 grid, capped);
* every accepted rate lies on the 1/64 grid, is the start rate minus a whole
  number of 3/64 steps, passed its trials (at most one failing frame of 32) and
  is at least 0.10; a disclosed slice has rate 0.
"""
import json
import os

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
M_SLICES = 5


def capacity_rule(snr, j, cap):
    k = int(np.floor(0.95 * oracle.slice_capacity(snr, M_SLICES, j) * 64 + 0.5))
    return min(max(k, 0), cap) / 64


def check_backoff(rate, start, errs):
    assert rate * 64 == int(rate * 64) and start * 64 == int(start * 64)
    assert 0.0 <= rate <= start
    if rate == 0.0:
        return
    assert rate >= 0.10 and errs <= 1
    assert (round(start * 64) - round(rate * 64)) % 3 == 0


def test_sweep_table_complete_and_consistent():
    t = json.load(open(os.path.join(ROOT, "sweep_rates.json")))
    assert t["columns"] == ["snr", "log2_n", "slice", "rate", "trial_frame_errors", "start_rate"]
    rows = {(r[0], r[1], r[2]): r[3:] for r in t["rates"]}
    keys = {(s, ln, j) for s in (3.0, 15.0) for ln in (12, 14, 16, 18, 20) for j in range(M_SLICES)}
    assert set(rows) == keys
    starts = {(s, j): capacity_rule(s, j, 63) for s in (3.0, 15.0) for j in range(M_SLICES)}
    for (s, ln, j), (rate, errs, start) in rows.items():
        assert start == pytest.approx(starts[(s, j)]), (s, ln, j)
        check_backoff(rate, start, errs)
    # longer codes decode closer to capacity: at the same point of the channel
    # the longest code's accepted rate is not below the shortest's by more than
    # one back-off step
    for s in (3.0, 15.0):
        for j in range(M_SLICES):
            r12, r20 = rows[(s, 12, j)][0], rows[(s, 20, j)][0]
            assert r20 >= r12 - 3 / 64


def test_uneven_table_complete_and_consistent():
    t = json.load(open(os.path.join(ROOT, "uneven_rates.json")))
    assert t["columns"] == ["n", "snr_bin", "slice", "rate", "trial_frame_errors", "start_rate"]
    bins = t["snr_bins"]
    assert bins[0][0] == 2.0 and bins[-1][1] == 15.0 and len(bins) == 13
    rows = {(r[0], r[1], r[2]): r[3:] for r in t["rates"]}
    keys = {(n, b, j) for n in (4096, 16384, 65536) for b in range(len(bins)) for j in range(M_SLICES)}
    assert set(rows) == keys
    for b, (lo, _) in enumerate(bins):
        for j in range(M_SLICES):
            start = capacity_rule(lo, j, 60)
            for n in (4096, 16384, 65536):
                rate, errs, st = rows[(n, b, j)]
                assert st == pytest.approx(start), (n, b, j)
                check_backoff(rate, st, errs)
