"""Host logic of the uneven batch's parts (no GPU): which part decodes each frame.

Every run of frames with one length is cut into consecutive pieces, one per
part, of near-equal size; a frame keeps its part for every slice (so a part
decodes a frame's slices in order, each after its lower slices).
"""
import numpy as np
import pytest

from paper_2108_08418_b300.uneven import frame_parts


def runs(lengths):
    out, f = [], 0
    while f < len(lengths):
        g = f + 1
        while g < len(lengths) and lengths[g] == lengths[f]:
            g += 1
        out.append((f, g))
        f = g
    return out


@pytest.mark.parametrize("parts", [1, 2, 3, 5])
def test_each_length_run_split_into_consecutive_near_equal_pieces(parts):
    g = np.random.default_rng(7)
    lengths = np.sort(g.choice([4096, 16384, 65536], size=301))
    p = frame_parts(lengths, parts)
    assert p.min() >= 0 and p.max() < parts
    for f, e in runs(lengths):
        piece = p[f:e]
        assert np.all(np.diff(piece) >= 0)                      # consecutive pieces
        sizes = np.bincount(piece, minlength=parts)
        assert sizes.max() - sizes.min() <= 1                   # near-equal
        if e - f >= parts:
            assert np.all(sizes > 0)                            # every part gets frames


def test_one_part_and_short_runs():
    assert np.array_equal(frame_parts([4096] * 5 + [8192], 1), np.zeros(6, np.int64))
    # a run shorter than the part count: its frames go to distinct parts
    assert frame_parts([4096, 8192, 8192], 2).tolist() == [0, 0, 1]
    assert frame_parts([4096, 4096], 3).tolist() == [0, 1]
    assert frame_parts([], 2).size == 0
