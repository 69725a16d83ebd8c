"""Host emulation of the pair kernel's tile-pair enumeration (Sec. 2: auto
counts take the pairs i < j, cross counts all n_a n_b pairs): item t of an auto
count is the tile pair (I, J) with I <= J, rows in order, and item t of a cross
count is (t / T_b, t mod T_b).  The kernel inverts the row offsets
off(I) = I T - I (I - 1) / 2 with an FP64 square root and then corrects the
row by integer steps; this evaluates the same FP64 steps in Python floats
(IEEE double, a correctly rounded square root as on the device) and checks
that every item maps to its tile pair, that the map is one to one onto the
upper triangle, and that the correction takes at most one step for catalogues
of up to 2^20 tiles (a billion points of 1024-point tiles)."""
import math

import numpy as np
import pytest


def item_to_tiles(t, T_a, T_b, is_auto):
    """The kernel's item_to_tiles, step by step; returns (I, J, correction steps)."""
    if not is_auto:
        return t // T_b, t - (t // T_b) * T_b, 0
    T = T_a
    b = 2.0 * float(T) + 1.0
    i = int(math.floor((b - math.sqrt(max(b * b - 8.0 * float(t), 0.0))) * 0.5))
    i = min(max(i, 0), T - 1)
    steps = 0
    while i > 0 and i * T - i * (i - 1) // 2 > t:
        i -= 1
        steps += 1
    while i + 1 < T and (i + 1) * T - (i + 1) * i // 2 <= t:
        i += 1
        steps += 1
    return i, i + (t - (i * T - i * (i - 1) // 2)), steps


@pytest.mark.parametrize("T", [1, 2, 3, 4, 5, 31, 32, 33, 40, 97, 128])
def test_auto_items_cover_the_upper_triangle_once(T):
    n = T * (T + 1) // 2
    seen = set()
    for t in range(n):
        I, J, steps = item_to_tiles(t, T, T, True)
        assert 0 <= I <= J < T, (T, t, I, J)
        assert steps <= 1
        seen.add((I, J))
    assert len(seen) == n
    # rows in order: item t + 1 follows item t along the row, then the next row
    prev = item_to_tiles(0, T, T, True)[:2]
    assert prev == (0, 0)
    for t in range(1, n):
        cur = item_to_tiles(t, T, T, True)[:2]
        assert cur == (prev[0], prev[1] + 1) or (cur == (prev[0] + 1, prev[0] + 1)
                                                 and prev[1] == T - 1)
        prev = cur


@pytest.mark.parametrize("T", [977, 1954, 9766, 97657, 1 << 20])
def test_auto_row_boundaries_of_large_counts(T):
    """Every row start, the item before it and the last item, plus random items:
    the tile pair is the closed form's, reached in at most one correction."""
    rng = np.random.default_rng(T)
    n = T * (T + 1) // 2
    rows = np.unique(np.concatenate([np.arange(min(T, 4096)),
                                     rng.integers(0, T, 4096), [T - 1]]))
    for I in rows.tolist():
        start = I * T - I * (I - 1) // 2
        for t, want in ((start, (I, I)), (start - 1, (I - 1, T - 1)),
                        (start + (T - 1 - I), (I, T - 1))):
            if t < 0:
                continue
            got_I, got_J, steps = item_to_tiles(t, T, T, True)
            assert (got_I, got_J) == want, (T, t)
            assert steps <= 1, (T, t, steps)
    for t in rng.integers(0, n, 20000).tolist():
        I, J, steps = item_to_tiles(t, T, T, True)
        assert 0 <= I <= J < T and steps <= 1
        assert I * T - I * (I - 1) // 2 + (J - I) == t


@pytest.mark.parametrize("T_a,T_b", [(1, 1), (3, 7), (977, 1954), (9766, 9766)])
def test_cross_items_are_row_major(T_a, T_b):
    rng = np.random.default_rng(T_a * 7 + T_b)
    for t in list(range(min(T_a * T_b, 5000))) + rng.integers(0, T_a * T_b, 5000).tolist():
        I, J, _ = item_to_tiles(t, T_a, T_b, False)
        assert 0 <= I < T_a and 0 <= J < T_b and I * T_b + J == t
