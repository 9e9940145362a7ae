"""The library's aliased-bin flag (bsp_bins_aliased, host only) against
brute-force triangle counts on a 12^3 grid: bins it leaves unflagged hold the
same triangles under the mod-n closure the FFT computes and under the exact
closure q1 + q2 + q3 = 0."""
import itertools

import numpy as np

import pytest


def _modes(n, lo, hi):
    f = [j if j < n // 2 else j - n for j in range(n)]
    return np.array([q for q in itertools.product(f, f, f) if lo * lo <= sum(x * x for x in q) < hi * hi])


def _wrap(v, n):
    return (v + n // 2) % n - n // 2


@pytest.fixture(scope="module")
def flags_of():
    from paper_1708_05303_gb300 import build, bsp

    build.build()
    return bsp.bsp_bins_aliased


def test_flag_matches_brute_force_closures(flags_of):
    n, edges = 12, [1.0, 2.5, 4.0, 5.5, 7.0]
    ns = len(edges) - 1
    modes = [_modes(n, edges[i], edges[i + 1]) for i in range(ns)]
    bins = [(a, b, c) for a in range(ns) for b in range(a + 1) for c in range(b + 1)]
    flag = flags_of(n, edges, bins)
    differ = []
    for (a, b, c), fl in zip(bins, flag):
        q3 = -(modes[a][:, None, :] + modes[b][None, :, :]).reshape(-1, 3)
        ex2 = np.sum(q3 * q3, axis=1)
        exact = int(np.sum((ex2 >= edges[c] ** 2) & (ex2 < edges[c + 1] ** 2)))
        w = _wrap(q3, n)
        w2 = np.sum(w * w, axis=1)
        modular = int(np.sum((w2 > 0) & (w2 >= edges[c] ** 2) & (w2 < edges[c + 1] ** 2)))
        if not fl:
            assert exact == modular, (a, b, c)
        differ.append(exact != modular)
    # the grid does wrap some triangles, and only in flagged bins
    assert any(differ)
    assert all(f for f, d in zip(flag, differ) if d)


def test_flag_rejects_bad_input(flags_of):
    from paper_1708_05303_gb300 import bsp

    with pytest.raises(bsp.BspError):
        flags_of(12, [1.0, 2.5, 2.0], [(0, 0, 0)])       # edges not ascending
    with pytest.raises(bsp.BspError):
        flags_of(12, [1.0, 2.5, 4.0], [(2, 0, 0)])       # shell index out of range
