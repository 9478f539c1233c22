"""Pins for the oracle's version of the paper's grid sampler (Section 3.1): the cardinality of
Eq. 1, the index -> (row, col) map of Eq. 2 against brute force and against the printed
closed form, the adaptive resolution of Section 3.1.2 against its quadratic, and the grid
barycentrics of Eq. 3 (third coordinate read as 1 - w1 - w2)."""
import math

import numpy as np

import oracle


def test_index_map_is_a_bijection_onto_the_triangle_grid():
    for r in (1, 2, 3, 7, 40, 2000):
        n = (r + 1) * (r + 2) // 2
        seen = set()
        # every index: brute force for small r, a sample for r = 2000
        idxs = range(n) if n < 200000 else np.random.default_rng(r).integers(0, n, 5000)
        for idx in idxs:
            row, col = oracle.grid_index(int(idx))
            assert 0 <= col <= row <= r
            assert row * (row + 1) // 2 + col == idx
            seen.add((row, col))
        if n < 200000:
            assert len(seen) == n


def test_index_map_matches_the_printed_ceiling_formula():
    # row = ceil((-3 + sqrt(8 idx + 9)) / 2) (Eq. 2) wherever the square root is not an integer
    for idx in range(0, 200000, 7):
        v = 8 * idx + 9
        s = math.isqrt(v)
        if s * s == v:
            continue
        row, col = oracle.grid_index(idx)
        assert row == math.ceil((-3 + math.sqrt(v)) / 2)
        assert col == idx - row * (row + 1) // 2


def test_adaptive_resolution_solves_the_quadratic():
    rng = np.random.default_rng(0)
    area = np.exp(rng.uniform(np.log(1e-6), np.log(1.0), 20000))
    k = np.exp(rng.uniform(np.log(10), np.log(1e5), 20000))
    r, rr = oracle.grid_resolution(area, k)
    D = 1 + 8 * k * area
    big = D >= 25
    # the real root gives exactly kA samples: (r+1)(r+2)/2 = kA
    assert np.allclose((rr[big] + 1) * (rr[big] + 2) / 2, k[big] * area[big], rtol=1e-12)
    assert np.all(r[~big] == 1) and np.all(r >= 1)
    assert np.all(np.abs(r[big] - rr[big]) <= 0.5)
    off = oracle.grid_offsets(r)
    assert np.array_equal(np.diff(off), (r + 1) * (r + 2) // 2)
    assert np.all(np.diff(off) >= 3)            # at least the three vertices


def test_grid_barycentrics_and_positions():
    tri = np.array([[0, 0, 0, 1, 0, 0, 0.5, np.sqrt(3) / 2, 0]], np.float32)   # equilateral, edge 1
    r = np.array([6])
    off = oracle.grid_offsets(r)
    s = oracle.grid_samples(tri, off, r)
    b = s["bary"]
    assert len(b) == 28 and np.allclose(b.sum(1), 1.0) and b.min() >= 0
    assert np.allclose(b * 6, np.round(b * 6))          # on the 1/r grid
    # the three vertices are samples, and all samples are distinct
    assert len({tuple(np.round(x, 9)) for x in s["xyz"]}) == 28
    corners = {tuple(np.round(tri[0, 3 * i:3 * i + 3].astype(float), 6)) for i in range(3)}
    pts = {tuple(np.round(x, 6)) for x in s["xyz"]}
    assert corners <= pts
    # even spacing on an equilateral triangle: every sample has a neighbour at distance 1/r
    from itertools import combinations
    d = np.linalg.norm(s["xyz"][:, None] - s["xyz"][None], axis=2)
    nn = np.sort(d, axis=1)[:, 1]
    assert np.allclose(nn, 1 / 6, atol=1e-6)
