"""The ensemble's tile planner (host code of the C library, no GPU): every
row of every lattice lies in exactly one band, and the plan and its score
equal a plain Python restatement of the planning rules (bands of round(M /
band) near-equal rows, first fit of the bands sorted longest first into
32-lane warps that close at 7/8 of their longest band, tiles ordered longest
first, tile costs max_len + 2 * depth; the score of a launch of 32 chunks:
32 * max(mean cost per warp, 1.2 * longest tile) plus the makespan of
longest-first list scheduling beyond the mean)."""
import heapq
import math

import numpy as np
import pytest


def restated_plan(M, N, band, depth, warps):
    bands = []
    for l, (m, n) in enumerate(zip(M, N)):
        m, n = int(m), int(n)
        W = (n + 63) // 64
        nb = max(1, min(m, int(math.floor(m / band + 0.5))))
        while (m + nb - 1) // nb > 65535:
            nb += 1
        base, rem = m // nb, m % nb
        r0 = 0
        for b in range(nb):
            ln = base + (1 if b < rem else 0)
            bands.append((ln, W, l, r0))
            r0 += ln
    bands.sort(key=lambda x: (-x[0], -x[1], x[2], x[3]))
    tiles, open_ = [], []
    for ln, W, l, r0 in bands:
        chosen = None
        for t in list(open_):
            if t["max"] * 7 > ln * 8:
                open_.remove(t)
                continue
            if 32 - t["used"] >= W:
                chosen = t
                break
        if chosen is None:
            chosen = {"max": ln, "used": 0}
            tiles.append(chosen)
            open_.append(chosen)
        chosen["used"] += W
        if chosen["used"] == 32:
            open_.remove(chosen)
    costs = sorted((t["max"] + 2 * depth for t in tiles), reverse=True)
    heap = [0] * warps
    makespan = 0
    for c in costs:
        f = heapq.heappop(heap) + c
        makespan = max(makespan, f)
        heapq.heappush(heap, f)
    mean = sum(costs) / warps
    return len(tiles), 32 * max(mean, 1.2 * costs[0]) + (makespan - mean)


@pytest.mark.parametrize("band", [16, 64, 448, 5000])
def test_plan_matches_restatement_and_covers_every_row(lib, band):
    rng = np.random.Generator(np.random.PCG64(band))
    M = rng.integers(1, 1500, size=200)
    N = rng.integers(1, 2049, size=200)
    M[:4] = [1, 70000, 2, 131071]   # one row; bands capped at 65535 rows
    N[:4] = [2048, 64, 1, 65]
    for depth, warps in [(8, 1776), (1, 7), (4, 300)]:
        tiles, score, rows = lib.bml_ensemble_plan(M, N, band, depth, warps)
        want_tiles, want_score = restated_plan(M, N, band, depth, warps)
        assert tiles == want_tiles
        assert score == pytest.approx(want_score, rel=1e-12)
        np.testing.assert_array_equal(rows, M)


def test_plan_rejects_bad_arguments(lib):
    for args in [([10], [4096], 16, 8, 100), ([10], [64], 0, 8, 100), ([0], [64], 16, 8, 100),
                 ([10], [64], 16, 0, 100), ([10], [64], 16, 8, 0)]:
        with pytest.raises(lib.BMLError) as e:
            lib.bml_ensemble_plan(*args)
        assert e.value.code == lib.BML_EINVAL
