"""The phase-diagram workload against the oracle: the same runs (seeded
placement, every step) computed by the oracle give the same velocities, jam
flags and per-density curves; the Fig. 1 lattices equal the oracle's."""
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def oracle_runs(N, densities, seeds, T, window):
    rho, v, jam = [], [], []
    for r in densities:
        for s in range(1, seeds + 1):
            g0 = oracle.init(N, N, s, r / 2, r / 2)
            _, lr, tb = oracle.run(g0, T, threads=os.cpu_count() or 1)
            tot = lr + tb
            cars = int(np.count_nonzero(g0))
            rho.append(r)
            v.append(tot[T - window:].sum() / (window * cars) if cars else 0.0)
            jam.append(bool(np.any(tot == 0)))
    return np.array(rho), np.array(v), np.array(jam)


def test_phase_runs_match_oracle(lib):
    """Sizes 32 and 64 through the batched ensemble, 96 through single
    lattices (ensemble_max_n = 64); densities 0.2..0.6, 1024 steps."""
    from paper_1804_07981_b300 import phase
    dens, T, window = [0.2, 0.3, 0.4, 0.5, 0.6], 1024, 128
    for N, seeds in [(32, 4), (64, 4), (96, 2)]:
        if N <= 64:
            got = phase._runs_ensemble(N, dens, seeds, T, window, None)
        else:
            got = phase._runs_single(N, dens, seeds, T, window, None, chunk=300)
        want = oracle_runs(N, dens, seeds, T, window)
        np.testing.assert_array_equal(got[0], want[0])
        np.testing.assert_allclose(got[1], want[1], rtol=1e-12, atol=0)
        np.testing.assert_array_equal(got[2], want[2])
        if N > 64:
            # the same runs with a given tiling for the concurrent lattices
            # (depth 8, 16-row bands, one word per lane)
            got = phase._runs_single(N, dens, seeds, T, window, None, chunk=300,
                                     tiling=(8, 16, 1))
            np.testing.assert_array_equal(got[0], want[0])
            np.testing.assert_allclose(got[1], want[1], rtol=1e-12, atol=0)
            np.testing.assert_array_equal(got[2], want[2])
    curves = phase.phase_diagram([32, 96], dens, 4, T, window, ensemble_max_n=64,
                                 single_seeds=2)
    for N, S in [(32, 4), (96, 2)]:
        rho, v, jam = oracle_runs(N, dens, S, T, window)
        c = curves[N]
        for i, r in enumerate(dens):
            assert c["runs"][i] == S
            assert c["jam_frac"][i] == jam[rho == r].mean()
            assert abs(c["v_mean"][i] - v[rho == r].mean()) < 1e-12


def test_phase_runs_in_the_shipped_tiling_match_oracle(lib):
    """The full diagram's tiling for its concurrent single lattices (two
    words per lane, depth 8, 32-row bands) on the smallest square lattice it
    applies to, 2176 x 2176 (17 word pairs per row, one cyclic lane group
    like a 4096-column row): velocities and jam flags equal the oracle's."""
    from paper_1804_07981_b300 import phase
    tiling = tuple(phase.FULL["single_tiling"])
    assert tiling[2] == 2
    N, dens, seeds, T, window = 2176, [0.3, 0.5], 1, 192, 64
    want = oracle_runs(N, dens, seeds, T, window)
    got = phase._runs_single(N, dens, seeds, T, window, None, chunk=100, tiling=tiling)
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_allclose(got[1], want[1], rtol=1e-12, atol=0)
    np.testing.assert_array_equal(got[2], want[2])


def test_fig1_lattices_match_oracle(lib, tmp_path):
    """256 x 256 after 4096 steps at densities 0.25, 0.32, 0.38 (the Fig. 1
    caption): the pictured lattices are the oracle's; 0.25 flows freely
    (nearly every vehicle moves), 0.32 is intermediate, 0.38 is jammed
    (nothing moves)."""
    from paper_1804_07981_b300 import phase
    res = phase.fig1(str(tmp_path / "fig1"), scale=1)
    for (path, vel), r in zip(res, (0.25, 0.32, 0.38)):
        want, lr, tb = oracle.run(oracle.init(256, 256, 1, r / 2, r / 2), 4096)
        data = open(path, "rb").read()
        head = b"P6\n256 256\n255\n"
        assert data.startswith(head)
        px = np.frombuffer(data[len(head):], dtype=np.uint8).reshape(256, 256, 3)
        np.testing.assert_array_equal(px, phase.COLOURS[want])
        cars = int(np.count_nonzero(want))
        assert abs(vel - (lr + tb)[-64:].mean() / cars) < 1e-12
    assert res[0][1] > 0.99
    assert 0.5 < res[1][1] < 0.99
    assert res[2][1] == 0.0
