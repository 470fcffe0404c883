"""GPU parity of Model III (Sec. 2 variant: a cell may hold an LR and a TB
vehicle; the reading: one synchronous phase per step, a vehicle moves iff
its target holds no vehicle, a contested empty cell receives both) against
the oracle, through the C ABI: lattices (byte 3 = one vehicle of each kind)
and every per-step count, bit for bit."""
import os

import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import random_lattice

pytestmark = pytest.mark.gpu

SHAPES = [
    (1, 1), (1, 2), (2, 1), (1, 70), (70, 1), (3, 3), (5, 64), (7, 63), (9, 65),
    (33, 127), (17, 129), (130, 200), (64, 2047), (40, 2048), (31, 2049),
    (23, 2100), (29, 4097), (19, 4160), (300, 1000),
]


def with_doubles(g, seed, frac=0.05):
    """g with a fraction of its cells turned into doubly occupied ones."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = g.copy()
    out[rng.random(g.shape) < frac] = 3
    return out


def counts_equal(sim_counts, mlr, mtb):
    tot, lr, tb = sim_counts
    np.testing.assert_array_equal(lr, mlr)
    np.testing.assert_array_equal(tb, mtb)
    np.testing.assert_array_equal(tot, mlr + mtb)


@pytest.mark.parametrize("M,N", SHAPES)
def test_model3_every_depth_matches_oracle(lib, M, N):
    """One word per lane at every depth, bands that do not divide M, bands
    shorter than the depth and one band; 37 steps from a lattice holding
    doubly occupied cells."""
    g0 = with_doubles(random_lattice(M, N, 3 * M + N, 0.2, 0.2), M + N)
    K = 37
    want, mlr, mtb = oracle.run_model(g0, K, 3)
    for k, band in [(1, 7), (2, 3), (4, 37), (8, 16), (8, M)]:
        with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=k) as sim:
            sim.set_model(lib.BML_MODEL_III)
            sim.set_tiling(k, band)
            sim.write(g0)
            sim.step(10)
            sim.step(K - 10)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            counts_equal(sim.moved_counts(), mlr, mtb)
            assert sim.model[0] == lib.BML_MODEL_III


@pytest.mark.parametrize("M,N", [(100, 4096), (77, 6144), (40, 32768), (5, 4224),
                                 (60, 128 * 63), (50, 128 * 17), (40, 128 * 62)])
def test_model3_two_words_per_lane_matches_oracle(lib, M, N):
    """The two-words-per-lane kernel (interleaved layout) at every
    depth and ragged bands."""
    g0 = with_doubles(random_lattice(M, N, 5 * M + N, 0.25, 0.25), N)
    K = 21
    want, mlr, mtb = oracle.run_model(g0, K, 3)
    for k, band in [(1, 7), (2, 16), (4, 33), (8, 19), (8, M)]:
        with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=k) as sim:
            sim.set_model(lib.BML_MODEL_III)
            sim.set_tiling(k, band, lane_words=2)
            assert sim.tiling == (k, band, 2)
            sim.write(g0)
            sim.step(K)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            counts_equal(sim.moved_counts(), mlr, mtb)


def test_model3_autotuned_from_the_seeded_placement(lib):
    """Autotuned (AUTO object) from the seeded placement, 256 x 256 and
    4096 x 4096 at density 0.5: doubly occupied cells arise and every
    lattice and count equals the oracle's."""
    for M, N, K in [(256, 256, 1024), (4096, 4096, 64)]:
        with lib.Lattice(M, N, seed=1, density=0.5, reserve_steps=K) as sim:
            sim.set_model(lib.BML_MODEL_III)
            g0 = oracle.init(M, N, 1, 0.25, 0.25)
            sim.step(K)
            want, mlr, mtb = oracle.run_model(g0, K, 3, threads=os.cpu_count() or 1)
            got = sim.read()
            assert (want == 3).any()
            np.testing.assert_array_equal(got, want)
            counts_equal(sim.moved_counts(), mlr, mtb)


def test_model3_switching_and_rejections(lib):
    """Model I steps, then Model III steps on the same object; leaving
    Model III with a doubly occupied cell is refused (BML_ESTATE), a lattice
    with the byte 3 is refused unless the object runs Model III, and objects
    without streaming kernels refuse Model III."""
    M, N = 77, 300
    g0 = random_lattice(M, N, 12, 0.2, 0.2)
    a, lr1, tb1 = oracle.run(g0, 10)
    b, lr2, tb2 = oracle.run_model(a, 20, 3)
    with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=4) as sim:
        sim.write(g0)
        sim.step(10)
        sim.set_model(lib.BML_MODEL_III)
        sim.step(20)
        np.testing.assert_array_equal(sim.read(), b)
        counts_equal(sim.moved_counts(), np.concatenate([lr1, lr2]),
                     np.concatenate([tb1, tb2]))
        assert (b == 3).any()
        with pytest.raises(lib.BMLError) as e:
            sim.set_model(lib.BML_MODEL_I)
        assert e.value.code == lib.BML_ESTATE
        assert sim.model[0] == lib.BML_MODEL_III
        sim.write(g0)  # no doubly occupied cell: leaving Model III is allowed
        sim.set_model(lib.BML_MODEL_I)
        with pytest.raises(lib.BMLError) as e:
            sim.write(b)
        assert e.value.code == lib.BML_EINVAL
    for kernel in ("byte", "bitplane", "fused"):
        with lib.Lattice(16, 64, seed=1, density=0.2, kernel=kernel) as sim:
            with pytest.raises(lib.BMLError) as e:
                sim.set_model(lib.BML_MODEL_III)
            assert e.value.code == lib.BML_EINVAL
            assert sim.model[0] == lib.BML_MODEL_I
