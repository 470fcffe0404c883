"""GPU parity of Model II (Sec. 2 variant: one synchronous phase per step, a
contested empty cell goes to one of its two candidates by the tie-break
bits) against the oracle, through the C ABI: lattices and every per-step
count, bit for bit."""
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


def counts_equal(sim_counts, mlr, mtb):
    tot, lr, tb = sim_counts
    np.testing.assert_array_equal(lr, mlr)
    np.testing.assert_array_equal(tb, mtb)
    np.testing.assert_array_equal(tot, mlr + mtb)


@pytest.mark.parametrize("M,N", SHAPES)
def test_model2_every_depth_matches_oracle(lib, M, N):
    """Every depth with bands that do not divide M, bands shorter than the
    depth and one band; 37 steps (not a multiple of any depth)."""
    g0 = random_lattice(M, N, 3 * M + N, 0.12, 0.12)
    K = 37
    want, mlr, mtb = oracle.run_model(g0, K, 2, tie_seed=77)
    for k, band in [(1, 7), (2, 3), (4, 37), (8, 16), (8, M)]:
        with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=k) as sim:
            sim.set_model(lib.BML_MODEL_II, 77)
            sim.set_tiling(k, band)
            sim.write(g0)
            sim.step(10)
            sim.step(K - 10)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            counts_equal(sim.moved_counts(), mlr, mtb)
            assert sim.model == (lib.BML_MODEL_II, 77)


@pytest.mark.parametrize("M,N", [(100, 4096), (77, 6144), (40, 32768), (5, 4224),
                                 (60, 128 * 63), (50, 128 * 17), (40, 128 * 62)])
def test_model2_two_words_per_lane_matches_oracle(lib, M, N):
    """The two-words-per-lane kernel (rows of full words, an even number of
    them, more than 32) at every depth and ragged bands."""
    g0 = random_lattice(M, N, 5 * M + N, 0.1, 0.1)
    K = 21
    want, mlr, mtb = oracle.run_model(g0, K, 2, tie_seed=13)
    for k, band in [(1, 7), (2, 16), (4, 33), (8, 19), (8, M)]:
        with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=k) as sim:
            sim.set_model(lib.BML_MODEL_II, 13)
            sim.set_tiling(k, band, lane_words=2)
            assert sim.tiling == (k, band, 2)
            sim.write(g0)
            sim.step(K)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            counts_equal(sim.moved_counts(), mlr, mtb)


def test_model2_autotuned_256_density_03_1024_steps(lib):
    M = N = 256
    with lib.Lattice(M, N, seed=1, p_lr=0.15, p_tb=0.15, reserve_steps=1024) as sim:
        sim.set_model(lib.BML_MODEL_II, 5)
        k, band, lw = sim.tiling
        assert lw == 1 and band >= 1
        g0 = oracle.init(M, N, 1, 0.15, 0.15)
        sim.step(1024)
        want, mlr, mtb = oracle.run_model(g0, 1024, 2, tie_seed=5)
        np.testing.assert_array_equal(sim.read(), want)
        counts_equal(sim.moved_counts(), mlr, mtb)


def test_switching_models_continues_the_step_index(lib):
    """10 Model I steps, then 20 Model II steps (tie-breaks of steps 10..29),
    then 5 Model I steps again."""
    M, N = 77, 300
    g0 = random_lattice(M, N, 12, 0.1, 0.1)
    a, lr1, tb1 = oracle.run(g0, 10)
    b, lr2, tb2 = oracle.run_model(a, 20, 2, tie_seed=3, t0=10)
    c, lr3, tb3 = oracle.run(b, 5)
    with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=4) as sim:
        sim.write(g0)
        sim.step(10)
        sim.set_model(lib.BML_MODEL_II, 3)
        sim.step(20)
        np.testing.assert_array_equal(sim.read(), b)
        sim.set_model(lib.BML_MODEL_I)
        sim.step(5)
        np.testing.assert_array_equal(sim.read(), c)
        counts_equal(sim.moved_counts(), np.concatenate([lr1, lr2, lr3]),
                     np.concatenate([tb1, tb2, tb3]))


def test_tie_seed_selects_the_run(lib):
    M, N = 128, 512
    g0 = random_lattice(M, N, 31, 0.2, 0.2)
    got = []
    for seed in (1, 2):
        want, _, _ = oracle.run_model(g0, 40, 2, tie_seed=seed)
        with lib.Lattice(M, N, seed=1, density=0.2, kernel="tblock", block_k=8) as sim:
            sim.set_model(lib.BML_MODEL_II, seed)
            sim.write(g0)
            sim.step(40)
            got.append(sim.read())
            np.testing.assert_array_equal(got[-1], want)
    assert np.any(got[0] != got[1])


def test_model2_checkpoint_resume(lib):
    """A written lattice restarts the step index at 0 (so do the tie-break
    bits): resuming a saved state equals running from it with t0 = 0."""
    M, N = 60, 190
    g0 = random_lattice(M, N, 8, 0.15, 0.15)
    with lib.Lattice(M, N, seed=1, density=0.3, kernel="tblock", block_k=2) as sim:
        sim.set_model(lib.BML_MODEL_II, 9)
        sim.step(13)
        sim.write(g0)
        assert sim.steps_done == 0
        sim.step(21)
        want, mlr, mtb = oracle.run_model(g0, 21, 2, tie_seed=9)
        np.testing.assert_array_equal(sim.read(), want)
        counts_equal(sim.moved_counts(), mlr, mtb)


def test_model2_4096_against_threaded_oracle(lib):
    M = N = 4096
    g0 = oracle.init(M, N, 1, 0.05, 0.05)
    want, mlr, mtb = oracle.run_model(g0, 256, 2, tie_seed=1, threads=os.cpu_count() or 1)
    with lib.Lattice(M, N, seed=1, density=0.1, reserve_steps=256) as sim:
        sim.set_model(lib.BML_MODEL_II, 1)
        sim.step(256)
        np.testing.assert_array_equal(sim.read(), want)
        counts_equal(sim.moved_counts(), mlr, mtb)


def test_model2_rejections(lib):
    with lib.Lattice(16, 64, seed=1, density=0.2, kernel="byte") as sim:
        with pytest.raises(lib.BMLError) as e:
            sim.set_model(lib.BML_MODEL_II, 1)
        assert e.value.code == lib.BML_EINVAL
        assert sim.model == (lib.BML_MODEL_I, 0)
    with lib.Lattice(16, 64 * 40, seed=1, density=0.2, kernel="tblock", block_k=2) as sim:
        with pytest.raises(lib.BMLError):
            sim.set_model(7, 1)
        sim.set_model(lib.BML_MODEL_II, 1)
        with pytest.raises(lib.BMLError):
            sim.set_tiling(1, 0)
        sim.set_tiling(2, 8)
        assert sim.tiling == (2, 8, 1)
        sim.set_tiling(2, 8, lane_words=2)
        assert sim.tiling == (2, 8, 2)
        sim.set_model(lib.BML_MODEL_I)          # a TBLOCK object keeps its tiling
        sim.set_model(lib.BML_MODEL_II, 2)
        assert sim.tiling == (2, 8, 2)
    with lib.Lattice(16, 100, seed=1, density=0.2, kernel="tblock", block_k=2) as sim:
        sim.set_model(lib.BML_MODEL_II, 1)
        with pytest.raises(lib.BMLError):       # N % 64 != 0: one word per lane only
            sim.set_tiling(2, 8, lane_words=2)
