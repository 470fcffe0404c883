"""Pins of the oracle's Model II (Sec. 2 of the paper: all vehicles move in
one synchronous phase; a contested empty cell goes to one of its two
candidates, chosen at random) and Model III (the same cell may hold an LR
and a TB vehicle; the reading: one synchronous phase, a vehicle moves iff
its target holds no vehicle, a contested empty cell receives both).

Nothing here retypes the oracle's per-cell formula: the checks are an
independent car-list formulation on every tiny lattice, reductions to the
(separately pinned) Model I, conservation and exclusivity laws, the
fairness of the random choice and the jamming the paper reports."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import random_lattice

EMPTY, LR, TB = 0, 1, 2


def lr_wins(tie_seed, t, M, N, i, j):
    """The Model II coin of cell (i, j) at step t (the stated reading: one
    SplitMix64 output per 64-cell word and step, one bit per cell)."""
    W = (N + 63) // 64
    n = t * M * W + i * W + j // 64 + 1
    return (oracle.splitmix64(tie_seed, n) >> (j % 64)) & 1


def carlist_step(g, model, tie_seed, t):
    """One step from the rule statement: every vehicle looks at the state at
    the start of the step; it may move into its target if the target holds
    no vehicle; a target wanted by one LR and one TB vehicle goes to one of
    them by the coin."""
    M, N = g.shape
    lr = {(i, j) for i in range(M) for j in range(N) if g[i, j] & LR}
    tb = {(i, j) for i in range(M) for j in range(N) if g[i, j] & TB}
    occupied = lr | tb
    go_lr = {c: (c[0], (c[1] + 1) % N) for c in lr if (c[0], (c[1] + 1) % N) not in occupied}
    go_tb = {c: ((c[0] + 1) % M, c[1]) for c in tb if ((c[0] + 1) % M, c[1]) not in occupied}
    # Model II: a contested cell goes to one of its candidates; Model III:
    # it receives both
    contested = set(go_lr.values()) & set(go_tb.values()) if model == 2 else set()
    for x in contested:
        if lr_wins(tie_seed, t, M, N, *x):
            go_tb = {c: d for c, d in go_tb.items() if d != x}
        else:
            go_lr = {c: d for c, d in go_lr.items() if d != x}
    new_lr = {go_lr.get(c, c) for c in lr}
    new_tb = {go_tb.get(c, c) for c in tb}
    out = np.zeros_like(g)
    for c in new_lr:
        out[c] |= LR
    for c in new_tb:
        out[c] |= TB
    return out, len(go_lr), len(go_tb)


def carlist_run(g, K, model, tie_seed=0, t0=0):
    lrs, tbs = [], []
    for t in range(K):
        g, a, b = carlist_step(g, model, tie_seed, t0 + t)
        lrs.append(a)
        tbs.append(b)
    return g, np.array(lrs), np.array(tbs)


def shapes_upto(cells):
    return [(M, N) for M in range(1, cells + 1) for N in range(1, cells + 1) if M * N <= cells]


@pytest.mark.parametrize("model,cells,values", [(2, 7, 3), (3, 6, 4)])
def test_every_tiny_lattice_matches_carlist(model, cells, values):
    """Every lattice with M*N <= 7 cells (Model III: <= 6 cells, doubly
    occupied cells included), 3 steps, lattices and counts."""
    for M, N in shapes_upto(cells):
        for flat in itertools.product(range(values), repeat=M * N):
            g = np.array(flat, dtype=np.uint8).reshape(M, N)
            want = carlist_run(g, 3, model, tie_seed=11)
            got = oracle.run_model(g, 3, model, tie_seed=11)
            np.testing.assert_array_equal(got[0], want[0], err_msg=str((M, N, flat)))
            np.testing.assert_array_equal(got[1], want[1])
            np.testing.assert_array_equal(got[2], want[2])


@pytest.mark.parametrize("model", [2, 3])
@pytest.mark.parametrize("M,N", [(7, 9), (12, 70), (5, 130)])
def test_random_lattices_match_carlist(model, M, N):
    g = random_lattice(M, N, M * 31 + N, 0.2, 0.2)
    want = carlist_run(g, 6, model, tie_seed=5, t0=3)
    got = oracle.run_model(g, 6, model, tie_seed=5, t0=3)
    for a, b in zip(got, want):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("model", [2, 3])
@pytest.mark.parametrize("M,N", [(1, 9), (16, 16), (33, 65), (64, 200)])
def test_one_species_is_model_I(model, M, N):
    """With vehicles of one kind there is no contest and no phase
    interaction: Models II and III step exactly like Model I (pinned against
    the paper's rules elsewhere)."""
    for p_lr, p_tb in [(0.4, 0.0), (0.0, 0.4)]:
        g = random_lattice(M, N, 7 * M + N, p_lr, p_tb)
        want = oracle.run(g, 20)
        got = oracle.run_model(g, 20, model, tie_seed=3)
        for a, b in zip(got, want):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("model", [2, 3])
def test_conservation_and_counts(model):
    """LR vehicles per row and TB vehicles per column never change; every
    counted move fills a cell that held no vehicle of that kind."""
    M, N = 40, 70
    g = random_lattice(M, N, 99, 0.22, 0.22)
    for t in range(30):
        h, a, b = oracle.run_model(g, 1, model, tie_seed=8, t0=t)
        np.testing.assert_array_equal((h & LR).astype(bool).sum(1), (g & LR).astype(bool).sum(1))
        np.testing.assert_array_equal((h & TB).astype(bool).sum(0), (g & TB).astype(bool).sum(0))
        assert a[0] == ((h & LR) & ~(g & LR) & LR).astype(bool).sum()
        assert b[0] == ((h & TB) & ~(g & TB) & TB).astype(bool).sum()
        g = h


def test_model_II_contested_cells_get_exactly_one_vehicle_fairly():
    """Model II never doubles a cell; each contested empty cell receives
    exactly one of its two candidates, the LR one about half of the time."""
    M, N = 256, 256
    g = random_lattice(M, N, 1, 0.2, 0.2)
    won_lr = contests = 0
    for t in range(8):
        h, _, _ = oracle.run_model(g, 1, 2, tie_seed=1234, t0=t)
        assert np.all(h <= TB)
        empty = g == EMPTY
        from_left = np.roll(g, 1, axis=1) == LR
        from_top = np.roll(g, 1, axis=0) == TB
        contested = empty & from_left & from_top
        assert np.all((h[contested] == LR) | (h[contested] == TB))
        won_lr += int((h[contested] == LR).sum())
        contests += int(contested.sum())
        g = h
    assert contests > 2000
    assert abs(won_lr - contests / 2) < 5 * np.sqrt(contests / 4)


def test_model_II_step_index_composes():
    """The coins depend on the step index: K steps from t0 equal k steps from
    t0 followed by K-k steps from t0+k, and a different t0 changes the run."""
    g = random_lattice(50, 100, 23, 0.25, 0.25)
    a, alr, atb = oracle.run_model(g, 20, 2, tie_seed=9, t0=4)
    m, mlr, mtb = oracle.run_model(g, 7, 2, tie_seed=9, t0=4)
    b, blr, btb = oracle.run_model(m, 13, 2, tie_seed=9, t0=11)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(alr, np.concatenate([mlr, blr]))
    c, _, _ = oracle.run_model(g, 20, 2, tie_seed=9, t0=5)
    assert np.any(a != c)


@pytest.mark.parametrize("model", [2, 3])
def test_threads_do_not_change_results(model):
    g = random_lattice(97, 301, 24, 0.2, 0.2)
    a = oracle.run_model(g, 10, model, tie_seed=2, threads=1)
    b = oracle.run_model(g, 10, model, tie_seed=2, threads=4)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


def test_density_regimes():
    """The paper: the variant shows Model I's behaviour, free flow at low
    density and a global jam at high density.  On 64 x 64 (seeds 1-3, 3000
    steps): at density 0.05 every vehicle moves every step at the end; at
    density 0.2 the lattice reaches a step with no move (absorbing).  The
    transition lies at a lower density than Model I's (which flows freely
    at 0.2)."""
    for seed in (1, 2, 3):
        g = random_lattice(64, 64, seed, 0.025, 0.025)
        _, a, b = oracle.run_model(g, 3000, 2, tie_seed=seed)
        assert np.all(a[-128:] + b[-128:] == int((g > 0).sum()))
        g = random_lattice(64, 64, seed, 0.1, 0.1)
        _, a, b = oracle.run_model(g, 3000, 2, tie_seed=seed)
        assert a[-1] + b[-1] == 0
        _, a1, b1 = oracle.run(g, 3000)
        assert a1[-1] + b1[-1] > 0


def test_model_III_worked_example():
    """The hand-worked 4 x 4 example (tests/golden/worked_model3_4x4.txt):
    every state and both counts of every step."""
    import os
    from paper_1804_07981_b300.inputs import parse_golden
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                        "worked_model3_4x4.txt")
    shape, blocks = parse_golden(path)
    g = blocks[0][2]
    assert g.shape == shape and blocks[0][0] == "t0"
    for label, (lr, tb), want in blocks[1:]:
        g, a, b = oracle.run_model(g, 1, 3)
        np.testing.assert_array_equal(g, want, err_msg=label)
        assert (a[0], b[0]) == (lr, tb), label
    final, a, b = oracle.run_model(blocks[0][2], len(blocks) - 1, 3)
    np.testing.assert_array_equal(final, blocks[-1][2])
    assert list(zip(a, b)) == [blk[1] for blk in blocks[1:]]


def _transpose_swap(g):
    """Transpose the lattice and swap the kinds (LR <-> TB)."""
    t = np.ascontiguousarray(g.T)
    return ((t & LR) << 1 | (t & TB) >> 1).astype(np.uint8)


def test_model_III_transpose_duality():
    """Model III has one synchronous phase, symmetric in the two kinds:
    transposing the lattice and swapping LR with TB commutes with a step,
    with the two counts exchanged (Model I's alternating phases break this
    symmetry)."""
    rng = np.random.Generator(np.random.PCG64(17))
    for M, N in [(9, 13), (32, 45), (1, 7)]:
        g = rng.integers(0, 4, size=(M, N), dtype=np.uint8)
        a, alr, atb = oracle.run_model(g, 12, 3)
        b, blr, btb = oracle.run_model(_transpose_swap(g), 12, 3)
        np.testing.assert_array_equal(_transpose_swap(a), b)
        np.testing.assert_array_equal(alr, btb)
        np.testing.assert_array_equal(atb, blr)


def test_model_III_contested_cells_receive_both():
    """Every empty cell with an LR vehicle on its left and a TB vehicle above
    holds one of each after the step; no other cell becomes doubly occupied
    except by keeping its vehicles."""
    g = random_lattice(128, 128, 5, 0.2, 0.2)
    for t in range(6):
        h, _, _ = oracle.run_model(g, 1, 3)
        empty = g == EMPTY
        from_left = (np.roll(g, 1, axis=1) & LR) > 0
        from_top = (np.roll(g, 1, axis=0) & TB) > 0
        both = empty & from_left & from_top
        assert both.sum() > 0
        assert np.all(h[both] == LR | TB)
        new_double = (h == (LR | TB)) & (g != (LR | TB))
        np.testing.assert_array_equal(new_double, both)
        g = h


def test_model_III_rejects_bytes_above_3():
    g = np.zeros((3, 3), dtype=np.uint8)
    g[1, 1] = 4
    with pytest.raises(RuntimeError):
        oracle.run_model(g, 1, 3)


def test_model_III_reading_flows_where_model_I_jams():
    """What this reading gives (the paper states that Model III behaves like
    Model I; this reading does not): at densities where Model I jams on
    64 x 64, vehicles still move after 3000 steps, because every contested
    cell absorbs both vehicles and frees two cells."""
    for seed in (1, 2):
        g = random_lattice(64, 64, seed, 0.3, 0.3)
        _, a1, b1 = oracle.run(g, 3000)
        assert a1[-1] + b1[-1] == 0          # Model I: globally jammed
        _, a3, b3 = oracle.run_model(g, 3000, 3)
        assert a3[-64:].min() + b3[-64:].min() > 0
