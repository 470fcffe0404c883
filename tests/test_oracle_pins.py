"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
not by the oracle itself (CPU only).

- hand-worked examples (tests/golden/), derived from the two rules of Sec. 2;
- exhaustive enumeration of every lattice with M*N <= 12 cells against an
  independent car-list formulation of the same rules;
- conservation laws, bounds, absorbing fixed points;
- symmetries: translation equivariance, the transpose duality of the phases;
- special cases: a lone car, a full lattice, and an LR-only lattice, which is
  M independent rings of elementary CA rule 184 with the textbook steady flux
  min(n, N - n);
- the initial placement: the published SplitMix64 sequence and the sampling
  frequencies.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import all_lattices, parse_golden, random_lattice

EMPTY, LR, TB = 0, 1, 2
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------
# An independent formulation: move cars, not cells.  For each phase, list the
# cars of the moving kind, decide for each one whether the cell ahead (with
# wrap) is empty in the state before the phase, then build the new lattice
# by placing every car at its source or destination.
# --------------------------------------------------------------------------
def carlist_phase(g: np.ndarray, kind: int):
    """g: (C, M, N) batch.  Returns (new batch, moved per lattice)."""
    C, M, N = g.shape
    cars = g == kind
    if kind == LR:
        ahead_empty = np.roll(g, -1, axis=2) == EMPTY  # cell (i, j+1)
    else:
        ahead_empty = np.roll(g, -1, axis=1) == EMPTY  # cell (i+1, j)
    go = cars & ahead_empty
    stay = cars & ~go
    out = np.where(cars, EMPTY, g).astype(np.uint8)
    out[stay] = kind
    if kind == LR:
        dest = np.roll(go, 1, axis=2)
    else:
        dest = np.roll(go, 1, axis=1)
    assert not np.any(out[dest] != EMPTY), "destination occupied"
    out[dest] = kind
    return out, go.reshape(C, -1).sum(axis=1).astype(np.int64)


def carlist_run(g: np.ndarray, K: int):
    g = g.copy()
    mlr, mtb = [], []
    for _ in range(K):
        g, a = carlist_phase(g, LR)
        g, b = carlist_phase(g, TB)
        mlr.append(a)
        mtb.append(b)
    return g, np.stack(mlr, 1), np.stack(mtb, 1)


def scalar_carlist_step(g: np.ndarray):
    """Pure-Python car list, one step of a single lattice (small cases)."""
    M, N = g.shape
    h = g.copy()
    lr = [(i, j) for i in range(M) for j in range(N) if g[i, j] == LR]
    movers = [(i, j) for (i, j) in lr if g[i, (j + 1) % N] == EMPTY]
    for (i, j) in movers:
        h[i, j] = EMPTY
    for (i, j) in movers:
        h[i, (j + 1) % N] = LR
    v = h.copy()
    tb = [(i, j) for i in range(M) for j in range(N) if h[i, j] == TB]
    movers2 = [(i, j) for (i, j) in tb if h[(i + 1) % M, j] == EMPTY]
    for (i, j) in movers2:
        v[i, j] = EMPTY
    for (i, j) in movers2:
        v[(i + 1) % M, j] = TB
    return v, len(movers), len(movers2)


# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["worked_4x4.txt", "worked_5x3.txt"])
def test_worked_examples(name):
    shape, blocks = parse_golden(os.path.join(GOLDEN, name))
    assert blocks[0][0] == "t0"
    g = blocks[0][2]
    assert g.shape == shape
    phases = blocks[1:]
    assert len(phases) % 2 == 0
    for idx in range(0, len(phases), 2):
        (lh, mh, gh), (lv, mv, gv) = phases[idx], phases[idx + 1]
        assert lh.startswith("H") and lv.startswith("V")
        h, moved_h = oracle.phase(g, 0)
        np.testing.assert_array_equal(h, gh, err_msg=lh)
        assert moved_h == mh, lh
        v, moved_v = oracle.phase(h, 1)
        np.testing.assert_array_equal(v, gv, err_msg=lv)
        assert moved_v == mv, lv
        g = v
    # the full-step driver agrees with the phase-by-phase walk
    final, mlr, mtb = oracle.run(blocks[0][2], len(phases) // 2)
    np.testing.assert_array_equal(final, phases[-1][2])
    assert list(mlr) == [b[1] for b in phases[0::2]]
    assert list(mtb) == [b[1] for b in phases[1::2]]


def test_worked_example_rejects_swapped_phase_order():
    """Running V before H on example B gives a different lattice after one
    step, so the fixture really pins the order."""
    _, blocks = parse_golden(os.path.join(GOLDEN, "worked_5x3.txt"))
    g0 = blocks[0][2]
    v, _ = oracle.phase(g0, 1)
    vh, _ = oracle.phase(v, 0)
    assert not np.array_equal(vh, blocks[2][2])


SHAPES_EXHAUSTIVE = [(M, N) for M in range(1, 13) for N in range(1, 13) if M * N <= 12]


@pytest.mark.parametrize("M,N", SHAPES_EXHAUSTIVE)
def test_exhaustive_tiny_lattices(M, N):
    """Every configuration of every lattice with at most 12 cells, 3 steps,
    oracle vs the car-list formulation: lattices and per-step counts."""
    gs = all_lattices(M, N)
    K = 3
    og, olr, otb = oracle.run_batch(gs, K)
    cg, clr, ctb = carlist_run(gs, K)
    np.testing.assert_array_equal(og, cg)
    np.testing.assert_array_equal(olr, clr)
    np.testing.assert_array_equal(otb, ctb)


@pytest.mark.parametrize("M,N,seed", [(7, 9, 1), (16, 13, 2), (5, 64, 3), (11, 65, 4)])
def test_scalar_carlist_random(M, N, seed):
    g = random_lattice(M, N, seed, 0.25, 0.2)
    K = 12
    og, olr, otb = oracle.run(g, K)
    h = g.copy()
    for t in range(K):
        h, a, b = scalar_carlist_step(h)
        assert a == olr[t] and b == otb[t]
    np.testing.assert_array_equal(og, h)


@pytest.mark.parametrize("M,N,rho,seed", [(33, 63, 0.3, 1), (40, 64, 0.38, 2),
                                          (17, 65, 0.5, 3), (64, 129, 0.2, 4),
                                          (9, 2047, 0.35, 5)])
def test_conservation_and_bounds(M, N, rho, seed):
    g = random_lattice(M, N, seed, rho / 2, rho / 2)
    lr_rows = (g == LR).sum(axis=1)
    tb_cols = (g == TB).sum(axis=0)
    n_lr, n_tb = int((g == LR).sum()), int((g == TB).sum())
    cur = g
    for _ in range(6):
        nxt, mlr, mtb = oracle.run(cur, 1)
        np.testing.assert_array_equal((nxt == LR).sum(axis=1), lr_rows)
        np.testing.assert_array_equal((nxt == TB).sum(axis=0), tb_cols)
        assert 0 <= mlr[0] <= n_lr and 0 <= mtb[0] <= n_tb
        # moved LR = number of LR cells that appear where there was none
        h, moved_h = oracle.phase(cur, 0)
        assert moved_h == int(((h == LR) & (cur != LR)).sum()) == mlr[0]
        v, moved_v = oracle.phase(h, 1)
        assert moved_v == int(((v == TB) & (h != TB)).sum()) == mtb[0]
        np.testing.assert_array_equal(v, nxt)
        cur = nxt


@pytest.mark.parametrize("M,N,rho,seed", [(16, 64, 0.3, 1), (9, 65, 0.5, 2), (33, 130, 0.7, 3),
                                          (5, 2, 0.6, 4)])
def test_horizontally_adjacent_cars_never_both_move(M, N, rho, seed):
    """A car cannot move while the cell to its right holds a car, so in the
    horizontal phase the cars of columns j and j + 1 (mod N) never both
    move (the GPU kernels count the two interleaved move masks of a column
    pair with one popcount because of this)."""
    cur = random_lattice(M, N, seed, rho / 2, rho / 2)
    total = 0
    for _ in range(8):
        h, moved = oracle.phase(cur, 0)
        mv = (cur == LR) & (h != LR)  # the cars that left their cell
        assert int(mv.sum()) == moved
        assert not (mv & np.roll(mv, -1, axis=1)).any()
        total += moved
        cur, _ = oracle.phase(h, 1)
    assert total > 0


@pytest.mark.parametrize("M,N", [(12, 63), (9, 64), (10, 65), (6, 127), (5, 129), (3, 2047)])
def test_translation_equivariance(M, N):
    g = random_lattice(M, N, M * 1000 + N, 0.2, 0.2)
    K = 20
    base, blr, btb = oracle.run(g, K)
    for di, dj in [(1, 0), (0, 1), (3, 7 % N), (M - 1, N - 1)]:
        s = np.roll(g, (di, dj), axis=(0, 1))
        out, slr, stb = oracle.run(s, K)
        np.testing.assert_array_equal(out, np.roll(base, (di, dj), axis=(0, 1)))
        np.testing.assert_array_equal(slr, blr)
        np.testing.assert_array_equal(stb, btb)


@pytest.mark.parametrize("K", [1, 2, 4, 8])
def test_light_cone_of_a_false_junction(K):
    """A cell's state after K steps depends only on the cells within K
    columns of it (Sec. 2: a car moves at most one cell per phase, and a
    cell's phase reads only its neighbours).  So a row ring assembled from
    pieces of the lattice that are not neighbours -- 64 columns right of a
    strip of 128-column pairs, then 64 columns left of it, then the strip,
    as the two-words-per-lane kernel's halo lane holds them -- gives every
    strip cell exactly after K <= 8 steps.  The cone is exactly K columns:
    pieces K columns wide still give the strip exactly, pieces K - 1
    columns wide do not (on this lattice)."""
    M, P = 48, 12                      # rows; the lattice is P pairs of 128 columns wide
    g = random_lattice(M, 128 * P, 17 + K, 0.19, 0.19)
    want, _, _ = oracle.run(g, K)
    first, n_own = 3, 5                # the strip: pairs 3..7
    right = np.arange(64) + 128 * (first + n_own)
    left = np.arange(64, 128) + 128 * (first - 1)
    strip = np.arange(128 * first, 128 * (first + n_own))
    cols = np.concatenate([right, left, strip])
    got, _, _ = oracle.run(np.ascontiguousarray(g[:, cols]), K)
    np.testing.assert_array_equal(got[:, 128:], want[:, strip])
    for w, exact in ((K, True), (K - 1, False)):
        ring = np.concatenate([right[:w], left[64 - w:], strip])
        out, _, _ = oracle.run(np.ascontiguousarray(g[:, ring]), K)
        assert np.array_equal(out[:, 2 * w:], want[:, strip]) == exact, w


def _swap_kinds(g):
    out = g.copy()
    out[g == LR] = TB
    out[g == TB] = LR
    return out


@pytest.mark.parametrize("M,N,seed", [(8, 13, 1), (31, 70, 2)])
def test_transpose_duality(M, N, seed):
    """H on g equals, transposed with kinds swapped, V on the transposed,
    kind-swapped lattice."""
    g = random_lattice(M, N, seed, 0.2, 0.25)
    h, mh = oracle.phase(g, 0)
    d = _swap_kinds(g.T.copy())
    v, mv = oracle.phase(d, 1)
    np.testing.assert_array_equal(_swap_kinds(v.T.copy()), h)
    assert mh == mv


@pytest.mark.parametrize("M,N", [(1, 1), (3, 5), (7, 64), (4, 130)])
def test_lone_car(M, N):
    g = np.zeros((M, N), dtype=np.uint8)
    g[M // 2, N // 3] = LR
    K = 2 * N + 3
    out, mlr, mtb = oracle.run(g, K)
    expect = np.zeros_like(g)
    if N > 1:
        expect[M // 2, (N // 3 + K) % N] = LR
        assert np.all(mlr == 1)
    else:
        expect[M // 2, 0] = LR  # its right neighbour is itself: never moves
        assert np.all(mlr == 0)
    assert np.all(mtb == 0)
    np.testing.assert_array_equal(out, expect)

    g = np.zeros((M, N), dtype=np.uint8)
    g[M // 3, N // 2] = TB
    K = 2 * M + 1
    out, mlr, mtb = oracle.run(g, K)
    expect = np.zeros_like(g)
    expect[(M // 3 + K) % M if M > 1 else 0, N // 2] = TB
    np.testing.assert_array_equal(out, expect)
    assert np.all(mtb == (1 if M > 1 else 0)) and np.all(mlr == 0)


def test_full_lattice_frozen():
    g = random_lattice(20, 30, 7, 0.5, 0.5)
    g[g == EMPTY] = LR
    out, mlr, mtb = oracle.run(g, 5)
    np.testing.assert_array_equal(out, g)
    assert mlr.sum() == 0 and mtb.sum() == 0
    # rows without any empty cell freeze their LR cars
    g2 = random_lattice(6, 10, 8, 0.3, 0.3)
    g2[2, :] = LR
    h, _ = oracle.phase(g2, 0)
    np.testing.assert_array_equal(h[2], g2[2])


def test_absorbing_fixed_point():
    """Once a step moves no car, the lattice never changes again."""
    g = random_lattice(24, 24, 11, 0.3, 0.3)  # rho = 0.6 jams fast
    out, mlr, mtb = oracle.run(g, 400)
    tot = mlr + mtb
    zeros = np.flatnonzero(tot == 0)
    assert zeros.size > 0, "expected a jam at rho = 0.6"
    t0 = zeros[0]
    assert np.all(tot[t0:] == 0)
    frozen, _, _ = oracle.run(g, t0 + 1)
    np.testing.assert_array_equal(frozen, out)
    again, a, b = oracle.run(frozen, 3)
    np.testing.assert_array_equal(again, frozen)
    assert a.sum() == 0 and b.sum() == 0


@pytest.mark.parametrize("N,seed", [(50, 1), (64, 2), (97, 3)])
def test_rule184_steady_flux(N, seed):
    """LR-only rows are independent rings of rule 184.  After the transient
    (at most N steps) the number of cars moving per step on a ring with n
    cars is min(n, N - n), i.e. velocity min(1, (1 - rho)/rho)."""
    M = 24
    rng = np.random.Generator(np.random.PCG64(seed))
    g = np.zeros((M, N), dtype=np.uint8)
    counts = rng.integers(0, N + 1, size=M)
    for i, n in enumerate(counts):
        g[i, rng.permutation(N)[:n]] = LR
    K = 2 * N
    _, mlr, mtb = oracle.run(g, K)
    assert np.all(mtb == 0)
    expect = int(np.minimum(counts, N - counts).sum())
    assert np.all(mlr[N:] == expect)


def test_splitmix64_published_sequence():
    """SplitMix64 from state 1234567: the first five outputs as published
    with the generator's reference code."""
    published = [6457827717110365317, 3203168211198807973, 9817491932198370423,
                 4593380528125082431, 16408922859458223821]
    assert [oracle.splitmix64(1234567, n) for n in range(1, 6)] == published


def test_thresholds():
    assert oracle.threshold(0.0) == 0
    assert oracle.threshold(1.0) == 2 ** 64 - 1
    assert oracle.threshold(0.5) == 2 ** 63
    assert oracle.threshold(0.25) == 2 ** 62
    assert oracle.threshold(0.15) == int(0.15 * 2 ** 64)


def test_init_definition_and_frequencies():
    M, N, seed = 200, 300, 1
    p_lr, p_tb = 0.15, 0.2
    g = oracle.init(M, N, seed, p_lr, p_tb)
    # a few cells re-derived one by one from the placement rule
    t_lr, t_tb = oracle.threshold(p_lr), oracle.threshold(p_tb)
    for (i, j) in [(0, 0), (0, 1), (17, 299), (199, 123)]:
        u = oracle.splitmix64(seed, i * N + j + 1)
        want = LR if u < t_lr else (TB if u - t_lr < t_tb else EMPTY)
        assert g[i, j] == want
    n = M * N
    for val, p in [(LR, p_lr), (TB, p_tb), (EMPTY, 1 - p_lr - p_tb)]:
        k = int((g == val).sum())
        assert abs(k - n * p) <= 5 * np.sqrt(n * p * (1 - p)), val
    # density 1 split evenly fills the lattice; density 0 leaves it empty
    assert not np.any(oracle.init(8, 8, 3, 0.5, 0.5) == EMPTY)
    assert not np.any(oracle.init(8, 8, 3, 0.0, 0.0))


def test_init_window_is_the_wrapped_slice_of_the_placement():
    """A window of the seeded placement (used for lattices too large to hold)
    equals the wrapped slice of the whole lattice, across both seams; cells
    re-derived one by one from the rule agree."""
    M, N, seed, p_lr, p_tb = 37, 53, 5, 0.2, 0.3
    g = oracle.init(M, N, seed, p_lr, p_tb)
    for i0, j0, R, C in [(30, 40, 20, 25), (0, 0, M, N), (36, 52, 3, 4), (5, 7, 80, 120)]:
        w = oracle.init_window(i0, j0, R, C, M, N, seed, p_lr, p_tb)
        rows = (np.arange(R) + i0) % M
        cols = (np.arange(C) + j0) % N
        np.testing.assert_array_equal(w, g[np.ix_(rows, cols)])
    # a window of a lattice too large to build: cells from the rule directly
    M, N = 1 << 20, 1 << 20
    t_lr, t_tb = oracle.threshold(p_lr), oracle.threshold(p_tb)
    w = oracle.init_window(M - 2, N - 3, 4, 5, M, N, seed, p_lr, p_tb)
    for a in range(4):
        for b in range(5):
            i, j = (M - 2 + a) % M, (N - 3 + b) % N
            u = oracle.splitmix64(seed, i * N + j + 1)
            assert w[a, b] == (LR if u < t_lr else (TB if u - t_lr < t_tb else EMPTY))


def test_threaded_oracle_identical():
    g = random_lattice(257, 300, 5, 0.19, 0.19)
    a, alr, atb = oracle.run(g, 25, threads=1)
    b, blr, btb = oracle.run(g, 25, threads=4)
    np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(alr, blr)
    np.testing.assert_array_equal(atb, btb)


def test_phase_transition_sanity():
    """Statistical sanity (Sec. 2, Fig. 1): at 256^2 and 4096 steps, rho=0.25
    is free-flowing (mean velocity over the last 64 steps above 0.95) and
    rho=0.5 is globally jammed (no car moves)."""
    g = oracle.init(256, 256, 1, 0.125, 0.125)
    _, mlr, mtb = oracle.run(g, 4096, threads=4)
    cars = int((g != EMPTY).sum())
    assert (mlr[-64:] + mtb[-64:]).mean() / cars > 0.95
    g = oracle.init(256, 256, 1, 0.25, 0.25)
    _, mlr, mtb = oracle.run(g, 4096, threads=4)
    assert mlr[-1] + mtb[-1] == 0
