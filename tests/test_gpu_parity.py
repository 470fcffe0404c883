"""GPU parity of every step kernel against the CPU oracle, through the C ABI.

The automaton is integer: lattices and per-step moved counts must match the
oracle bit for bit.  Shapes are chosen to cover one word and many words per
row, whole-warp rows and multi-strip rows, every tail length class (N mod 64
= 0, 1, 63, other), rows that need the two-word halo, several row bands with
a ragged last band, and the degenerate 1-row / 1-column / 1-cell lattices.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import parse_golden, random_lattice

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

KERNEL_CASES = [
    ("byte", 0), ("bitplane", 0), ("fused", 0),
    ("tblock", 1), ("tblock", 2), ("tblock", 4), ("tblock", 8), ("auto", 0), ("resident", 0),
]

SHAPES = [
    (1, 1), (1, 2), (2, 1), (1, 70), (70, 1), (3, 3), (5, 64), (7, 63), (9, 65),
    (33, 127), (17, 129), (130, 200), (64, 2047), (40, 2048), (31, 2049),
    (23, 2100), (29, 4097), (19, 4160), (300, 1000),
]


def make(lib, M, N, kernel, block_k, seed=1, p_lr=0.15, p_tb=0.15):
    return lib.Lattice(M, N, seed=seed, p_lr=p_lr, p_tb=p_tb, kernel=kernel, block_k=block_k)


def oracle_counts_equal(sim_counts, mlr, mtb):
    tot, lr, tb = sim_counts
    np.testing.assert_array_equal(lr, mlr)
    np.testing.assert_array_equal(tb, mtb)
    np.testing.assert_array_equal(tot, mlr + mtb)


@pytest.mark.parametrize("kernel,block_k", [("byte", 0), ("fused", 0)])
@pytest.mark.parametrize("M,N", [(256, 256), (37, 65), (5, 1), (1, 200), (100, 2047), (3, 4100)])
def test_seeded_placement_matches_oracle(lib, kernel, block_k, M, N):
    for seed, p_lr, p_tb in [(1, 0.15, 0.15), (7, 0.3, 0.1), (123456789, 0.5, 0.5), (2, 0.0, 1.0)]:
        with make(lib, M, N, kernel, block_k, seed, p_lr, p_tb) as sim:
            np.testing.assert_array_equal(sim.read(), oracle.init(M, N, seed, p_lr, p_tb))


@pytest.mark.parametrize("kernel,block_k", KERNEL_CASES)
@pytest.mark.parametrize("M,N", SHAPES)
def test_random_lattices_match_oracle(lib, kernel, block_k, M, N):
    K = 37  # not a multiple of any block depth: exercises the remainders
    for seed, rho in [(M * 7919 + N, 0.3), (M + 3 * N, 0.6)]:
        g0 = random_lattice(M, N, seed, rho / 2, rho / 2)
        with make(lib, M, N, kernel, block_k) as sim:
            sim.write(g0)
            np.testing.assert_array_equal(sim.read(), g0)
            sim.step(10)
            sim.step(K - 10)
            want, mlr, mtb = oracle.run(g0, K)
            np.testing.assert_array_equal(sim.read(), want)
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)
            assert sim.steps_done == K


@pytest.mark.parametrize("kernel,block_k", KERNEL_CASES)
def test_config_256_density_03_1024_steps(lib, kernel, block_k):
    """256 x 256, each cell LR w.p. 0.15 and TB w.p. 0.15, seed 1, 1024 steps:
    final lattice and every per-step count."""
    M = N = 256
    with make(lib, M, N, kernel, block_k, 1, 0.15, 0.15) as sim:
        g0 = oracle.init(M, N, 1, 0.15, 0.15)
        np.testing.assert_array_equal(sim.read(), g0)
        sim.step(1024)
        want, mlr, mtb = oracle.run(g0, 1024)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)


@pytest.mark.parametrize("kernel,block_k", KERNEL_CASES)
@pytest.mark.parametrize("name", ["worked_4x4.txt", "worked_5x3.txt"])
def test_worked_examples_on_gpu(lib, kernel, block_k, name):
    shape, blocks = parse_golden(os.path.join(GOLDEN, name))
    g0 = blocks[0][2]
    states = [b[2] for b in blocks[2::2]]  # lattice after each full step
    with make(lib, shape[0], shape[1], kernel, block_k) as sim:
        sim.write(g0)
        for t, want in enumerate(states):
            sim.step(1)
            np.testing.assert_array_equal(sim.read(), want)
        tot, lr, tb = sim.moved_counts()
        assert list(lr) == [b[1] for b in blocks[1::2]]
        assert list(tb) == [b[1] for b in blocks[2::2]]


@pytest.mark.parametrize("kernel,block_k", [("byte", 0), ("tblock", 8), ("auto", 0)])
def test_checkpoint_resume(lib, kernel, block_k):
    M, N, k = 90, 333, 25
    with make(lib, M, N, kernel, block_k, 5, 0.18, 0.2) as a:
        a.step(2 * k)
        full = a.read()
        _, lr_full, tb_full = a.moved_counts()
    with make(lib, M, N, kernel, block_k, 5, 0.18, 0.2) as b:
        b.step(k)
        mid = b.read()
    with make(lib, M, N, kernel, block_k, 99, 0.3, 0.3) as c:
        c.write(mid)
        assert c.steps_done == 0
        c.step(k)
        np.testing.assert_array_equal(c.read(), full)
        _, lr2, tb2 = c.moved_counts()
        np.testing.assert_array_equal(lr2, lr_full[k:])
        np.testing.assert_array_equal(tb2, tb_full[k:])


@pytest.mark.parametrize("kernel,block_k", [("byte", 0), ("fused", 0), ("tblock", 4)])
def test_invalid_lattice_rejected_and_state_kept(lib, kernel, block_k):
    M, N = 20, 70
    with make(lib, M, N, kernel, block_k, 3, 0.2, 0.2) as sim:
        sim.step(5)
        before = sim.read()
        bad = before.copy()
        bad[7, 13] = 3
        with pytest.raises(lib.BMLError) as e:
            sim.write(bad)
        assert e.value.code == lib.BML_EINVAL
        np.testing.assert_array_equal(sim.read(), before)
        assert sim.steps_done == 5


def test_count_range_errors(lib):
    with make(lib, 16, 16, "fused", 0) as sim:
        sim.step(3)
        with pytest.raises(lib.BMLError):
            lib.bml_moved_counts(sim.handle, 2, 5)
        with pytest.raises(lib.BMLError):
            lib.bml_moved_counts(sim.handle, -1, 1)
        tot, _, _ = lib.bml_moved_counts(sim.handle, 1, 2)
        assert tot.shape == (2,)


def test_async_counts_equal_synchronous_counts(lib):
    """Counts copied without waiting (into page-locked host memory, read
    after a synchronise) equal the synchronous read, across history growth."""
    import torch
    M, N = 40, 300
    with lib.Lattice(M, N, seed=2, density=0.3, kernel="tblock", block_k=4,
                     reserve_steps=16) as sim:
        lr = torch.zeros(200, dtype=torch.int64, pin_memory=True).numpy()
        tb = torch.zeros(200, dtype=torch.int64, pin_memory=True).numpy()
        for s in range(20):
            sim.step(10)
            lib.bml_moved_counts_async(sim.handle, 10 * s, 10, lr[10 * s:10 * s + 10],
                                       tb[10 * s:10 * s + 10])
        sim.synchronize()
        tot, a, b = sim.moved_counts()
        np.testing.assert_array_equal(lr, a)
        np.testing.assert_array_equal(tb, b)
        with pytest.raises(lib.BMLError):
            lib.bml_moved_counts_async(sim.handle, 195, 10, lr[:10], tb[:10])


@pytest.mark.parametrize("memory", ["pinned", "pageable", "pinned_lr_only"])
def test_async_counts_every_host_memory_kind(lib, memory):
    """Page-locked arrays are written by the dependent copy kernel, pageable
    ones by cudaMemcpyAsync; both give the synchronous counts, with either
    output omitted as well."""
    import torch
    M, N = 64, 640
    with lib.Lattice(M, N, seed=3, density=0.35, kernel="tblock", block_k=8,
                     reserve_steps=400) as sim:
        if memory == "pageable":
            lr = np.zeros(320, dtype=np.int64)
            tb = np.zeros(320, dtype=np.int64)
        else:
            lr = torch.zeros(320, dtype=torch.int64, pin_memory=True).numpy()
            tb = torch.zeros(320, dtype=torch.int64, pin_memory=True).numpy()
        for s in range(40):
            sim.step(8)
            lib.bml_moved_counts_async(sim.handle, 8 * s, 8, lr[8 * s:8 * s + 8],
                                       None if memory == "pinned_lr_only" else tb[8 * s:8 * s + 8])
        sim.synchronize()
        _, a, b = sim.moved_counts()
        np.testing.assert_array_equal(lr, a)
        if memory == "pinned_lr_only":
            assert not tb.any()
        else:
            np.testing.assert_array_equal(tb, b)


def test_count_history_grows(lib):
    M, N = 24, 100
    with lib.Lattice(M, N, seed=4, density=0.3, kernel="tblock", block_k=8,
                     reserve_steps=16) as sim:
        g0 = sim.read()
        sim.step(5000)  # forces several reallocations of the history
        want, mlr, mtb = oracle.run(g0, 5000)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)


def test_device_read_write_with_torch_memory(lib):
    import torch
    M, N = 123, 321
    g0 = random_lattice(M, N, 77, 0.2, 0.2)
    d_in = torch.from_numpy(g0).cuda()
    d_out = torch.empty((M, N), dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    with make(lib, M, N, "tblock", 2) as sim:
        lib.bml_write_lattice_device(sim.handle, d_in.data_ptr())
        sim.step(11)
        lib.bml_read_lattice_device(sim.handle, d_out.data_ptr())
        sim.synchronize()
        want, _, _ = oracle.run(g0, 11)
        np.testing.assert_array_equal(d_out.cpu().numpy(), want)


def test_torch_caching_allocator_owns_device_memory(lib):
    import torch
    lib.use_torch_allocator(True)
    try:
        before = torch.cuda.memory_allocated()
        M, N = 512, 1000
        with lib.Lattice(M, N, seed=9, density=0.35, kernel="tblock", block_k=4) as sim:
            assert torch.cuda.memory_allocated() > before + M * N // 4
            g0 = oracle.init(M, N, 9, 0.175, 0.175)
            sim.step(40)
            want, mlr, mtb = oracle.run(g0, 40)
            np.testing.assert_array_equal(sim.read(), want)
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)
        assert torch.cuda.memory_allocated() == before
    finally:
        lib.use_torch_allocator(False)


def test_user_stream(lib):
    import torch
    s = torch.cuda.Stream()
    M, N = 64, 640
    with lib.Lattice(M, N, seed=2, density=0.3, kernel="fused", stream=s) as sim:
        g0 = oracle.init(M, N, 2, 0.15, 0.15)
        sim.step(9)
        want, mlr, mtb = oracle.run(g0, 9)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)


@pytest.mark.parametrize("M,N", [(130, 200), (77, 4097), (300, 2100), (64, 64), (5, 129)])
def test_explicit_tilings_match_oracle(lib, M, N):
    """Every temporal depth with band heights that do not divide M, bands
    shorter than the depth, one band, and the one-pass fused kernel."""
    g0 = random_lattice(M, N, M + N, 0.17, 0.19)
    K = 19
    want, mlr, mtb = oracle.run(g0, K)
    tilings = [(1, 0)] + [(k, b) for k in (1, 2, 4, 8) for b in (1, 3, 16, 37, M)]
    for k, band in tilings:
        with make(lib, M, N, "tblock", k) as sim:
            sim.set_tiling(k, band)
            sim.write(g0)
            sim.step(K)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)
            assert sim.config[1:] == (k, band)


def test_resident_kernel_long_calls(lib):
    """The resident kernel runs a call's steps in launches of up to 4096:
    5000 steps in one call, then 3 more; lattice and every count."""
    M, N = 48, 200
    g0 = random_lattice(M, N, 5, 0.15, 0.15)
    want, mlr, mtb = oracle.run(g0, 5003)
    with make(lib, M, N, "resident", 0) as sim:
        assert sim.config[0] == lib.BML_KERNEL_RESIDENT
        assert sim.tiling == (0, M, 0)
        sim.write(g0)
        sim.step(5000)
        sim.step(3)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)
        with pytest.raises(lib.BMLError):
            sim.set_tiling(1, 16)


RESIDENT_CLUSTER_SHAPES = [(2, 64), (3, 3), (8, 65), (9, 70), (33, 127), (100, 300),
                           (256, 256), (64, 2000), (17, 2048)]


@pytest.mark.parametrize("blocks", [2, 4, 8])
@pytest.mark.parametrize("M,N", RESIDENT_CLUSTER_SHAPES)
def test_resident_cluster_matches_oracle(lib, M, N, blocks):
    """The resident kernel with the rows split over a cluster of 2, 4 or 8
    blocks (bands of ceil(M / blocks) rows, the last one shorter, rows next
    to a band read from the neighbouring block's shared memory) gives the
    oracle's lattices and counts; more blocks than rows are refused."""
    with make(lib, M, N, "resident", 0) as sim:
        if blocks > M:
            with pytest.raises(lib.BMLError):
                sim.set_resident_blocks(blocks)
            return
        sim.set_resident_blocks(blocks)
        assert sim.tiling == (0, -(-M // blocks), 0)
        for seed, rho in [(M * 31 + N, 0.3), (M + 5 * N, 0.7)]:
            g0 = random_lattice(M, N, seed, rho / 2, rho / 2)
            sim.write(g0)
            sim.step(37)
            sim.step(5)
            want, mlr, mtb = oracle.run(g0, 42)
            np.testing.assert_array_equal(sim.read(), want)
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)


def test_resident_cluster_long_calls_and_rejections(lib):
    """5003 steps over a cluster of 4 blocks (two launches); the call is
    refused for objects that do not run the resident kernel and for block
    counts other than 1, 2, 4, 8."""
    M, N = 48, 200
    g0 = random_lattice(M, N, 6, 0.2, 0.2)
    want, mlr, mtb = oracle.run(g0, 5003)
    with make(lib, M, N, "resident", 0) as sim:
        sim.set_resident_blocks(4)
        sim.write(g0)
        sim.step(5000)
        sim.step(3)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)
        for bad in (0, 3, 16, -1):
            with pytest.raises(lib.BMLError):
                sim.set_resident_blocks(bad)
        sim.set_resident_blocks(1)
        assert sim.tiling == (0, M, 0)
    with make(lib, M, N, "tblock", 4) as sim:
        with pytest.raises(lib.BMLError):
            sim.set_resident_blocks(2)


def test_set_tiling_rejects_bad_values(lib):
    with make(lib, 32, 64, "tblock", 2) as sim:
        for k, band in [(3, 16), (2, 0), (1, -1), (16, 8)]:
            with pytest.raises(lib.BMLError):
                sim.set_tiling(k, band)
    with make(lib, 32, 64, "byte", 0) as sim:
        with pytest.raises(lib.BMLError):
            sim.set_tiling(1, 16)
    with make(lib, 32, 64, "fused", 0) as sim:
        with pytest.raises(lib.BMLError):
            sim.set_tiling(2, 16)
        sim.set_tiling(1, 0)


@pytest.mark.parametrize("M,N", [(100, 4096), (77, 6144), (40, 32768), (5, 2112 * 2)])
def test_two_words_per_lane_tilings_match_oracle(lib, M, N):
    """The streaming kernel with two 64-cell words per lane (rows of full
    words, an even number of them) at every depth and ragged bands."""
    g0 = random_lattice(M, N, M * 3 + N, 0.18, 0.2)
    K = 21
    want, mlr, mtb = oracle.run(g0, K)
    for k, band in [(1, 7), (2, 16), (4, 33), (8, 19), (8, M)]:
        with make(lib, M, N, "tblock", k) as sim:
            sim.set_tiling(k, band, lane_words=2)
            assert sim.tiling == (k, band, 2)
            sim.write(g0)
            sim.step(K)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((k, band)))
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)


# Row widths in pairs of words (128 columns) that exercise every lane-group
# form of the two-words-per-lane kernel: the whole row ring in one cyclic
# group (17, 31, 32 pairs), full segments of 31 pairs with no remainder (62),
# a remainder group of one pair (63: 16 such groups share a warp), of two (33)
# and of eight pairs (256 would be the bench row; 39 and 93 are narrower).
PAIR_WIDTHS = [17, 31, 32, 33, 39, 62, 63, 93]


@pytest.mark.parametrize("pairs", PAIR_WIDTHS)
def test_two_words_per_lane_lane_groups_match_oracle(lib, pairs):
    """Every lane-group form of the two-words-per-lane kernel, with bands of
    different heights in one warp (a short last band packed beside full ones)
    and a lattice shorter than one band: lattice and every count against
    the oracle."""
    N = 128 * pairs
    for M, bands in [(100, [(8, 7), (8, 33), (4, 45), (2, 99), (1, 100)]), (3, [(8, 16)])]:
        g0 = random_lattice(M, N, 7 * pairs + M, 0.19, 0.19)
        K = 19
        want, mlr, mtb = oracle.run(g0, K)
        for k, band in bands:
            with make(lib, M, N, "tblock", k) as sim:
                sim.set_tiling(k, band, lane_words=2)
                sim.write(g0)
                sim.step(K)
                np.testing.assert_array_equal(sim.read(), want, err_msg=str((M, k, band)))
                oracle_counts_equal(sim.moved_counts(), mlr, mtb)


@pytest.mark.parametrize("band", [300, 700, 12000])
def test_two_words_per_lane_tall_bands_count_exactly(lib, band):
    """Bands taller than the 16-bit per-lane count fields can hold without a
    flush: free flow at density 0.2 moves about 13 LR and 13 TB cars per lane
    (128 cells) and row, so one 12000-row band puts about 150000 moves of
    each kind on every lane and stage.  Lattice and every count against the
    oracle."""
    import os
    M, N, K = 12000, 4096, 16
    g0 = random_lattice(M, N, 4242, 0.1, 0.1)
    want, mlr, mtb = oracle.run(g0, K, threads=os.cpu_count() or 1)
    assert mlr.min() // (N // 128) > 65535    # per lane of a one-band tile, every step
    with make(lib, M, N, "tblock", 8) as sim:
        sim.set_tiling(8, band, lane_words=2)
        sim.write(g0)
        sim.step(K)
        np.testing.assert_array_equal(sim.read(), want)
        oracle_counts_equal(sim.moved_counts(), mlr, mtb)


def test_pair_layout_conversions_between_kernels(lib):
    """The two-words-per-lane kernel keeps its planes interleaved; the
    object converts them whenever the next kernel (one word per lane, the
    Model II pair kernel), a read or a device read needs the plain order.
    Switching tilings, models and reads between calls in every order gives
    the oracle's lattice and counts at every point."""
    import torch
    M, N = 70, 4096
    g0 = random_lattice(M, N, 99, 0.17, 0.19)
    plan = [("pair", 8, 5), ("one", 4, 3), ("pair", 1, 2), ("read", 0, 0), ("pair", 8, 9),
            ("m2pair", 4, 6), ("pair", 2, 7), ("devread", 0, 0), ("one", 8, 8), ("pair", 4, 4)]
    want, done = g0, 0
    lrs, tbs = [], []
    with make(lib, M, N, "tblock", 8) as sim:
        sim.write(g0)
        for what, k, n in plan:
            if what == "read":
                np.testing.assert_array_equal(sim.read(), want)
                continue
            if what == "devread":
                d = torch.empty(M * N, dtype=torch.uint8, device="cuda")
                lib.bml_read_lattice_device(sim.handle, d.data_ptr())
                np.testing.assert_array_equal(d.cpu().numpy().reshape(M, N), want)
                continue
            if what == "m2pair":
                sim.set_model(lib.BML_MODEL_II, 5)
                sim.set_tiling(k, 16, lane_words=2)
                want, a, b = oracle.run_model(want, n, 2, tie_seed=5, t0=done)
                sim.step(n)
                sim.set_model(lib.BML_MODEL_I)
            else:
                sim.set_tiling(k, 16, lane_words=2 if what == "pair" else 1)
                want, a, b = oracle.run(want, n)
                sim.step(n)
            done += n
            lrs.append(a)
            tbs.append(b)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((what, k, n)))
        oracle_counts_equal(sim.moved_counts(), np.concatenate(lrs), np.concatenate(tbs))


def test_two_words_per_lane_rejected_where_it_does_not_apply(lib):
    with make(lib, 16, 100, "tblock", 2) as sim:       # N % 64 != 0
        with pytest.raises(lib.BMLError):
            sim.set_tiling(2, 8, lane_words=2)
    with make(lib, 16, 64 * 33, "tblock", 2) as sim:   # odd number of words
        with pytest.raises(lib.BMLError):
            sim.set_tiling(2, 8, lane_words=2)


@pytest.mark.parametrize("fail_at", [1, 2, 3, 5])
def test_allocation_failure_mid_creation_frees_everything(lib, fail_at):
    """The n-th device allocation fails: creation returns BML_ENOMEM and every
    allocation made before it is released (no leak); the next creation with
    a working allocator succeeds."""
    import torch
    live = {}
    count = [0]

    @lib.ALLOC_FN
    def alloc(nbytes, stream, ctx):
        count[0] += 1
        if count[0] == fail_at:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                               stream or 0)
        live[p] = nbytes
        return p

    @lib.FREE_FN
    def free(ptr, nbytes, stream, ctx):
        assert ptr in live
        del live[ptr]
        torch.cuda.caching_allocator_delete(ptr)

    lib._check(lib._lib_set_allocator(alloc, free, None))
    try:
        with pytest.raises(lib.BMLError) as e:
            lib.bml_create_ex(64, 300, 1, 0.1, 0.1, kernel=lib.BML_KERNEL_TBLOCK, block_k=2)
        assert e.value.code == lib.BML_ENOMEM
        assert not live, "allocations leaked"
    finally:
        lib.use_torch_allocator(False)
    with make(lib, 64, 300, "tblock", 2) as sim:
        sim.step(3)


@pytest.mark.parametrize("M,N", [(1, (1 << 22) + 37), ((1 << 22) + 5, 1), (2, (1 << 21) + 64),
                                 ((1 << 20) + 3, 3), (3, 128 * 1024)])
def test_extreme_aspect_ratios_every_kernel(lib, M, N):
    """A single row of 4M cells (ragged tail), a single column of 4M rows,
    and near-degenerate widths: every kernel and depth against the oracle
    (lattice and every count), 9 steps in calls of 4 and 5."""
    g0 = random_lattice(M, N, M + 3 * N, 0.2, 0.2)
    K = 9
    want, mlr, mtb = oracle.run(g0, K)
    for kernel, block_k in KERNEL_CASES:
        if kernel == "resident":
            continue  # larger than one block's shared memory
        with make(lib, M, N, kernel, block_k) as sim:
            sim.write(g0)
            sim.step(4)
            sim.step(5)
            np.testing.assert_array_equal(sim.read(), want, err_msg=str((kernel, block_k)))
            oracle_counts_equal(sim.moved_counts(), mlr, mtb)
