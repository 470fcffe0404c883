"""GPU parity of the batched ensemble against the CPU oracle (per lattice),
through the C ABI."""
import os

import numpy as np
import pytest

import oracle
from paper_1804_07981_b300.inputs import all_lattices, ensemble_params

pytestmark = pytest.mark.gpu


def oracle_ensemble(Ms, Ns, seeds, plr, ptb, K):
    outs, lrs, tbs = [], [], []
    for M, N, s, a, b in zip(Ms, Ns, seeds, plr, ptb):
        g0 = oracle.init(int(M), int(N), int(s), float(a), float(b))
        g, lr, tb = oracle.run(g0, K)
        outs.append(g)
        lrs.append(lr)
        tbs.append(tb)
    return outs, np.stack(lrs), np.stack(tbs)


def mixed_shapes(count, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    M = rng.integers(1, 140, size=count)
    N = rng.integers(1, 2049, size=count)
    n = min(count, 6)
    N[:n] = [1, 63, 64, 65, 2047, 2048][:n]
    M[:n] = [1, 2, 3, 17, 5, 1][:n]
    rho = rng.uniform(0.1, 0.7, size=count)
    f = rng.uniform(0.3, 0.7, size=count)
    return M, N, np.arange(1, count + 1, dtype=np.uint64), rho * f, rho * (1 - f)


@pytest.mark.parametrize("block_k,band", [(1, 16), (2, 37), (4, 64), (8, 128), (8, 9), (0, 0)])
def test_ensemble_mixed_shapes_match_oracle(lib, block_k, band):
    M, N, seeds, plr, ptb = mixed_shapes(48, 7)
    K = 29
    want, wlr, wtb = oracle_ensemble(M, N, seeds, plr, ptb, K)
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=block_k, band_rows=band) as ens:
        ens.step(10)
        ens.step(K - 10)
        got = ens.read_all()
        lr, tb = ens.traces()
        for l in range(len(M)):
            np.testing.assert_array_equal(got[l], want[l], err_msg="lattice %d" % l)
        np.testing.assert_array_equal(lr, wlr)
        np.testing.assert_array_equal(tb, wtb)
        tot, a, b = ens.moved_counts(5)
        np.testing.assert_array_equal(tot, wlr[5] + wtb[5])
        np.testing.assert_array_equal(ens.read(5), want[5])


def test_ensemble_tall_bands_count_exactly(lib):
    """One band of 16000 rows per lattice group: at density 0.24 about 6 LR
    and 6 TB cars move per lane (64 cells) and row, over 90000 per lane and
    stage over the band, more than one 16-bit count field holds between
    flushes.  Lattices and traces against the oracle."""
    M = np.array([16000, 16000, 15999, 16000])
    N = np.array([64, 128, 100, 2048])
    seeds = np.arange(11, 15, dtype=np.uint64)
    plr, ptb = np.full(4, 0.12), np.full(4, 0.12)
    K = 16
    want, wlr, wtb = oracle_ensemble(M, N, seeds, plr, ptb, K)
    assert wlr[0].min() > 65535        # lattice 0: one lane per row
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=8, band_rows=16000) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    for l in range(len(M)):
        np.testing.assert_array_equal(got[l], want[l], err_msg="lattice %d" % l)
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)


@pytest.mark.parametrize("M,N", [(1, 12), (2, 6), (3, 4), (4, 3), (6, 2), (12, 1), (1, 11),
                                 (3, 3), (2, 5), (5, 2), (1, 1), (1, 2), (2, 1), (2, 2)])
def test_ensemble_exhaustive_tiny_lattices(lib, M, N):
    """Every configuration of an M x N lattice (M*N <= 12) as one ensemble
    member each, 3 steps, against the oracle."""
    gs = all_lattices(M, N)
    count = gs.shape[0]
    K = 3
    og, olr, otb = oracle.run_batch(gs, K)
    with lib.Ensemble(np.full(count, M), np.full(count, N), np.arange(count), np.zeros(count),
                      np.zeros(count), block_k=2, band_rows=M, reserve_steps=8) as ens:
        ens.write_all(gs)
        ens.step(K)
        got = np.stack(ens.read_all())
        lr, tb = ens.traces()
    np.testing.assert_array_equal(got, og)
    np.testing.assert_array_equal(lr, olr)
    np.testing.assert_array_equal(tb, otb)


def test_ensemble_config4_style_subset(lib):
    """A subset of the batched-ensemble workload (M, N uniform on
    {64..2048}, density in [0.1, 0.6], LR fraction in [0.3, 0.7])."""
    p = ensemble_params(4096, seed=1)
    idx = np.arange(0, 4096, 256)  # 16 lattices
    M, N = p["M"][idx], p["N"][idx]
    K = 64
    want, wlr, wtb = oracle_ensemble(M, N, p["seed"][idx], p["p_lr"][idx], p["p_tb"][idx], K)
    with lib.Ensemble(M, N, p["seed"][idx], p["p_lr"][idx], p["p_tb"][idx]) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    for l in range(len(M)):
        np.testing.assert_array_equal(got[l], want[l])
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)


@pytest.mark.parametrize("block_k", [2, 8])
def test_ensemble_early_exit_exact(lib, block_k):
    """High densities jam; skipping frozen lattices must not change anything."""
    rng = np.random.Generator(np.random.PCG64(3))
    count = 40
    M = rng.integers(8, 60, size=count)
    N = rng.integers(8, 200, size=count)
    rho = rng.uniform(0.45, 0.9, size=count)
    seeds = np.arange(100, 100 + count, dtype=np.uint64)
    K = 300
    want, wlr, wtb = oracle_ensemble(M, N, seeds, rho / 2, rho / 2, K)
    jam_want = np.array([np.flatnonzero(a + b == 0)[0] if np.any(a + b == 0) else -1
                         for a, b in zip(wlr, wtb)])
    assert (jam_want >= 0).sum() > count // 2
    with lib.Ensemble(M, N, seeds, rho / 2, rho / 2, block_k=block_k, band_rows=16,
                      flags=lib.BML_ENS_EARLY_EXIT) as ens:
        for _ in range(5):
            ens.step(K // 5)
        got = ens.read_all()
        lr, tb = ens.traces()
        jam = ens.jam_steps()
    for l in range(count):
        np.testing.assert_array_equal(got[l], want[l])
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)
    np.testing.assert_array_equal(jam, jam_want)


def test_ensemble_graph_and_direct_launches_agree(lib):
    import torch
    M, N, seeds, plr, ptb = mixed_shapes(20, 11)
    st = torch.cuda.Stream()
    res = []
    for flags in (0, lib.BML_ENS_NO_GRAPH):
        with lib.Ensemble(M, N, seeds, plr, ptb, block_k=4, band_rows=32, flags=flags,
                          stream=st) as ens:
            for _ in range(4):
                ens.step(12)
            assert ens.config[2] == (flags == 0)
            res.append((ens.read_all(), ens.traces()))
    for a, b in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(res[0][1][0], res[1][1][0])
    np.testing.assert_array_equal(res[0][1][1], res[1][1][1])


def test_ensemble_write_rejects_bad_values(lib):
    M, N, seeds, plr, ptb = mixed_shapes(5, 2)
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=1, band_rows=8) as ens:
        ens.step(3)
        before = ens.read_all()
        bad = [g.copy() for g in before]
        bad[2].flat[0] = 7
        with pytest.raises(lib.BMLError) as e:
            ens.write_all(bad)
        assert e.value.code == lib.BML_EINVAL
        for a, b in zip(ens.read_all(), before):
            np.testing.assert_array_equal(a, b)
        assert ens.steps_done == 3


def test_ensemble_barrier_timeout_is_reported(lib):
    """A wait between chunks that can never complete (test hook: it waits
    for one band more than its lattice has) gives up after its time limit;
    the call reports BML_ETIMEOUT, the ensemble refuses further work, and
    the GPU context stays usable."""
    M, N, seeds, plr, ptb = mixed_shapes(8, 5)
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=2, band_rows=16,
                      flags=lib.BML_ENS_TEST_STALL | lib.BML_ENS_NO_GRAPH) as ens:
        with pytest.raises(lib.BMLError) as e:
            ens.step(8)  # four chunks: waits before the last three
        assert e.value.code == lib.BML_ETIMEOUT
        with pytest.raises(lib.BMLError) as e:
            ens.step(2)
        assert e.value.code == lib.BML_ESTATE
    K = 9
    want, wlr, wtb = oracle_ensemble(M, N, seeds, plr, ptb, K)
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=2, band_rows=16) as ens:
        ens.step(K)
        lr, tb = ens.traces()
    np.testing.assert_array_equal(lr, wlr)


def test_ensemble_rejects_bad_arguments(lib):
    with pytest.raises(lib.BMLError):
        lib.bml_ensemble_create_ex([10], [4096], [1], [0.1], [0.1], 1, 16)
    with pytest.raises(lib.BMLError):
        lib.bml_ensemble_create_ex([10], [100], [1], [0.6], [0.6], 1, 16)
    with pytest.raises(lib.BMLError):
        lib.bml_ensemble_create_ex([10], [100], [1], [0.1], [0.1], 3, 16)
    with pytest.raises(lib.BMLError):
        lib.bml_ensemble_create_ex([10], [100], [1], [0.1], [0.1], 2, 0)


def test_features_and_labels_match_oracle(lib):
    """Surrogate inputs and labels computed on the device from the ensemble's
    traces equal the oracle's, computed from the oracle's own runs."""
    from oracle import features as F
    M, N, seeds, plr, ptb = mixed_shapes(30, 13)
    K, points, window = 128, 16, 32
    want, wlr, wtb = oracle_ensemble(M, N, seeds, plr, ptb, K)
    cars = np.array([int(((oracle.init(int(m), int(n), int(s), float(a), float(b))) != 0).sum())
                     for m, n, s, a, b in zip(M, N, seeds, plr, ptb)])
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=4, band_rows=32) as ens:
        ens.step(K)
        np.testing.assert_array_equal(ens.car_counts(), cars)
        f = ens.features(0, K, points).cpu().numpy()
        v, jam = (t.cpu().numpy() for t in ens.labels(window))
    wf = F.features(wlr + wtb, cars, M, N, 0, K, points)
    wv, wj = F.labels(wlr + wtb, cars, window)
    np.testing.assert_allclose(f, wf, rtol=1e-6, atol=1e-7)
    np.testing.assert_allclose(v, wv, rtol=1e-6, atol=1e-7)
    np.testing.assert_array_equal(jam, wj)


@pytest.mark.parametrize("early_exit", [False, True])
def test_ensemble_retire_stops_lattices_and_others_continue(lib, early_exit):
    """Retired lattices keep the state they had at the retirement step and
    count 0 afterwards; jam steps and labels of a retired lattice are those
    of its trajectory before the retirement; the others match the oracle
    over the whole run."""
    M, N, seeds, plr, ptb = mixed_shapes(24, 17)
    K1, K2 = 37, 29
    w1, l1, t1 = oracle_ensemble(M, N, seeds, plr, ptb, K1)
    w2, l2, t2 = oracle_ensemble(M, N, seeds, plr, ptb, K1 + K2)
    gone = np.array([0, 3, 4, 11, 23, 3])  # with a repeat
    flags = lib.BML_ENS_EARLY_EXIT if early_exit else 0
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=4, band_rows=16, flags=flags,
                      reserve_steps=K1 + K2) as ens:
        ens.step(K1)
        ens.retire(gone)
        ens.retire([])
        ens.step(K2)
        got = ens.read_all()
        lr, tb = ens.traces()
        jam = ens.jam_steps()
        v, jf = (t.cpu().numpy() for t in ens.labels(8))
        with pytest.raises(lib.BMLError):
            ens.retire([len(M)])
    for l in range(len(M)):
        if l in gone:
            np.testing.assert_array_equal(got[l], w1[l])
            np.testing.assert_array_equal(lr[l], np.concatenate([l1[l], np.zeros(K2, np.int64)]))
            np.testing.assert_array_equal(tb[l], np.concatenate([t1[l], np.zeros(K2, np.int64)]))
            tot = l1[l] + t1[l]
            zero = np.flatnonzero(tot == 0)
            assert jam[l] == (zero[0] if zero.size else -1)
            cars = np.count_nonzero(w1[l])
            want_v = tot[-8:].sum() / (8 * cars) if cars else 0.0
            assert abs(v[l] - want_v) < 1e-6 and jf[l] == float(zero.size > 0)
        else:
            np.testing.assert_array_equal(got[l], w2[l])
            np.testing.assert_array_equal(lr[l], l2[l])
            np.testing.assert_array_equal(tb[l], t2[l])


def test_ensemble_retire_plans_the_tiles_again(lib):
    """An autotuned ensemble of 1024 lattices of 1024 x 1024 (bands of a few
    hundred rows): retiring all but 6 plans the tiles again for those 6 with
    shorter bands (more tiles for the warps), and they go on exactly as the
    oracle's runs; retired lattices keep their state.  An ensemble with its
    band height given at creation keeps it."""
    count, M, N, K1, K2 = 1024, 1024, 1024, 24, 40
    rho = np.linspace(0.15, 0.45, count)
    seeds = np.arange(1, count + 1, dtype=np.uint64)
    keep = np.array([3, 170, 400, 401, 777, 1023])
    gone = np.setdiff1d(np.arange(count), keep)
    Ms, Ns = np.full(count, M), np.full(count, N)
    with lib.Ensemble(Ms, Ns, seeds, rho / 2, rho / 2, reserve_steps=K1 + K2) as ens:
        ens.step(K1)
        k0, band0, _ = ens.config
        mid = {int(l): ens.read(int(l)) for l in gone[::97]}
        ens.retire(gone)
        k1, band1, _ = ens.config
        ens.step(K2)
        for l, g in mid.items():
            np.testing.assert_array_equal(ens.read(l), g)
        got = {int(l): ens.read(int(l)) for l in keep}
        lr, tb = ens.traces()
    assert k1 == k0 and band1 < band0, (band0, band1)
    for l in keep:
        g0 = oracle.init(M, N, int(seeds[l]), rho[l] / 2, rho[l] / 2)
        want, wlr, wtb = oracle.run(g0, K1 + K2, threads=os.cpu_count() or 1)
        np.testing.assert_array_equal(got[int(l)], want)
        np.testing.assert_array_equal(lr[l], wlr)
        np.testing.assert_array_equal(tb[l], wtb)
    with lib.Ensemble(Ms[:8], Ns[:8], seeds[:8], rho[:8] / 2, rho[:8] / 2, block_k=4,
                      band_rows=128) as ens:
        ens.step(8)
        ens.retire(np.arange(6))
        assert ens.config[:2] == (4, 128)


@pytest.mark.parametrize("block_k,band", [(1, 16), (4, 64), (8, 21), (0, 0)])
def test_ensemble_full_word_tiles_match_oracle(lib, block_k, band):
    """Lattices whose rows are whole 64-cell words only (every tile takes the
    stage form without ragged terms), mixed widths and heights."""
    rng = np.random.Generator(np.random.PCG64(21))
    count = 30
    N = 64 * rng.integers(1, 33, size=count)
    M = rng.integers(1, 150, size=count)
    rho = rng.uniform(0.1, 0.7, size=count)
    seeds = np.arange(50, 50 + count, dtype=np.uint64)
    K = 33
    want, wlr, wtb = oracle_ensemble(M, N, seeds, rho / 2, rho / 2, K)
    with lib.Ensemble(M, N, seeds, rho / 2, rho / 2, block_k=block_k, band_rows=band) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    for l in range(count):
        np.testing.assert_array_equal(got[l], want[l], err_msg="lattice %d" % l)
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)


def test_ensemble_write_makes_retired_lattices_active_again(lib):
    M, N, seeds, plr, ptb = mixed_shapes(10, 23)
    K = 17
    with lib.Ensemble(M, N, seeds, plr, ptb, block_k=2, band_rows=8, reserve_steps=64) as ens:
        ens.step(5)
        start = ens.read_all()
        ens.retire(np.arange(10))
        ens.step(3)
        for a, b in zip(ens.read_all(), start):   # nothing moved
            np.testing.assert_array_equal(a, b)
        ens.write_all(start)                        # restart: every lattice active
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    for l in range(10):
        want, wlr, wtb = oracle.run(start[l], K)
        np.testing.assert_array_equal(got[l], want)
        np.testing.assert_array_equal(lr[l], wlr)
        np.testing.assert_array_equal(tb[l], wtb)
