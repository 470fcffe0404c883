"""Parity at the workloads' full sizes.

Against the oracle's own full-length results (tests/golden/oracle_*.json,
written by tests/golden/make_oracle_refs.py, which runs only the oracle and
records each final lattice and count trace by its SHA-256): all nine
4096^2 x 4096-step runs through both the byte-per-cell and the bit-packed
kernels, the 32768^2 lattice after 1024 steps through eight (2t + 33)^2
windows in the benchmark's launch configuration and after 4096 steps through
four, 32 lattices of the ensemble workload at its size quantiles and the
seeded 256-lattice subset (every 16th) for the full 10^4 steps, and every
lattice of that workload for 512 steps.  Beside them: oracle runs on
sampled windows computed here, exact cross-checks between independent GPU
paths, and properties that hold at any size."""
import hashlib
import json
import os

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

EMPTY, LR, TB = 0, 1, 2
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def _count_digest(lr, tb):
    return _digest(np.concatenate([np.asarray(lr).astype("<i8"), np.asarray(tb).astype("<i8")]))


def _lattice_digest(g, lr, tb):
    """First 32 hex digits of the SHA-256 of a final lattice followed by its
    count traces (the oracle_ensemble_all_512.json record)."""
    h = hashlib.sha256(np.ascontiguousarray(g).tobytes())
    h.update(np.concatenate([np.asarray(lr).astype("<i8"), np.asarray(tb).astype("<i8")]).tobytes())
    return h.hexdigest()[:32]


@pytest.mark.parametrize("kernel", ["byte", "auto"])
def test_4096_nine_full_runs_against_oracle(lib, kernel):
    """Single lattice 4096 x 4096, densities {0.20, 0.35, 0.50} split evenly,
    seeds 1-3, 4096 steps, placement by the seeded rule: every final lattice
    and the whole LR / TB count trace of each run equal the oracle's."""
    ref = _golden("oracle_4096_runs.json")
    assert len(ref["runs"]) == 9 and ref["steps"] == 4096
    for r in ref["runs"]:
        with lib.Lattice(4096, 4096, seed=r["seed"], density=r["rho"], kernel=kernel,
                         reserve_steps=4096) as sim:
            sim.step(4096)
            g = sim.read()
            _, lr, tb = sim.moved_counts()
        what = (kernel, r["rho"], r["seed"])
        assert int(lr.sum()) == r["lr_sum"] and int(tb.sum()) == r["tb_sum"], what
        assert int(lr[-1]) == r["lr_last"] and int(tb[-1]) == r["tb_last"], what
        assert _count_digest(lr, tb) == r["counts_sha256"], what
        assert _digest(g) == r["lattice_sha256"], what


@pytest.mark.parametrize("config", ["auto", (8, 231, 2), (8, 251, 2)],
                         ids=["auto", "depth8-band231-pairs", "depth8-band251-pairs"])
def test_32768_windows_after_1024_steps_against_oracle(lib, config):
    """32768 x 32768, density 0.38, seed 1, 1024 steps in the benchmark's
    launch configuration (autotuned, and the tiling it picks on a B300 --
    depth 8, 231-row bands, two words per lane -- given explicitly; 251-row
    bands as another band height): the 33 x 33 centres of eight
    (2t + 33)^2 windows, one across both wrap seams, equal the oracle's run
    of each window as its own torus."""
    ref = _golden("oracle_32768_windows.json")
    M, N, t, c = ref["M"], ref["N"], ref["steps"], ref["centre"]
    kw = {} if config == "auto" else {"kernel": "tblock", "block_k": 8}
    with lib.Lattice(M, N, seed=ref["seed"], density=ref["rho"], reserve_steps=t, **kw) as sim:
        if config != "auto":
            sim.set_tiling(*config[:2], lane_words=config[2])
        sim.step(t)
        got = sim.read()
    assert len(ref["windows"]) == 8
    for w in ref["windows"]:
        rows = (np.arange(t, t + c) + w["i0"]) % M
        cols = (np.arange(t, t + c) + w["j0"]) % N
        want = np.array([[int(ch) for ch in r] for r in w["centre_rows"]], dtype=np.uint8)
        np.testing.assert_array_equal(got[np.ix_(rows, cols)], want, err_msg=str(w["i0"]))


def test_32768_windows_after_4096_steps_against_oracle(lib):
    """32768 x 32768, density 0.38, seed 1, 4096 steps, autotuned as the
    benchmark runs it: the 33 x 33 centres of four (2t + 33)^2 windows (t =
    4096), one across both wrap seams, equal the oracle's run of each window
    as its own torus."""
    ref = _golden("oracle_32768_windows_4096.json")
    M, N, t, c = ref["M"], ref["N"], ref["steps"], ref["centre"]
    assert t == 4096 and len(ref["windows"]) == 4
    with lib.Lattice(M, N, seed=ref["seed"], density=ref["rho"], reserve_steps=t) as sim:
        sim.step(t)
        got = sim.read()
    for w in ref["windows"]:
        rows = (np.arange(t, t + c) + w["i0"]) % M
        cols = (np.arange(t, t + c) + w["j0"]) % N
        want = np.array([[int(ch) for ch in r] for r in w["centre_rows"]], dtype=np.uint8)
        np.testing.assert_array_equal(got[np.ix_(rows, cols)], want, err_msg=str(w["i0"]))


def test_ensemble_workload_full_10000_steps_against_oracle(lib):
    """The batched-ensemble workload (4096 lattices), autotuned as the
    benchmark runs it, 10^4 steps, with and without the jam early exit: 32
    lattices spread over the range of sizes and the seeded 256-lattice
    subset (every 16th; N mod 64 != 0 included) end with the oracle's
    lattice and count trace, and the jam steps of the early-exit ensemble
    equal the oracle's first step with no move."""
    from paper_1804_07981_b300.inputs import ensemble_params
    sub = _golden("oracle_ensemble_subset.json")
    every16 = _golden("oracle_ensemble_256.json")
    K = sub["steps"]
    assert every16["steps"] == K == 10000
    p = ensemble_params(4096, seed=1)
    recs = sub["lattices"] + every16["lattices"]
    assert len(sub["lattices"]) == 32 and len(every16["lattices"]) == 256
    assert [r["index"] for r in every16["lattices"]] == list(range(0, 4096, 16))
    assert any(r["N"] % 64 for r in recs)
    for flags in (0, lib.BML_ENS_EARLY_EXIT):
        with lib.Ensemble(p["M"], p["N"], p["seed"], p["p_lr"], p["p_tb"], flags=flags,
                          reserve_steps=K) as ens:
            ens.step(K)
            jam = ens.jam_steps()
            for r in recs:
                l = r["index"]
                assert (int(p["M"][l]), int(p["N"][l])) == (r["M"], r["N"])
                _, lr, tb = ens.moved_counts(l)
                assert _count_digest(lr, tb) == r["counts_sha256"], (flags, l)
                assert _digest(ens.read(l)) == r["lattice_sha256"], (flags, l)
                if flags:
                    assert jam[l] == r["first_zero_step"], l
    assert any(r["first_zero_step"] >= 0 for r in recs)
    assert any(r["first_zero_step"] < 0 for r in recs)


@pytest.mark.parametrize("rho", [0.20, 0.35, 0.50])
def test_4096_byte_and_bitplane_agree_for_4096_steps(lib, rho):
    """Single lattice 4096 x 4096, densities {0.20, 0.35, 0.50} split evenly,
    seeds 1-3, 4096 steps: the byte-per-cell kernel and the bit-packed
    autotuned kernel give the same lattice and per-step counts."""
    M = N = 4096
    for seed in (1, 2, 3):
        out = []
        for kernel in ("byte", "auto"):
            with lib.Lattice(M, N, seed=seed, density=rho, kernel=kernel,
                             reserve_steps=4096) as sim:
                sim.step(4096)
                out.append((sim.read(), sim.moved_counts()))
        np.testing.assert_array_equal(out[0][0], out[1][0])
        for a, b in zip(out[0][1], out[1][1]):
            np.testing.assert_array_equal(a, b)


def test_4096_against_threaded_oracle(lib):
    """One 4096^2 run against the oracle itself (threaded, identical results
    for any thread count) for 512 steps: lattice and every count."""
    import os
    bml = lib
    M = N = 4096
    g0 = oracle.init(M, N, 1, 0.175, 0.175)
    want, mlr, mtb = oracle.run(g0, 512, threads=os.cpu_count() or 1)
    with bml.Lattice(M, N, seed=1, density=0.35) as sim:
        np.testing.assert_array_equal(sim.read(), g0)
        sim.step(512)
        np.testing.assert_array_equal(sim.read(), want)
        _, lr, tb = sim.moved_counts()
    np.testing.assert_array_equal(lr, mlr)
    np.testing.assert_array_equal(tb, mtb)


def _window_init(i0, j0, S, M, N, seed, p):
    """Cells of rows i0..i0+S-1, columns j0..j0+S-1 (mod M, N) of the seeded
    placement, computed one by one with the oracle's generator."""
    t = oracle.threshold(p)
    w = np.zeros((S, S), dtype=np.uint8)
    for a in range(S):
        i = (i0 + a) % M
        for b in range(S):
            j = (j0 + b) % N
            u = oracle.splitmix64(seed, i * N + j + 1)
            w[a, b] = LR if u < t else (TB if u - t < t else EMPTY)
    return w


def test_32768_sampled_windows_in_bench_configuration(lib):
    """32768 x 32768, density 0.38, seed 1, in the launch configuration the
    benchmark times (autotuned depth and band): after 8 steps every cell's
    state depends only on the 17 x 17 cells around it, so the oracle run on
    a 33 x 33 window (wrapped as its own small torus) gives the exact state
    of the 17 x 17 centre of the window."""
    M = N = 32768
    t, S = 8, 33
    with lib.Lattice(M, N, seed=1, density=0.38) as sim:
        sim.step(t)
        got = sim.read()
    rng = np.random.Generator(np.random.PCG64(5))
    corners = rng.integers(0, M, size=(32, 2))
    corners[0] = [M - 16, N - 16]  # a window across both wrap seams
    for i0, j0 in corners:
        w = _window_init(int(i0), int(j0), S, M, N, 1, 0.19)
        w_t, _, _ = oracle.run(w, t)
        rows = (np.arange(t, S - t) + i0) % M
        cols = (np.arange(t, S - t) + j0) % N
        np.testing.assert_array_equal(got[np.ix_(rows, cols)], w_t[t:S - t, t:S - t])


def test_32768_full_run_properties(lib):
    """The benchmark's full job (10^4 steps at 32768^2): LR cars per row and
    TB cars per column are conserved; every LR move adds 1 to the column
    index of one car (mod N) and every TB move adds 1 to a row index
    (mod M), so the summed counts equal the change of those index sums
    modulo N and M; no step moves more cars than exist."""
    M = N = 32768
    with lib.Lattice(M, N, seed=1, density=0.38, reserve_steps=10000) as sim:
        g0 = sim.read()
        sim.step(10000)
        g1 = sim.read()
        _, lr, tb = sim.moved_counts()
    cols = np.arange(N, dtype=np.int64)
    rows = np.arange(M, dtype=np.int64)
    per = {}
    for name, g in (("0", g0), ("1", g1)):
        is_lr, is_tb = g == LR, g == TB
        per[name] = (is_lr.sum(axis=1), is_tb.sum(axis=0),   # LR per row, TB per column
                     is_lr.sum(axis=0), is_tb.sum(axis=1))   # LR per column, TB per row
        del is_lr, is_tb
    np.testing.assert_array_equal(per["0"][0], per["1"][0])
    np.testing.assert_array_equal(per["0"][1], per["1"][1])
    s_lr0, s_lr1 = int(per["0"][2] @ cols), int(per["1"][2] @ cols)
    s_tb0, s_tb1 = int(per["0"][3] @ rows), int(per["1"][3] @ rows)
    assert (int(lr.sum()) - (s_lr1 - s_lr0)) % N == 0
    assert (int(tb.sum()) - (s_tb1 - s_tb0)) % M == 0
    n_lr, n_tb = int(per["0"][0].sum()), int(per["0"][1].sum())
    assert lr.min() >= 0 and lr.max() <= n_lr and tb.min() >= 0 and tb.max() <= n_tb


def test_32768_one_pass_and_depth_8_agree_and_match_windows(lib):
    """32768 x 32768, density 0.38, seed 1, 16 steps: the one-pass
    configuration (depth 1, 16-row bands, two words per lane) and the
    bench's depth-8 configuration give the same lattice and counts, and
    sampled 33 x 33 windows match the oracle (8 steps at a time)."""
    M = N = 32768
    out = []
    for k, band in ((1, 16), (8, 231)):
        with lib.Lattice(M, N, seed=1, density=0.38, kernel="tblock", block_k=k) as sim:
            sim.set_tiling(k, band, lane_words=2)
            sim.step(8)
            g8 = sim.read()
            sim.step(8)
            out.append((g8, sim.read(), sim.moved_counts()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    for a, b in zip(out[0][2], out[1][2]):
        np.testing.assert_array_equal(a, b)
    t, S = 8, 33
    rng = np.random.Generator(np.random.PCG64(9))
    corners = rng.integers(0, M, size=(16, 2))
    corners[0] = [0, N - 20]
    for i0, j0 in corners:
        rows = (np.arange(S) + i0) % M
        cols = (np.arange(S) + j0) % N
        w = out[0][0][np.ix_(rows, cols)]          # state after 8 steps
        w_t, _, _ = oracle.run(w, t)
        np.testing.assert_array_equal(out[0][1][np.ix_(rows[t:S - t], cols[t:S - t])],
                                      w_t[t:S - t, t:S - t])


def test_32768_full_job_byte_kernel_agrees(lib):
    """The benchmark's full job, 32768 x 32768, density 0.38, seed 1, 10^4
    steps: the byte-per-cell kernels (an independent GPU path: one byte per
    cell, one kernel per phase) and the bit-packed kernel in the bench's
    launch configuration (depth 8, 231-row bands, two words per lane) end
    with the same lattice and the same count at every step."""
    M = N = 32768
    K = 10000
    out = []
    for kernel, tiling in (("byte", None), ("tblock", (8, 231, 2))):
        with lib.Lattice(M, N, seed=1, density=0.38, kernel=kernel,
                         block_k=8 if tiling else 0, reserve_steps=K) as sim:
            if tiling:
                sim.set_tiling(*tiling)
            sim.step(K)
            out.append((sim.read(), sim.moved_counts()))
    assert np.array_equal(out[0][0], out[1][0])
    for a, b in zip(out[0][1], out[1][1]):
        np.testing.assert_array_equal(a, b)
    tot = out[1][1][0]
    assert tot.shape == (K,) and tot.min() > 0  # flows at 0.38 at this size


def _byte_runs(lib, M, N, seeds, plr, ptb, K):
    """Each lattice alone through the byte-per-cell kernels (K steps)."""
    outs, lrs, tbs = [], [], []
    for m, n, s, a, b in zip(M, N, seeds, plr, ptb):
        with lib.Lattice(int(m), int(n), seed=int(s), p_lr=float(a), p_tb=float(b),
                         kernel="byte", reserve_steps=K) as sim:
            sim.step(K)
            outs.append(sim.read())
            _, lr, tb = sim.moved_counts()
            lrs.append(lr)
            tbs.append(tb)
    return outs, np.stack(lrs), np.stack(tbs)


def test_ensemble_workload_all_lattices_512_steps_against_oracle(lib):
    """The batched-ensemble workload (4096 lattices, M, N uniform on
    {64..2048}, density in [0.1, 0.6], LR fraction in [0.3, 0.7]), autotuned
    as the bench runs it, 512 steps: every lattice's final state and count
    traces equal the oracle's (tests/golden/oracle_ensemble_all_512.json),
    and also the lattice run alone through the byte-per-cell kernels (an
    independent GPU path)."""
    from paper_1804_07981_b300.inputs import ensemble_params
    ref = _golden("oracle_ensemble_all_512.json")
    p = ensemble_params(4096, seed=1)
    K = ref["steps"]
    assert K == 512 and len(ref["digests"]) == 4096
    with lib.Ensemble(p["M"], p["N"], p["seed"], p["p_lr"], p["p_tb"],
                      reserve_steps=K) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    bad = [l for l in range(4096) if _lattice_digest(got[l], lr[l], tb[l]) != ref["digests"][l]]
    assert not bad, "lattices differing from the oracle: %s" % bad[:16]
    assert int(lr.sum()) == ref["lr_sum"] and int(tb.sum()) == ref["tb_sum"]
    want, wlr, wtb = _byte_runs(lib, p["M"], p["N"], p["seed"], p["p_lr"], p["p_tb"], K)
    for l in range(len(want)):
        assert np.array_equal(got[l], want[l]), l
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)


def test_ensemble_workload_256_lattices_full_10000_steps_against_byte_kernel(lib):
    """A seeded 256-lattice subset of the ensemble workload (every 16th
    lattice) for the full 10^4 steps, with the jam early exit: lattices,
    counts and jam steps equal the byte kernels' runs."""
    from paper_1804_07981_b300.inputs import ensemble_params
    p = ensemble_params(4096, seed=1)
    idx = np.arange(0, 4096, 16)
    M, N, s, a, b = p["M"][idx], p["N"][idx], p["seed"][idx], p["p_lr"][idx], p["p_tb"][idx]
    K = 10000
    with lib.Ensemble(M, N, s, a, b, flags=lib.BML_ENS_EARLY_EXIT, reserve_steps=K) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
        jam = ens.jam_steps()
    want, wlr, wtb = _byte_runs(lib, M, N, s, a, b, K)
    for l in range(len(want)):
        assert np.array_equal(got[l], want[l]), l
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)
    tot = wlr + wtb
    want_jam = np.array([np.flatnonzero(t == 0)[0] if np.any(t == 0) else -1 for t in tot])
    np.testing.assert_array_equal(jam, want_jam)
    assert (want_jam >= 0).any() and (want_jam < 0).any()


def test_ensemble_extreme_shapes_against_byte_kernel(lib):
    """An ensemble holding a 4M-row single-column lattice, a one-row lattice
    of 2048 cells, a 2048-wide lattice of 40000 rows and small ones,
    autotuned: every lattice and count equals the byte kernels' runs."""
    M = np.array([(1 << 22) + 7, 1, 40000, 3, 64, 129])
    N = np.array([1, 2048, 2048, 5, 64, 1000])
    seeds = np.arange(1, 7, dtype=np.uint64)
    plr, ptb = np.full(6, 0.2), np.full(6, 0.15)
    K = 20
    with lib.Ensemble(M, N, seeds, plr, ptb, reserve_steps=K) as ens:
        ens.step(K)
        got = ens.read_all()
        lr, tb = ens.traces()
    want, wlr, wtb = _byte_runs(lib, M, N, seeds, plr, ptb, K)
    for l in range(len(M)):
        assert np.array_equal(got[l], want[l]), l
    np.testing.assert_array_equal(lr, wlr)
    np.testing.assert_array_equal(tb, wtb)
