"""Write the oracle's results for the full-size workloads into tests/golden/.

Calls only the oracle (and the shared seeded input generators, which hold
none of the automaton's arithmetic); nothing here runs or reads the CUDA
library.  The GPU tests compare their full-length runs with these files.
The lattices themselves are too large to store, so each run is recorded by
the SHA-256 of its final lattice (M*N bytes, row-major, 0/1/2) and of its
count traces (moved_lr then moved_tb, int64 little-endian), plus a few plain
numbers for diagnostics.

    python tests/golden/make_oracle_refs.py [4096] [windows] [windows4096] [ensemble]
                                            [ensemble512] [ensemble256]

With no argument all six files are written.  On 8 host threads the 4096^2
runs take about 30 minutes, the t = 1024 windows about 2 (the four t = 4096
windows about an hour), the 32-lattice ensemble
subset about 20, all 4096 lattices for 512 steps about 2 hours and the
256-lattice subset for 10^4 steps about 80 minutes (one single-threaded
oracle run per lattice, as many processes as host threads).

- oracle_4096_runs.json: the single-lattice workload 4096 x 4096, densities
  0.20, 0.35, 0.50 split evenly between LR and TB, seeds 1-3, 4096 steps,
  placement by the seeded rule (every cell independently LR w.p. rho/2, TB
  w.p. rho/2).
- oracle_32768_windows.json: the 32768 x 32768 lattice at density 0.38,
  seed 1, after t = 1024 steps, sampled through windows: the state of a
  cell after t steps depends only on the cells within t rows and t columns
  of it (one cell per phase at most), so the oracle run for t steps on a
  (2t + 33) x (2t + 33) window of the initial lattice, wrapped as its own
  torus, gives the exact state of the window's 33 x 33 centre.  Eight
  windows; the first straddles both wrap seams.
- oracle_32768_windows_4096.json: the same lattice after t = 4096 steps,
  four (2t + 33) x (2t + 33) windows (the first across both seams).
- oracle_ensemble_subset.json: 32 lattices of the batched-ensemble workload
  (4096 lattices, M, N uniform on {64..2048}, density uniform on [0.1, 0.6],
  LR fraction uniform on [0.3, 0.7], numpy PCG64 seed 1; lattice l uses
  placement seed l + 1), one at each of 32 evenly spaced quantiles of the
  cell count, run for the full 10^4 steps; with the first step index at
  which no car moved (-1 if none).
- oracle_ensemble_all_512.json: every lattice of that workload for 512
  steps, each recorded by the first 32 hex digits of the SHA-256 of its
  final lattice followed by its count traces (moved_lr then moved_tb, int64
  little-endian).
- oracle_ensemble_256.json: the seeded 256-lattice subset l = 0, 16, 32, ...
  of that workload for the full 10^4 steps, full records as above.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1804_07981_b300.inputs import ensemble_params  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
THREADS = os.cpu_count() or 1


def digest(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def count_digest(lr: np.ndarray, tb: np.ndarray) -> str:
    return digest(np.concatenate([lr.astype("<i8"), tb.astype("<i8")]))


def record(g, lr, tb) -> dict:
    tot = lr + tb
    zero = np.flatnonzero(tot == 0)
    return {"lattice_sha256": digest(g), "counts_sha256": count_digest(lr, tb),
            "lr_sum": int(lr.sum()), "tb_sum": int(tb.sum()),
            "lr_last": int(lr[-1]), "tb_last": int(tb[-1]),
            "first_zero_step": int(zero[0]) if zero.size else -1}


def runs_4096(path):
    M = N = 4096
    K = 4096
    out = {"M": M, "N": N, "steps": K, "runs": []}
    for rho in (0.20, 0.35, 0.50):
        for seed in (1, 2, 3):
            t = time.time()
            g0 = oracle.init(M, N, seed, rho / 2, rho / 2)
            g, lr, tb = oracle.run(g0, K, threads=THREADS)
            rec = {"rho": rho, "seed": seed}
            rec.update(record(g, lr, tb))
            out["runs"].append(rec)
            print("4096^2 rho %.2f seed %d: %.0f s" % (rho, seed, time.time() - t), flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


WINDOW_T = 1024
WINDOW_CORE = 33


def window_corners(M, N, t=WINDOW_T, count=8):
    rng = np.random.Generator(np.random.PCG64(t))
    corners = rng.integers(0, M, size=(count, 2))
    half = t + WINDOW_CORE // 2
    corners[0] = [M - half, N - half]  # the centre sits on both wrap seams
    return [(int(i), int(j)) for i, j in corners]


def windows_32768(path, t=WINDOW_T, count=8):
    M = N = 32768
    c = WINDOW_CORE
    S = 2 * t + c
    out = {"M": M, "N": N, "rho": 0.38, "seed": 1, "steps": t, "window": S, "centre": c,
           "windows": []}
    for i0, j0 in window_corners(M, N, t, count):
        tic = time.time()
        w = oracle.init_window(i0, j0, S, S, M, N, 1, 0.19, 0.19)
        w_t, _, _ = oracle.run(w, t, threads=THREADS)
        core = w_t[t:t + c, t:t + c]
        out["windows"].append({"i0": i0, "j0": j0,
                               "centre_rows": ["".join(str(int(v)) for v in r) for r in core]})
        print("window (%d, %d): %.0f s" % (i0, j0, time.time() - tic), flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


ENS_STEPS = 10000


def ensemble_subset_indices(p, count=32):
    cells = p["M"] * p["N"]
    order = np.argsort(cells, kind="stable")
    q = ((np.arange(count) + 0.5) / count * len(order)).astype(np.int64)
    return sorted(int(order[k]) for k in q)


def ensemble_subset(path):
    p = ensemble_params(4096, seed=1)
    idx = ensemble_subset_indices(p)
    out = {"workload": "ensemble_params(4096, seed=1)", "steps": ENS_STEPS, "lattices": []}
    for l in idx:
        tic = time.time()
        M, N = int(p["M"][l]), int(p["N"][l])
        g0 = oracle.init(M, N, int(p["seed"][l]), float(p["p_lr"][l]), float(p["p_tb"][l]))
        g, lr, tb = oracle.run(g0, ENS_STEPS, threads=THREADS)
        rec = {"index": l, "M": M, "N": N}
        rec.update(record(g, lr, tb))
        out["lattices"].append(rec)
        print("lattice %d (%d x %d): %.0f s" % (l, M, N, time.time() - tic), flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def lattice_digest(g, lr, tb) -> str:
    h = hashlib.sha256(np.ascontiguousarray(g).tobytes())
    h.update(np.concatenate([lr.astype("<i8"), tb.astype("<i8")]).tobytes())
    return h.hexdigest()[:32]


def _ens_run(args):
    """One ensemble lattice through the oracle (a worker process)."""
    M, N, seed, p_lr, p_tb, K = args
    g0 = oracle.init(M, N, seed, p_lr, p_tb)
    return oracle.run(g0, K, threads=1)


def _ens_pool_runs(p, idx, K, reduce):
    import multiprocessing as mp
    jobs = [(int(p["M"][l]), int(p["N"][l]), int(p["seed"][l]), float(p["p_lr"][l]),
             float(p["p_tb"][l]), K) for l in idx]
    # largest first, so the pool ends evenly
    order = sorted(range(len(jobs)), key=lambda k: -jobs[k][0] * jobs[k][1])
    out = [None] * len(jobs)
    tic = time.time()
    with mp.get_context("spawn").Pool(THREADS) as pool:
        for n, (k, res) in enumerate(zip(order, pool.imap(_ens_run, [jobs[k] for k in order]))):
            out[k] = reduce(*res)
            if n % 256 == 255:
                print("%d of %d lattices: %.0f s" % (n + 1, len(jobs), time.time() - tic),
                      flush=True)
    return out


def ensemble_all_512(path):
    p = ensemble_params(4096, seed=1)
    K = 512
    recs = _ens_pool_runs(p, range(4096), K,
                          lambda g, lr, tb: (lattice_digest(g, lr, tb), int(lr.sum()),
                                             int(tb.sum())))
    out = {"workload": "ensemble_params(4096, seed=1)", "steps": K,
           "lr_sum": sum(r[1] for r in recs), "tb_sum": sum(r[2] for r in recs),
           "digests": [r[0] for r in recs]}
    with open(path, "w") as f:
        json.dump(out, f, indent=0)


def ensemble_256(path):
    p = ensemble_params(4096, seed=1)
    idx = list(range(0, 4096, 16))
    recs = _ens_pool_runs(p, idx, ENS_STEPS, record)
    out = {"workload": "ensemble_params(4096, seed=1)", "steps": ENS_STEPS, "lattices": []}
    for l, r in zip(idx, recs):
        rec = {"index": l, "M": int(p["M"][l]), "N": int(p["N"][l])}
        rec.update(r)
        out["lattices"].append(rec)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def main(argv):
    which = set(argv) or {"4096", "windows", "windows4096", "ensemble", "ensemble512",
                          "ensemble256"}
    if "windows" in which:
        windows_32768(os.path.join(HERE, "oracle_32768_windows.json"))
    if "windows4096" in which:
        windows_32768(os.path.join(HERE, "oracle_32768_windows_4096.json"), t=4096, count=4)
    if "ensemble" in which:
        ensemble_subset(os.path.join(HERE, "oracle_ensemble_subset.json"))
    if "4096" in which:
        runs_4096(os.path.join(HERE, "oracle_4096_runs.json"))
    if "ensemble512" in which:
        ensemble_all_512(os.path.join(HERE, "oracle_ensemble_all_512.json"))
    if "ensemble256" in which:
        ensemble_256(os.path.join(HERE, "oracle_ensemble_256.json"))


if __name__ == "__main__":
    main(sys.argv[1:])
