"""Phase diagram of the BML model: mean velocity and jam probability against
density for several lattice sizes, and the lattice pictures of Fig. 1.

Sec. 2 of the paper: below a critical density that depends on the lattice
size the vehicles settle into a free-flowing state (every vehicle moves
every step); above it a global jam develops (no vehicle moves); in an
interval around the critical density both outcomes have non-zero
probability (coexistence).  This module measures those three statements on
N x N lattices, density rho split evenly into LR and TB (p_lr = p_tb =
rho/2), seeds 1..S per density, T steps:

- velocity of a run = moved vehicles per vehicle and step, averaged over
  the last `window` steps of the T (a step with no move is an absorbing
  fixed point, so every step after it moves nothing);
- jammed = some step up to T moved no vehicle (exact);
- per (N, rho): mean velocity, jam fraction with a Wilson 95% interval;
- per N: the coexistence interval (densities whose jam fraction is strictly
  between 0 and 1) and rho_c, where the jam fraction crosses 1/2 (linear
  interpolation between the grid densities).

Lattices up to `ensemble_max_n` columns run as one batched ensemble per size
(jam early exit); larger ones run on the single-lattice kernels, several at
a time on their own streams, each stopping at its first step with no move.  Every step, count and trace comes
from the CUDA library; this module orders the calls and averages integers.
"""
from __future__ import annotations

import json
import math
import time

import numpy as np

from . import bml

EMPTY, LR, TB = 0, 1, 2
# Fig. 1 colours: LR red, TB blue, empty white
COLOURS = np.array([[255, 255, 255], [215, 25, 28], [44, 90, 200]], dtype=np.uint8)


def write_ppm(path: str, lattice: np.ndarray, scale: int = 1) -> None:
    """Binary PPM (P6) of a lattice, one pixel (or scale x scale pixels) per
    cell, row 0 at the top."""
    g = np.asarray(lattice, dtype=np.uint8)
    if g.ndim != 2 or g.max(initial=0) > TB:
        raise ValueError("lattice must be 2-D with cells 0, 1, 2")
    rgb = COLOURS[g]
    if scale > 1:
        rgb = rgb.repeat(scale, axis=0).repeat(scale, axis=1)
    h, w = rgb.shape[:2]
    with open(path, "wb") as f:
        f.write(b"P6\n%d %d\n255\n" % (w, h))
        f.write(np.ascontiguousarray(rgb).tobytes())


def wilson(k: int, n: int, z: float = 1.96):
    """Wilson score interval of a binomial proportion k / n."""
    if n == 0:
        return 0.0, 1.0
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return max(0.0, c - h), min(1.0, c + h)


def _runs_ensemble(N, densities, seeds, T, window, stream):
    rho = np.repeat(np.asarray(densities, dtype=np.float64), seeds)
    seed = np.tile(np.arange(1, seeds + 1, dtype=np.uint64), len(densities))
    M = np.full(rho.size, N, dtype=np.int64)
    with bml.Ensemble(M, M.copy(), seed, rho / 2, rho / 2, flags=bml.BML_ENS_EARLY_EXIT,
                      stream=stream, reserve_steps=T) as ens:
        cars = ens.car_counts()
        ens.step(T)
        lr, tb = ens.traces(T - window, window)
        jam = ens.jam_steps() >= 0
    moved = (lr + tb).sum(axis=1)
    v = np.where(cars > 0, moved / (window * np.maximum(cars, 1)), 0.0)
    return rho, v, jam


def _runs_single(N, densities, seeds, T, window, stream, chunk=1024, lanes=6, tiling=None):
    """Lattices too wide for the ensemble, each through the autotuned
    single-lattice kernel (or the given (depth, band rows, words per lane)),
    `lanes` of them at a time on their own streams (one lattice of this size
    occupies only part of the GPU): every `chunk` steps the counts are read
    and a run stops at its first step with no move."""
    import torch
    jobs = [(r, s) for r in densities for s in range(1, seeds + 1)]
    out = [None] * len(jobs)
    streams = [torch.cuda.Stream() for _ in range(lanes)]
    active = []  # [job, sim, cars, done, jammed, stream slot]
    nxt = 0
    free = list(range(lanes))
    while nxt < len(jobs) or active:
        while free and nxt < len(jobs):
            r, s = jobs[nxt]
            slot = free.pop()
            sim = bml.Lattice(N, N, seed=s, density=r, stream=streams[slot], reserve_steps=T)
            if tiling:
                sim.set_tiling(*tiling)
            active.append([nxt, sim, int(np.count_nonzero(sim.read())), 0, False, slot])
            nxt += 1
        for a in active:  # enqueue one chunk of every run, then read them
            a[1].step(min(chunk, T - a[3]))
        still = []
        for a in active:
            job, sim, cars, done, _, slot = a
            n = min(chunk, T - done)
            tot, _, _ = sim.moved_counts(done, n)
            done += n
            jammed = bool(np.any(tot == 0))
            if done < T and not jammed:
                a[3] = done
                still.append(a)
                continue
            # steps not run (after a jam) move nothing
            start = T - window
            moved = 0
            if done > start:
                tot, _, _ = sim.moved_counts(start, done - start)
                moved = int(tot.sum())
            out[job] = (jobs[job][0], moved / (window * cars) if cars else 0.0, jammed)
            sim.close()
            free.append(slot)
        active = still
    torch.cuda.synchronize()
    return (np.array([o[0] for o in out]), np.array([o[1] for o in out]),
            np.array([o[2] for o in out]))


def phase_diagram(sizes, densities, seeds, T, window, ensemble_max_n=2048, stream=None,
                  single_seeds=None, single_tiling=None) -> dict:
    """Curves per size: {N: {"rho", "v_mean", "jam_frac", "jam_ci", "runs",
    "coexistence", "rho_c", "seconds"}}."""
    out = {}
    for N in sizes:
        t0 = time.perf_counter()
        if N <= ensemble_max_n:
            S = seeds
            rho, v, jam = _runs_ensemble(N, densities, S, T, window, stream)
        else:
            S = single_seeds or seeds
            rho, v, jam = _runs_single(N, densities, S, T, window, stream,
                                       tiling=single_tiling)
        secs = time.perf_counter() - t0
        keys = np.asarray(densities, dtype=np.float64)
        v_mean = np.array([v[rho == k].mean() for k in keys])
        k_jam = np.array([int(jam[rho == k].sum()) for k in keys])
        n_run = np.array([int((rho == k).sum()) for k in keys])
        frac = k_jam / n_run
        ci = [wilson(int(a), int(b)) for a, b in zip(k_jam, n_run)]
        coex = [float(k) for k, f in zip(keys, frac) if 0.0 < f < 1.0]
        rho_c = None
        for i in range(len(keys) - 1):
            if frac[i] < 0.5 <= frac[i + 1]:
                rho_c = float(keys[i] + (0.5 - frac[i]) * (keys[i + 1] - keys[i])
                              / (frac[i + 1] - frac[i]))
                break
        out[int(N)] = {"rho": keys.tolist(), "v_mean": v_mean.tolist(),
                       "jam_frac": frac.tolist(), "jam_ci": ci, "runs": n_run.tolist(),
                       "coexistence": [min(coex), max(coex)] if coex else None,
                       "rho_c": rho_c, "seeds": S, "seconds": secs,
                       "cell_steps_upper_bound": float(N) * N * T * len(keys) * S}
    return out


def fig1(prefix: str, N: int = 256, densities=(0.25, 0.32, 0.38), steps: int = 4096,
         seed: int = 1, scale: int = 2, stream=None) -> list:
    """The three Fig. 1 configurations (N x N after `steps` steps, seeded
    placement at each density); writes <prefix>_rho<rho>.ppm and returns
    (path, velocity over the last 64 steps) per density."""
    res = []
    for r in densities:
        with bml.Lattice(N, N, seed=seed, density=r, stream=stream,
                         reserve_steps=steps) as sim:
            cars = int(np.count_nonzero(sim.read()))
            sim.step(steps)
            g = sim.read()
            tot, _, _ = sim.moved_counts(steps - 64, 64)
        path = "%s_rho%.2f.ppm" % (prefix, r)
        write_ppm(path, g, scale)
        res.append((path, float(tot.mean() / max(cars, 1))))
    return res


# single_tiling: the 4096^2 runs go six at a time, so each takes a share of
# the GPU; two words per lane at depth 8 with bands of 32 rows (a 4096-column
# row is one cyclic group of 32 lanes) beat the tiling autotuned for a lattice
# alone (depth 4, band 16) by 12% and one word per lane with 64-row bands by
# 27% on six concurrent lattices.
FULL = {"sizes": [256, 512, 1024, 2048, 4096],
        "densities": [round(0.20 + 0.01 * i, 2) for i in range(31)],
        "seeds": 32, "single_seeds": 8, "T": 100000, "window": 1024,
        "single_tiling": (8, 32, 2)}

SMALL = {"sizes": [64, 128, 256], "densities": [round(0.20 + 0.04 * i, 2) for i in range(8)],
         "seeds": 8, "single_seeds": 4, "T": 8192, "window": 256}


if __name__ == "__main__":
    import os
    import sys
    cfg = FULL if "--full" in sys.argv else SMALL
    out_dir = next((a.split("=", 1)[1] for a in sys.argv if a.startswith("--out=")), ".")
    os.makedirs(out_dir, exist_ok=True)
    t0 = time.perf_counter()
    curves = phase_diagram(cfg["sizes"], cfg["densities"], cfg["seeds"], cfg["T"],
                           cfg["window"], single_seeds=cfg["single_seeds"],
                           single_tiling=cfg.get("single_tiling"))
    total = time.perf_counter() - t0
    pics = fig1(os.path.join(out_dir, "fig1"))
    print(json.dumps({"config": cfg, "seconds": total, "curves": curves, "fig1": pics}))
