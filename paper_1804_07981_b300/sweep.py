"""Surrogate-guided density sweep: allocating long-run step budgets.

A density sweep asks, for every (density, seed) run of an L x L lattice, for
the steady-state velocity and whether the run jams within T_long steps (the
phase behaviour of Sec. 2 of the paper: free-flowing below the transition,
globally jammed above it, coexistence near it).  Running every run to T_long
is the exact answer; most runs are settled long before.

Every step of the automaton, the features, the labels and the network run in
the CUDA library; this module only orders the calls.

Arms:

- exact: all runs to T_long in one ensemble with jam early exit (a run that
  jammed costs nothing afterwards, and its answer is exact).
- surrogate: all runs to B0 (jam early exit).  At step `probe` the network
  reads the features (density, size, `points` window means of the moved
  fraction over the first `probe` steps) and predicts the jam probability.
  A run jammed by B0 is answered exactly (jam, velocity 0).  A run that is
  flowing freely at B0 (velocity over the last `window` steps >= v_free)
  and that the network is confident will not jam (p < tau) stops at B0 and
  is answered by that velocity.  Every other run continues exactly to
  T_long in a second ensemble.
- no surrogate (what the method gives without the network): the same B0
  stage, then every run not jammed by B0 must continue to T_long, since
  nothing tells which of them will still jam.

The exact arm judges the others: per-density mean velocity and jam fraction.
It also judges the network itself (network_scores): the error of its
velocity prediction v_hat and how often its jam probability is on the wrong
side of 0.5 and of the allocator's threshold.  The answers of runs stopped
at B0 are their measured window velocities, not v_hat: the measurement is
the closer of the two (its error against the exact arm is reported beside
v_hat's), so the velocity head is trained and scored as the network's
velocity predictor, and the allocation reads only the jam head.
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import bml
from .inputs import ensemble_params

POINTS = 64
PROBE = 512


def _sync(torch):
    torch.cuda.synchronize()


def training_set(count, T, window, seed, lo=64, hi=2048, stream=None):
    """Batched-ensemble runs with M, N uniform on {lo..hi}, density uniform on
    [0.1, 0.6], LR fraction uniform on [0.3, 0.7]; returns device tensors
    (features at PROBE steps, velocity label, jam label) and the seconds."""
    import torch
    p = ensemble_params(count, seed=seed, lo=lo, hi=hi)
    t0 = time.perf_counter()
    ens = bml.Ensemble(p["M"], p["N"], p["seed"] + np.uint64(seed * 100003), p["p_lr"],
                       p["p_tb"], flags=bml.BML_ENS_EARLY_EXIT, stream=stream,
                       reserve_steps=T)
    ens.step(PROBE)
    X = ens.features(0, PROBE, POINTS)
    ens.step(T - PROBE)
    v, jam = ens.labels(window)
    _sync(torch)
    secs = time.perf_counter() - t0
    ens.close()
    return X, v, jam, secs


def train(X, v, jam, steps=2000, batch=1024, lr=1e-3, wd=1e-4, seed=0, stream=None,
          loss_tail=50):
    """AdamW on mini-batches drawn on the device (bml_mlp_train: one call,
    the draw, gather and steps all enqueued on the network's stream);
    returns the network and the losses of the first step and of the last
    `loss_tail` steps."""
    from .inputs import mlp_init_params
    net = bml.MLP(stream=stream)
    net.set_params(mlp_init_params(X.shape[1], seed).astype(np.float32))
    losses = net.train(X, v, jam, steps, min(batch, X.shape[0]), lr=lr, weight_decay=wd,
                       seed=seed + 1)
    return net, [float(losses[0])] + [float(x) for x in losses[-loss_tail:]]


def sweep_runs(densities, n_seeds, L):
    rho = np.repeat(np.asarray(densities, dtype=np.float64), n_seeds)
    seeds = np.tile(np.arange(1, n_seeds + 1, dtype=np.uint64), len(densities))
    M = np.full(rho.size, L, dtype=np.int64)
    return M, M.copy(), seeds, rho / 2, rho / 2, rho


def exact_arm(runs, T_long, window, stream=None):
    import torch
    M, N, seeds, plr, ptb, _ = runs
    t0 = time.perf_counter()
    ens = bml.Ensemble(M, N, seeds, plr, ptb, flags=bml.BML_ENS_EARLY_EXIT, stream=stream,
                       reserve_steps=T_long)
    ens.step(T_long)
    v, jam = ens.labels(window)
    _sync(torch)
    secs = time.perf_counter() - t0
    out = (v.cpu().numpy().astype(np.float64), jam.cpu().numpy().astype(np.float64))
    ens.close()
    return out, secs


def surrogate_arm(runs, net, T_long, B0, window, tau, v_free=0.99, stream=None, use_net=True,
                  predictions=None):
    """Returns ((v, jam) answers, seconds, number of runs extended to T_long).
    predictions (a dict, optional) receives the network's own outputs per run:
    "v_hat" (predicted steady-state velocity) and "p_jam"."""
    import torch
    M, N, seeds, plr, ptb, _ = runs
    t0 = time.perf_counter()
    ens = bml.Ensemble(M, N, seeds, plr, ptb, flags=bml.BML_ENS_EARLY_EXIT, stream=stream,
                       reserve_steps=T_long)
    ens.step(PROBE)
    if use_net:
        X = ens.features(0, PROBE, POINTS)
        out = net.forward(X)
        p_jam = torch.sigmoid(out[:, 1]).cpu().numpy()
        if predictions is not None:
            predictions["v_hat"] = out[:, 0].cpu().numpy().astype(np.float64)
            predictions["p_jam"] = p_jam.astype(np.float64)
    ens.step(B0 - PROBE)
    v0, jam0 = (t.cpu().numpy().astype(np.float64) for t in ens.labels(window))
    jammed = jam0 > 0
    if use_net:
        extend = ~jammed & ((p_jam >= tau) | (v0 < v_free))
    else:
        extend = ~jammed
    v, jam = np.where(jammed, 0.0, v0), jam0.copy()
    idx = np.flatnonzero(extend)
    if use_net and predictions is not None:
        predictions["v_B0"] = v0
        predictions["stopped"] = ~jammed & ~extend
    if idx.size:
        # the other runs stop here; the extended ones go on in the same ensemble
        ens.retire(np.flatnonzero(~extend))
        ens.step(T_long - B0)
        ve, je = (t.cpu().numpy().astype(np.float64) for t in ens.labels(window))
        v[idx], jam[idx] = ve[idx], je[idx]
    _sync(torch)
    secs = time.perf_counter() - t0
    ens.close()
    return (v, jam), secs, int(idx.size)


def plain_byte_estimate(runs, T_long, every, sample_stride, chunk=1024, stream=None):
    """The plain per-lattice GPU form on the same sweep: one lattice at a time
    with the byte-per-cell kernel, stepping in chunks of `chunk` and stopping
    a run once a step moved no car (the same early exit as the other arms).
    Times every `sample_stride`-th density with one seed and extrapolates
    each sampled time to that density's runs and to the densities skipped
    between samples."""
    import torch
    M, N, seeds, plr, ptb, rho = runs
    keys = np.unique(rho)
    per_key = {}
    sampled = keys[::sample_stride]
    for k in sampled:
        i = int(np.flatnonzero(rho == k)[0])
        _sync(torch)
        t0 = time.perf_counter()
        sim = bml.Lattice(int(M[i]), int(N[i]), seed=int(seeds[i]), p_lr=float(plr[i]),
                          p_tb=float(ptb[i]), kernel="byte", stream=stream,
                          reserve_steps=T_long)
        done = 0
        while done < T_long:
            n = min(chunk, T_long - done)
            sim.step(n)
            tot, _, _ = sim.moved_counts(done, n)
            done += n
            if np.any(tot == 0):
                break
        sim.close()
        per_key[float(k)] = time.perf_counter() - t0
    sk = np.array(sorted(per_key))
    est = 0.0
    for k in keys:
        nearest = sk[np.argmin(np.abs(sk - k))]
        est += per_key[float(nearest)] * np.sum(rho == k)
    return est, {"sampled_densities": len(sk), "seconds_sampled": float(sum(per_key.values()))}


def per_density(rho, v, jam):
    keys = np.unique(rho)
    return (keys, np.array([v[rho == k].mean() for k in keys]),
            np.array([jam[rho == k].mean() for k in keys]))


def compare(runs, answer, exact):
    rho = runs[5]
    _, ve, je = per_density(rho, *exact)
    _, va, ja = per_density(rho, *answer)
    return {"max_abs_dv": float(np.max(np.abs(va - ve))),
            "max_abs_djam_fraction": float(np.max(np.abs(ja - je))),
            "run_velocity_mae": float(np.mean(np.abs(answer[0] - exact[0]))),
            "run_jam_misclassified": float(np.mean(answer[1] != exact[1]))}


# density bands of the network's score table (a band holds its lower bound)
SCORE_BANDS = (0.25, 0.30, 0.35, 0.40, 0.45)
# jam-probability bins of the calibration table
CAL_BINS = (0.0, 0.01, 0.1, 0.5, 0.9, 0.99, 1.0)


def network_scores(pred, exact, rho, tau, bands=SCORE_BANDS):
    """The network's own accuracy against the exact runs to T_long: its
    velocity prediction v_hat (absolute error, cars per step per car,
    overall and per density band) and its jam probability (misclassified
    runs at p = 0.5 with the false negatives and positives, the same at the
    allocator's threshold tau, and a calibration table: per probability bin
    the runs and the fraction that jammed)."""
    v_hat, p = pred["v_hat"], pred["p_jam"]
    v, jam = exact[0], exact[1] > 0
    err = np.abs(v_hat - v)
    out = {"runs": int(v.size), "v_mae": float(err.mean()), "v_max_abs_err": float(err.max()),
           "v_mae_flowing": float(err[~jam].mean()) if (~jam).any() else None,
           "v_mae_jammed": float(err[jam].mean()) if jam.any() else None}
    per = []
    edges = list(bands)
    for lo, hi in zip(edges[:-1], edges[1:]):
        last = hi == edges[-1]
        sel = (rho >= lo - 1e-9) & ((rho <= hi + 1e-9) if last else (rho < hi - 1e-9))
        if sel.any():
            per.append({"rho": [lo, hi], "runs": int(sel.sum()), "v_mae": float(err[sel].mean()),
                        "jam_fraction": float(jam[sel].mean()),
                        "jam_misclassified": float(np.mean((p[sel] >= 0.5) != jam[sel]))})
    out["per_density_band"] = per
    # reference predictors that know the exact per-density outcome of the
    # sweep itself (not available to an allocator): the per-density jam
    # fraction thresholded at 1/2, and the per-density mean velocity; and
    # the trivial one (the sweep's majority class, its mean velocity)
    keys = np.unique(rho)
    dens_jam_err = sum(min(jam[rho == k].mean(), 1 - jam[rho == k].mean()) * np.sum(rho == k)
                       for k in keys) / rho.size
    dens_v_err = sum(np.abs(v[rho == k] - v[rho == k].mean()).sum() for k in keys) / rho.size
    out["reference_predictors"] = {
        "jam_misclassified_per_density_fraction": float(dens_jam_err),
        "jam_misclassified_majority": float(min(jam.mean(), 1 - jam.mean())),
        "v_mae_per_density_mean": float(dens_v_err),
        "v_mae_global_mean": float(np.abs(v - v.mean()).mean())}
    if "stopped" in pred and pred["stopped"].any():
        st = pred["stopped"]
        # the runs the allocator stopped at B0: their answer (the measured
        # window velocity) against the network's prediction
        out["stopped_at_B0"] = {"runs": int(st.sum()),
                                "answer_v_mae": float(np.mean(np.abs(pred["v_B0"][st] - v[st]))),
                                "v_hat_mae": float(err[st].mean()),
                                "jammed_later": int(np.sum(jam[st]))}
    for name, thr in (("p0.5", 0.5), ("tau", tau)):
        said = p >= thr
        out["jam_" + name] = {"threshold": thr,
                              "misclassified": float(np.mean(said != jam)),
                              "false_negatives": int(np.sum(jam & ~said)),
                              "false_positives": int(np.sum(~jam & said))}
    cal = []
    for lo, hi in zip(CAL_BINS[:-1], CAL_BINS[1:]):
        sel = (p >= lo) & ((p <= hi) if hi == CAL_BINS[-1] else (p < hi))
        cal.append({"p": [lo, hi], "runs": int(sel.sum()),
                    "jammed": float(jam[sel].mean()) if sel.any() else None})
    out["calibration"] = cal
    return out


def run(cfg: dict, stream=None) -> dict:
    """Train the surrogate, then run the three arms on one sweep; returns a
    summary dict (times in seconds)."""
    import torch
    X, v, jam, t_data = training_set(cfg["train_count"], cfg["train_T"], cfg["window"],
                                     seed=cfg.get("train_seed", 7), lo=cfg["train_lo"],
                                     hi=cfg["train_hi"], stream=stream)
    t0 = time.perf_counter()
    net, losses = train(X, v, jam, steps=cfg["train_steps"], stream=stream)
    _sync(torch)
    t_train = time.perf_counter() - t0
    runs = sweep_runs(cfg["densities"], cfg["seeds"], cfg["L"])
    exact, t_exact = exact_arm(runs, cfg["T_long"], cfg["window"], stream)
    pred = {}
    sur, t_sur, n_ext = surrogate_arm(runs, net, cfg["T_long"], cfg["B0"], cfg["window"],
                                      cfg["tau"], cfg["v_free"], stream, predictions=pred)
    base, t_base, n_base = surrogate_arm(runs, None, cfg["T_long"], cfg["B0"], cfg["window"],
                                         cfg["tau"], cfg["v_free"], stream, use_net=False)
    plain = None
    if cfg.get("plain_sample_stride"):
        est, info = plain_byte_estimate(runs, cfg["T_long"], every=1,
                                        sample_stride=cfg["plain_sample_stride"], stream=stream)
        plain = {"seconds_estimated": est, **info}
    saved = t_exact - t_sur
    return {
        "plain_byte_per_lattice": plain,
        "config": cfg, "runs": int(runs[0].size),
        "training": {"seconds_data": t_data, "seconds_train": t_train,
                     "loss_first": losses[0], "loss_last": float(np.mean(losses[-50:])),
                     # sweeps after which the one-time training has paid for itself
                     # against the exact batched arm (None if no sweep saves time)
                     "break_even_sweeps_vs_exact":
                         (t_data + t_train) / saved if saved > 0 else None},
        "network": network_scores(pred, exact, runs[5], cfg["tau"]),
        "exact": {"seconds": t_exact},
        "surrogate": {"seconds": t_sur, "extended_runs": n_ext, **compare(runs, sur, exact)},
        "no_surrogate": {"seconds": t_base, "extended_runs": n_base,
                         **compare(runs, base, exact)},
    }


FULL = {
    "densities": [round(0.25 + 0.005 * i, 3) for i in range(41)], "seeds": 64, "L": 1024,
    "T_long": 100000, "B0": 10000, "window": 1024, "tau": 0.01, "v_free": 0.99,
    "train_count": 4096, "train_T": 100000, "train_lo": 64, "train_hi": 2048,
    "train_steps": 4000, "plain_sample_stride": 4,
}

SMALL = {
    "densities": [round(0.25 + 0.02 * i, 3) for i in range(11)], "seeds": 16, "L": 128,
    "T_long": 8192, "B0": 2048, "window": 256, "tau": 0.01, "v_free": 0.99,
    "train_count": 4096, "train_T": 8192, "train_lo": 64, "train_hi": 256,
    "train_steps": 3000,
}


if __name__ == "__main__":
    import sys
    cfg = FULL if "--full" in sys.argv else SMALL
    print(json.dumps(run(cfg)))
