"""Throughput benchmark of the BML lattice step on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload: one 32768 x 32768 periodic lattice per GPU (1.07 G cells, 256 MB
of bitplanes), density 0.38 split evenly LR/TB, seeded placement (seed 1 on
rank 0, 1 + rank elsewhere), moved counts recorded every step.  One bench
step is bml_step(sim, 8): eight full lattice steps, so the default 1250
steps are 10^4 lattice steps.  Metric: cell-updates/s over the whole job.

The bitplane state (2 x 256 MB, ping-pong) is larger than the 126 MB L2, so
no flush is needed between timed steps.  With --gpus N > 1 (torchrun) each
rank runs an independent replica (weak scaling); there is no data-path
collective.

Sub-measurements on the same JSON line: "ensemble" (4096 lattices, the
batched API, the workload's full 10^4 steps timed; with "cpu_oracle", the
oracle on all host cores on a subset of the lattices, extrapolated), "model2" (the Sec. 2 Model II variant on the bench lattice,
tie-break seed = placement seed, 1024 steps; --no-model2 skips it and "model3"),
"model3" (the Model III reading on the bench lattice, 1024 steps),
"byte_kernel" (the plain byte-per-cell form on the bench lattice, 16 steps,
against the HBM peak), "two_phase" (the two-phase bitplane form, a horizontal and
a vertical kernel per step, 64 steps, against the HBM peak), "one_pass" (one full step
per DRAM pass on the bench lattice, 256 steps, against the HBM peak), "configs" (256^2
for 1024 steps; 4096^2 byte vs
bit-packed over 3 densities x 3 seeds x 4096 steps, with the oracle's one-core time per run
estimated from a bounded sample; rank 0 of a 1-GPU run), "mlp" (the
surrogate network: AdamW step time at batch 1024, forward on 2624 samples, and its tcgen05
GEMM kernel on a 2^22 x 128 x 128 product against the HBM peak; 1-GPU runs).
The line ends with "summary", the headline number of each of them again.

--impl reference times the CPU oracle (test infrastructure) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

M_ROWS = N_COLS = 32768
DENSITY = 0.38
STEPS_PER_BENCH_STEP = 8
BYTES_PER_CELL_STEP = 0.5  # 2 bits read + 2 bits written per cell per step
WORKLOAD = "bml_32768x32768_rho0.38"


def workload_name(M, N):
    return "bml_%dx%d_rho%.2f" % (M, N, DENSITY)
# 32-bit integer ALU operations the bitplane step needs per 64-cell word:
# E, Er, mvH, in, Lh, mvV, T' (two 32-bit operations each; mvV = T_{x-1} &
# ~(Lh_x | T_x) is one three-input operation) and the two count additions;
# popcounts run on another pipe and are not counted
ALU_OPS_PER_CELL_STEP = 16.0 / 64.0
# Model II (one synchronous phase, random tie-break), per 64-cell word and
# step: E, fromL (funnel), inLR (2: E & fromL & (~T_{x-1} | coin)), inTB (2),
# mvH (funnel), L', T' = 9 operations per 32-bit half = 18; the tie-break
# word (SplitMix64: three xor-shifts of 64 bits = 12, a 64-bit add = 2; its
# multiplies run on the FMA pipe); 2 count additions: 34 per 64 cell-steps
MODEL2_ALU_OPS_PER_CELL_STEP = 34.0 / 64.0
SMS = 148
ALU_LANES_PER_SM_CLK = 64  # integer ALU pipe: 2 warp instructions per clock per SM
SM_MAX_MHZ = 2032.0
# DRAM bytes (read + write, as counted by ncu for one launch) per cell, from
# the captures summarised in profiles/ (32768 x 32768, the kernels as they are
# now), keyed by kernel and band rows (the captured tiling); scaled by the
# cell count of the run.  A kernel or tiling without an entry (or a kernel
# changed since its capture) reports traffic null.
TRAFFIC_PER_CELL = {("stream2_kernel<8>", 231): 0.4719, ("stream2_kernel<1>", 16): 0.4520,
                    ("stream2_kernel<4, Model II>", 154): 0.4671}
# the ensemble kernel per cell and chunk of 8 steps (bands of 608 rows, the
# autotuner's pick on a B300: one launch of 8 chunks captured, 20.69 GB over
# 4.55e9 cells)
ENS_TRAFFIC_PER_CELL_CHUNK = {(8, 608): 0.5686}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.tmp = None

    def start(self):
        try:
            self.tmp = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.tmp, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.tmp.flush()
        with open(self.tmp.name) as fh:
            rows = [r for r in csv.reader(io.StringIO(fh.read())) if len(r) >= 9]
        os.unlink(self.tmp.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4)
                          if r[5 + k].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def dist_max(x: float, world: int, device: str = "cuda") -> float:
    """Maximum of x over all ranks (x itself when world == 1)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    units_per_rank units, timed by the slowest rank (weak scaling)."""
    return world * units_per_rank / seconds


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _cpu_sample(budget_s: float, threads: int):
    """Time the oracle, as it stands, on a band of rows of the workload
    (periodic R x 32768 lattice, same density and placement rule), repeating
    8-step runs until about `budget_s` seconds of CPU work.  Returns
    (cell-updates/s, description, seconds)."""
    import oracle
    rows = 2048
    g = oracle.init(rows, N_COLS, 1, DENSITY / 2, DENSITY / 2)
    done = 0
    t0 = time.perf_counter()
    while True:
        g, _, _ = oracle.run(g, STEPS_PER_BENCH_STEP, threads=threads)
        done += STEPS_PER_BENCH_STEP
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    rate = rows * N_COLS * done / dt
    desc = ("oracle (C, OpenMP rows, %d threads) on a %d x %d periodic band of the workload "
            "(density %.2f), %d steps in %.1f s" % (threads, rows, N_COLS, DENSITY, done, dt))
    return rate, desc, dt


def _oracle_ensemble_sample(budget_s: float, threads: int):
    """The oracle, as it stands, on a subset of the ensemble workload (every
    64th lattice; 8-step runs per lattice, row-parallel on `threads` cores,
    repeated until about `budget_s` seconds), extrapolated to the whole
    ensemble: lattice-steps/s at the workload's mean lattice size."""
    import oracle
    from paper_1804_07981_b300.inputs import ensemble_params
    p = ensemble_params(4096, seed=1)
    idx = np.arange(0, 4096, 64)
    gs = [oracle.init(int(p["M"][l]), int(p["N"][l]), int(p["seed"][l]), float(p["p_lr"][l]),
                      float(p["p_tb"][l])) for l in idx]
    cells = 0
    t0 = time.perf_counter()
    while True:
        for j, g in enumerate(gs):
            gs[j], _, _ = oracle.run(g, 8, threads=threads)
            cells += g.size * 8
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    rate = cells / dt
    mean_cells = float((p["M"] * p["N"]).sum()) / 4096
    return {"value": rate / mean_cells, "unit": "lattice-steps/s", "cores": threads,
            "kind": "oracle", "cell_updates_per_s": rate,
            "sample": "64 lattices of the workload (every 64th), 8-step runs, %.1f s; "
                      "extrapolated at the mean lattice size" % dt}


def _cpu_ladder_sample(threads: int, N: int = 2048, steps: int = 64):
    """The paper's CPU implementations (oracle/cpu_ladder.c: serial with
    ghost cells, OpenMP, SIMD, OpenMP+SIMD, and a bit-packed OpenMP form) on
    an N x N lattice at the Fig. 3 density 0.3, `steps` steps each (a bounded
    sample of the paper's protocol; the full one: python -m oracle.ladder
    --fig3).  Each result is checked against the oracle.  Reported baselines,
    not targets."""
    import oracle
    from oracle import ladder
    g0 = oracle.init(N, N, 1, 0.15, 0.15)
    t0 = time.perf_counter()
    want, _, _ = oracle.run(g0, steps, threads=1)
    out = {"serial (oracle)": N * N * steps / (time.perf_counter() - t0)}
    for form, name in sorted(ladder.FORMS.items()):
        got, dt = ladder.run(form, g0, steps, threads)
        assert np.array_equal(got, want), name
        out[name] = N * N * steps / dt
    return {"unit": "cell-updates/s", "cores": threads, "kind": "cpu implementations of the "
            "paper (Secs. 3-5)", "sample": "%d x %d, density 0.3, %d steps" % (N, N, steps),
            "value_by_form": out}


def _oracle_1core_4096(budget_s: float):
    """The oracle on one core, one 4096 x 4096 run (density 0.35, seed 1),
    timed over whole 8-step runs for about `budget_s` seconds and scaled to the
    4096 steps of a run."""
    import oracle
    g = oracle.init(4096, 4096, 1, 0.175, 0.175)
    steps = 0
    t0 = time.perf_counter()
    while True:
        g, _, _ = oracle.run(g, 8, threads=1)
        steps += 8
        dt = time.perf_counter() - t0
        if dt >= budget_s:
            break
    return {"cell_updates_per_s": 4096 * 4096 * steps / dt,
            "seconds_per_run_estimate": dt / steps * 4096, "cores": 1,
            "sample": "%d steps of one 4096^2 run in %.1f s" % (steps, dt)}


def _ensemble_bench(bml, torch, stream, steps, seed_base=1, tiling=None, sm_mhz=SM_MAX_MHZ):
    """Batched ensemble of 4096 lattices (M, N uniform on {64..2048}, density
    uniform on [0.1, 0.6], LR fraction uniform on [0.3, 0.7]), autotuned,
    graph-replayed; `steps` steps timed with CUDA events after a warm-up.
    Roofline: the integer ALU pipe, the bitplane step's algorithmic
    operations (ALU_OPS_PER_CELL_STEP) against 148 SMs x 64 lanes x the SM
    clock."""
    from paper_1804_07981_b300.inputs import ensemble_params
    p = ensemble_params(4096, seed=1)
    k, band = tiling if tiling else (0, 0)  # 0, 0: autotuned
    ens = bml.Ensemble(p["M"], p["N"], p["seed"] + np.uint64(seed_base - 1), p["p_lr"],
                       p["p_tb"], block_k=k, band_rows=band, stream=stream,
                       reserve_steps=steps + 64)
    ens.step(32)
    ens.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ens.step(steps)
    e1.record(stream)
    e1.synchronize()
    ens.synchronize()
    ms = e0.elapsed_time(e1)
    cells = int((p["M"] * p["N"]).sum())
    k, band, graphs = ens.config
    ens.close()
    cu = cells * steps / (ms / 1e3)
    ops = cu * ALU_OPS_PER_CELL_STEP / 1e12
    peak = SMS * ALU_LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    return {"metric": "ensemble lattice-steps/s", "lattices": 4096, "steps": steps,
            "seconds": ms / 1e3, "unit": "lattice-steps/s",
            "cell_updates_per_s": cu, "cells": cells,
            "roofline": {"bound": "alu", "kernel": "ens_kernel<%d>" % k, "achieved": ops,
                         "peak": peak, "unit": "Tops/s", "frac": ops / peak,
                         "ops_per_cell_step": ALU_OPS_PER_CELL_STEP,
                         "traffic_per_chunk": (ENS_TRAFFIC_PER_CELL_CHUNK[(k, band)] * cells
                                               if (k, band) in ENS_TRAFFIC_PER_CELL_CHUNK
                                               else None),
                         "chunk_steps": k},
            "temporal_depth": k, "band_rows": band, "graph": graphs,
            "workload": "4096 lattices, M,N ~ U{64..2048}, rho ~ U[0.1,0.6], "
                        "LR fraction ~ U[0.3,0.7], seeds 1..4096"}


def _model2_bench(bml, torch, stream, M, N, steps, sm_mhz, seed=1, tiling=None, model=2):
    """Model II (model=2) or Model III (model=3) on the bench lattice (same
    placement), autotuned, `steps` steps timed with CUDA events after a
    warm-up; the counts of the timed steps are checked for plausibility."""
    # explicit tiling: a TBLOCK object (no autotuning launches); else AUTO
    kernel, bk = ("tblock", tiling[0]) if tiling else ("auto", 0)
    with bml.Lattice(M, N, seed=seed, density=DENSITY, kernel=kernel, block_k=bk,
                     stream=stream, reserve_steps=steps + 64) as sim:
        sim.set_model(bml.BML_MODEL_II if model == 2 else bml.BML_MODEL_III, seed)
        if tiling:
            sim.set_tiling(*tiling)
        k, band, lw = sim.tiling
        sim.step(3 * k)
        sim.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        tot, _, _ = sim.moved_counts(3 * k, steps)
        cells = M * N
        assert (tot >= 0).all() and (tot <= cells).all()
    launches = (steps + k - 1) // k
    # Model III's step is the paper's model's with the vertical moves read
    # from the step's start: the same operation count
    per = MODEL2_ALU_OPS_PER_CELL_STEP if model == 2 else ALU_OPS_PER_CELL_STEP
    ops = per * cells * steps
    achieved = ops / (ms / 1e3) / 1e12
    peak = SMS * ALU_LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12
    if model == 2:
        kname = ("stream2_kernel<%d, Model II>" if lw == 2 else "model2_kernel<%d>") % k
    else:
        kname = ("stream2_kernel<%d, Model III>" if lw == 2 else "stream_kernel<%d, Model III>") % k
    return {"metric": "cell-updates/s", "value": cells * steps / (ms / 1e3),
            "unit": "cell-updates/s", "steps": steps, "seconds": ms / 1e3,
            "workload": workload_name(M, N) + ("_model2_tie1" if model == 2 else "_model3"),
            "kernel": kname,
            "temporal_depth": k, "band_rows": band, "lane_words": lw,
            "gpu_launches": launches,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak,
                         "traffic": (TRAFFIC_PER_CELL[(kname, band)] * cells
                                     if (kname, band) in TRAFFIC_PER_CELL else None),
                         "ops_per_cell_step": per}}


def _timed_steps(torch, stream, sim, steps):
    """Milliseconds of `steps` steps on the object's stream (CUDA events)."""
    sim.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def _byte_bench(bml, torch, stream, M, N, steps, hbm_peak, seed=1):
    """The plain byte-per-cell form (one byte per cell, a horizontal and a
    vertical kernel per step: 4 B of DRAM traffic per cell-step) on the bench
    lattice."""
    with bml.Lattice(M, N, seed=seed, density=DENSITY, kernel="byte", stream=stream,
                     reserve_steps=steps + 8) as sim:
        sim.step(2)
        ms = _timed_steps(torch, stream, sim, steps)
    cells = M * N
    gbs = 4.0 * cells * steps / (ms / 1e3) / 1e9
    return {"metric": "cell-updates/s", "value": cells * steps / (ms / 1e3),
            "unit": "cell-updates/s", "steps": steps, "seconds": ms / 1e3,
            "kernel": "byte_h + byte_v", "gpu_launches": 2 * steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "bytes_per_cell_step": 4.0}}


def _two_phase_bench(bml, torch, stream, M, N, steps, hbm_peak, seed=1):
    """The two-phase bitplane form on the bench lattice: a horizontal-phase
    kernel (reads L and T, writes L') and a vertical-phase kernel (reads L'
    and T, writes T') per step, 3 + 3 bitplane passes = 0.75 B of DRAM
    traffic per cell-step."""
    with bml.Lattice(M, N, seed=seed, density=DENSITY, kernel="bitplane", stream=stream,
                     reserve_steps=steps + 8) as sim:
        sim.step(2)
        ms = _timed_steps(torch, stream, sim, steps)
    cells = M * N
    gbs = 0.75 * cells * steps / (ms / 1e3) / 1e9
    return {"metric": "cell-updates/s", "value": cells * steps / (ms / 1e3),
            "unit": "cell-updates/s", "steps": steps, "seconds": ms / 1e3,
            "kernel": "plane_h + plane_v", "gpu_launches": 2 * steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "bytes_per_cell_step": 0.75}}


def _one_pass_bench(bml, torch, stream, M, N, steps, hbm_peak, seed=1):
    """One full step per DRAM pass (depth 1) on the bench lattice: the
    two-words-per-lane streaming kernel at depth 1 with 16-row bands (the
    one-word kernel where N does not allow pairs); HBM-bound, 0.5 B per
    cell-step of algorithmic traffic."""
    lw = 2 if (N % 64 == 0 and (N // 64) % 2 == 0 and N // 64 > 32) else 1
    with bml.Lattice(M, N, seed=seed, density=DENSITY, kernel="tblock", block_k=1,
                     stream=stream, reserve_steps=steps + 8) as sim:
        sim.set_tiling(1, 16, lane_words=lw)
        sim.step(3)
        ms = _timed_steps(torch, stream, sim, steps)
    cells = M * N
    gbs = BYTES_PER_CELL_STEP * cells * steps / (ms / 1e3) / 1e9
    kname = "stream2_kernel<1>" if lw == 2 else "stream_kernel<1>"
    traffic = TRAFFIC_PER_CELL.get((kname, 16))
    return {"metric": "cell-updates/s", "value": cells * steps / (ms / 1e3),
            "unit": "cell-updates/s", "steps": steps, "seconds": ms / 1e3,
            "kernel": kname, "temporal_depth": 1, "band_rows": 16, "lane_words": lw,
            "gpu_launches": steps,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak, "unit": "GB/s",
                         "frac": gbs / hbm_peak, "bytes_per_cell_step": BYTES_PER_CELL_STEP,
                         "traffic": traffic * cells if traffic else None}}


def _mlp_bench(bml, torch, stream, hbm_peak, seed=1, gemm_rows=1 << 22):
    """The surrogate network (67 -> 3 x [128, ReLU] -> 2, BF16 on the tcgen05
    GEMM): its GEMM kernel alone on a gemm_rows x 128 x 128 product (C fp32 =
    A bf16 . B^T; at N <= 128 it moves 2 B of A and 4 B of C per 256 flops,
    far below the tensor-core ridge, so its roof is HBM; algorithmic bytes A
    + B + C; one warm-up call, then ten timed ones), then AdamW steps at
    batch 1024 (the sweep's training batch; enqueued back to back, no loss
    read back) and the forward pass on 2624 samples (the sweep's inference
    batch; wall clock per call, which waits)."""
    from paper_1804_07981_b300.inputs import mlp_init_params
    g = torch.Generator(device="cuda").manual_seed(seed)
    out = {}
    with torch.cuda.stream(stream):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        Mg, Ng, Kg = gemm_rows, 128, 128
        A = (torch.rand((Mg, Kg), device="cuda", generator=g) - 0.5).to(torch.bfloat16)
        Bw = (torch.rand((Ng, Kg), device="cuda", generator=g) - 0.5).to(torch.bfloat16)
        C = torch.empty((Mg, Ng), device="cuda", dtype=torch.float32)
        call = lambda: bml.bml_gemm_bf16(A.data_ptr(), Kg, Bw.data_ptr(), Kg, C.data_ptr(), Ng,
                                         Mg, Ng, Kg, stream)
        call()
        ms = []
        for _ in range(10):
            stream.synchronize()
            e0.record(stream)
            call()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms = statistics.median(ms)
        byts = Mg * Kg * 2 + Ng * Kg * 2 + Mg * Ng * 4
        gbs = byts / (ms / 1e3) / 1e9
        out["gemm"] = {"kernel": "umma_gemm_kernel", "shape": [Mg, Ng, Kg], "ms": ms,
                       "tflops": 2.0 * Mg * Ng * Kg / (ms / 1e3) / 1e12,
                       "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm_peak,
                                    "unit": "GB/s", "frac": gbs / hbm_peak,
                                    "bytes": byts,
                                    "note": "event time of one call, including its flag reset "
                                            "and read-back copies"}}
        del A, Bw, C
        net = bml.MLP(stream=stream)
        net.set_params(mlp_init_params(67, seed).astype(np.float32))
        B = 1024
        X = torch.rand((B, 67), device="cuda", generator=g)
        V = torch.rand((B,), device="cuda", generator=g)
        J = (torch.rand((B,), device="cuda", generator=g) > 0.5).float()
        for _ in range(10):
            net.train_step(X, V, J, lr=1e-3, weight_decay=1e-4, want_loss=False)
        steps = 400
        stream.synchronize()
        t0 = time.perf_counter()
        e0.record(stream)
        for _ in range(steps):
            net.train_step(X, V, J, lr=1e-3, weight_decay=1e-4, want_loss=False)
        e1.record(stream)
        e1.synchronize()
        host_s = time.perf_counter() - t0
        out["train_step_us"] = e0.elapsed_time(e1) * 1e3 / steps
        out["train_step_host_us"] = host_s * 1e6 / steps
        out["train_batch"] = B
        out["train_gpu_launches_per_step"] = 17
        Xf = torch.rand((2624, 67), device="cuda", generator=g)
        net.forward(Xf)
        reps = 50
        t0 = time.perf_counter()
        for _ in range(reps):
            net.forward(Xf)
        out["forward_2624_us"] = (time.perf_counter() - t0) * 1e6 / reps
        net.close()
    out["metric"] = "AdamW steps/s"
    out["value"] = 1e6 / out["train_step_us"]
    out["unit"] = "steps/s"
    out["bound"] = "latency (17 launches per step on 1024 samples)"
    return out


def _config_benches(bml, torch, stream):
    """The two smaller workloads: 256 x 256 at density 0.3 (seed 1, 1024
    steps; latency-bound) and 4096 x 4096 at densities 0.20/0.35/0.50,
    seeds 1-3, 4096 steps, byte-per-cell kernel against the autotuned
    bit-packed kernel (lattice creation and autotuning outside the timed
    steps)."""
    out = {}
    with bml.Lattice(256, 256, seed=1, p_lr=0.15, p_tb=0.15, stream=stream,
                     reserve_steps=1024 + 64) as sim:
        ms = _timed_steps(torch, stream, sim, 1024)
        k, band, lw = sim.tiling
    out["256x256_rho0.30_1024steps"] = {"seconds": ms / 1e3,
                                        "cell_updates_per_s": 65536 * 1024 / (ms / 1e3),
                                        "tiling": [k, band, lw]}
    tot = {"byte": 0.0, "auto": 0.0}
    tilings = set()
    for rho in (0.20, 0.35, 0.50):
        for seed in (1, 2, 3):
            for kernel in ("byte", "auto"):
                with bml.Lattice(4096, 4096, seed=seed, density=rho, kernel=kernel,
                                 stream=stream, reserve_steps=4096 + 64) as sim:
                    tot[kernel] += _timed_steps(torch, stream, sim, 4096) / 1e3
                    if kernel == "auto":
                        tilings.add(tuple(sim.tiling))
    cs = 9 * 4096 * 4096 * 4096
    out["4096x4096_rho0.20-0.50_seeds1-3_4096steps"] = {
        "byte_seconds": tot["byte"], "bitplane_seconds": tot["auto"],
        "byte_cell_updates_per_s": cs / tot["byte"],
        "bitplane_cell_updates_per_s": cs / tot["auto"],
        "bitplane_over_byte": tot["byte"] / tot["auto"],
        "bitplane_tilings": sorted(list(t) for t in tilings)}
    return out


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    threads = os.cpu_count() or 1
    # size each reference step so that warmup + steps take ~2 minutes
    budget = 120.0 / max(1, args.steps + args.warmup)
    rows = 64
    g = oracle.init(rows, N_COLS, 1, DENSITY / 2, DENSITY / 2)
    t0 = time.perf_counter()
    oracle.run(g, 1, threads=threads)
    per_row_step = max(time.perf_counter() - t0, 1e-6) / rows
    rows = int(min(M_ROWS, max(8, budget / (per_row_step * STEPS_PER_BENCH_STEP))))
    g = oracle.init(rows, N_COLS, 1, DENSITY / 2, DENSITY / 2)
    for _ in range(args.warmup):
        g, _, _ = oracle.run(g, STEPS_PER_BENCH_STEP, threads=threads)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g, _, _ = oracle.run(g, STEPS_PER_BENCH_STEP, threads=threads)
    dt = time.perf_counter() - t0
    value = rows * N_COLS * STEPS_PER_BENCH_STEP * args.steps / dt
    sample = ("each step: %d lattice steps of a %d x %d periodic band of the workload "
              "(density %.2f)" % (STEPS_PER_BENCH_STEP, rows, N_COLS, DENSITY))
    line = {
        "impl": "reference", "metric": "cell-updates/s", "value": value,
        "unit": "cell-updates/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt * 1e3 / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "M": M_ROWS, "N": N_COLS, "density": DENSITY,
                   "lattice_steps_per_step": STEPS_PER_BENCH_STEP, "impl": "cpu oracle"},
        "cpu_baseline": {"value": value, "unit": "cell-updates/s", "cores": threads,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "cell-updates/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(local)
    from paper_1804_07981_b300 import bml

    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream(device=dev)
    seed = 1 + rank
    M, N = args.M, args.N
    cells = M * N
    K, W = args.steps, args.warmup

    def barrier():
        dist_barrier(world)
        torch.cuda.synchronize()

    def max_over_ranks(x: float) -> float:
        return dist_max(x, world)

    # ---------------- device-resident run (value, roofline) ----------------
    sim = bml.Lattice(M, N, seed=seed, p_lr=DENSITY / 2, p_tb=DENSITY / 2, kernel=args.kernel,
                      block_k=args.block_k, stream=stream,
                      reserve_steps=(K + W) * STEPS_PER_BENCH_STEP)
    if args.band is not None:
        sim.set_tiling(args.block_k or 1, args.band, args.lane_words)
    kernel_id, block_k, band_rows = sim.config
    lane_words = sim.tiling[2] if kernel_id in (bml.BML_KERNEL_TBLOCK, bml.BML_KERNEL_FUSED) else 1
    for _ in range(W):
        sim.step(STEPS_PER_BENCH_STEP)
    sim.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(K):
        sim.step(STEPS_PER_BENCH_STEP)
    e1.record(stream)
    e1.synchronize()
    barrier()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms)
    lattice_steps = K * STEPS_PER_BENCH_STEP
    value = job_rate(world, cells * lattice_steps, ms_max / 1e3)
    # counts of the timed steps must be complete and plausible
    tot, _, _ = sim.moved_counts(W * STEPS_PER_BENCH_STEP, lattice_steps)
    assert (tot >= 0).all() and (tot <= cells).all()

    # dominant kernel: every launch in the timed region is the same kernel
    hbm_peak, peak_kind = _peaks()
    sm_mhz = (clk or {}).get("sm_mhz") or SM_MAX_MHZ
    if kernel_id in (bml.BML_KERNEL_TBLOCK, bml.BML_KERNEL_FUSED):
        depth = max(1, block_k)
        launches_per_step = STEPS_PER_BENCH_STEP // depth
        kname = ("fused_rows_kernel" if band_rows == 0 else
                 ("stream2_kernel<%d>" if lane_words == 2 else "stream_kernel<%d>") % depth)
    elif kernel_id == bml.BML_KERNEL_BITPLANE:
        depth, launches_per_step, kname = 1, 2 * STEPS_PER_BENCH_STEP, "plane_h/plane_v"
    else:
        depth, launches_per_step, kname = 1, 2 * STEPS_PER_BENCH_STEP, "byte_h/byte_v"
    launch_ms = ms / (K * launches_per_step)
    cell_steps_per_launch = cells * depth
    effective = BYTES_PER_CELL_STEP * cells * lattice_steps / (ms / 1e3) / 1e9
    traffic = TRAFFIC_PER_CELL.get((kname, band_rows))
    if depth >= 2:
        # bit logic with k steps per DRAM pass: bound by the integer ALU pipe
        ops = ALU_OPS_PER_CELL_STEP * cell_steps_per_launch
        achieved = ops / (launch_ms / 1e3) / 1e12
        peak = SMS * ALU_LANES_PER_SM_CLK * sm_mhz * 1e6 / 1e12
        roofline = {"bound": "alu", "kernel": kname, "achieved": achieved, "peak": peak,
                    "unit": "Tops/s", "frac": achieved / peak,
                    "traffic": traffic * cells if traffic else None,
                    "peak_kind": "derived: %d SMs x %d int32 lanes/clk x %.0f MHz sampled"
                                 % (SMS, ALU_LANES_PER_SM_CLK, sm_mhz),
                    "ops_per_cell_step": ALU_OPS_PER_CELL_STEP}
    else:
        bytes_per_launch = {"byte_h/byte_v": 2.0, "plane_h/plane_v": 0.375}.get(
            kname, BYTES_PER_CELL_STEP) * cells
        achieved = bytes_per_launch / (launch_ms / 1e3) / 1e9
        roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": hbm_peak,
                    "unit": "GB/s", "frac": achieved / hbm_peak,
                    "traffic": traffic * cells if traffic else None,
                    "peak_kind": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"}
    roofline.update({"launch_ms": launch_ms, "temporal_depth": depth,
                     "hbm_effective_GBps": effective,
                     "hbm_effective_frac": effective / hbm_peak,
                     "hbm_peak_GBps": hbm_peak})
    gpu_launches = K * launches_per_step

    # ---------------- end to end through the C ABI with host buffers -------
    e2e = None
    if not args.no_e2e:
        host_in = torch.empty((M, N), dtype=torch.uint8, pin_memory=True)
        host_out = torch.empty((M, N), dtype=torch.uint8, pin_memory=True)
        sim.synchronize()
        hin = host_in.numpy()  # the seeded lattice, as a user's host input
        bml.bml_read_lattice(sim.handle, M, N, out=hin)
        hout = host_out.numpy()
        # every step's counts are copied to page-locked host memory as the
        # step's result, without stalling the stream; the final lattice read
        # synchronises
        cnt_lr = torch.zeros(K * STEPS_PER_BENCH_STEP, dtype=torch.int64,
                             pin_memory=True).numpy()
        cnt_tb = torch.zeros(K * STEPS_PER_BENCH_STEP, dtype=torch.int64,
                             pin_memory=True).numpy()
        barrier()
        t0 = time.perf_counter()
        bml.bml_write_lattice(sim.handle, hin)  # H2D + pack, restarts the trajectory
        for s in range(K):
            bml.bml_step(sim.handle, STEPS_PER_BENCH_STEP)
            sl = slice(s * STEPS_PER_BENCH_STEP, (s + 1) * STEPS_PER_BENCH_STEP)
            bml.bml_moved_counts_async(sim.handle, s * STEPS_PER_BENCH_STEP,
                                       STEPS_PER_BENCH_STEP, cnt_lr[sl], cnt_tb[sl])
        bml.bml_read_lattice(sim.handle, M, N, out=hout)
        total = cnt_lr + cnt_tb
        dt = time.perf_counter() - t0
        want_tot, _, _ = bml.bml_moved_counts(sim.handle, 0, K * STEPS_PER_BENCH_STEP)
        assert np.array_equal(total, want_tot)
        dt = max_over_ranks(dt)
        e2e = {"value": job_rate(world, cells * lattice_steps, dt), "unit": "cell-updates/s",
               "h2d_bytes_per_step": cells / K,
               "d2h_bytes_per_step": cells / K + STEPS_PER_BENCH_STEP * 2 * 8,
               "seconds": dt}
    sim.close()

    ens = None
    if not args.no_ensemble:
        ens = _ensemble_bench(bml, torch, stream, args.ensemble_steps, seed_base=1 + 4096 * rank,
                              tiling=_ints(args.ensemble_tiling),
                              sm_mhz=(clk or {}).get("sm_mhz") or SM_MAX_MHZ)
        ens_max = max_over_ranks(ens["seconds"])
        ens["value"] = job_rate(world, ens["lattices"] * ens["steps"], ens_max)

    byte = None
    if not args.no_byte:
        byte = _byte_bench(bml, torch, stream, M, N, args.byte_steps, hbm_peak, seed=1 + rank)
        byte["value"] = job_rate(world, M * N * byte["steps"], max_over_ranks(byte["seconds"]))

    two = None
    if not args.no_two_phase:
        two = _two_phase_bench(bml, torch, stream, M, N, args.two_phase_steps, hbm_peak,
                               seed=1 + rank)
        two["value"] = job_rate(world, M * N * two["steps"], max_over_ranks(two["seconds"]))

    one = None
    if not args.no_one_pass:
        one = _one_pass_bench(bml, torch, stream, M, N, args.one_pass_steps, hbm_peak,
                              seed=1 + rank)
        one["value"] = job_rate(world, M * N * one["steps"], max_over_ranks(one["seconds"]))

    small = None
    if not args.no_configs and world == 1:
        small = _config_benches(bml, torch, stream)

    mlp = None
    if not args.no_mlp and world == 1:
        mlp = _mlp_bench(bml, torch, stream, hbm_peak, gemm_rows=args.mlp_gemm_rows)

    m2 = m3 = None
    if not args.no_model2:
        m2 = _model2_bench(bml, torch, stream, M, N, args.model2_steps,
                           (clk or {}).get("sm_mhz") or SM_MAX_MHZ, seed=1 + rank,
                           tiling=_ints(args.model2_tiling))
        m2_max = max_over_ranks(m2["seconds"])
        m2["value"] = job_rate(world, M * N * m2["steps"], m2_max)
        m3 = _model2_bench(bml, torch, stream, M, N, args.model2_steps,
                           (clk or {}).get("sm_mhz") or SM_MAX_MHZ, seed=1 + rank, model=3)
        m3["value"] = job_rate(world, M * N * m3["steps"], max_over_ranks(m3["seconds"]))

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        threads = os.cpu_count() or 1
        rate, desc, _ = _cpu_sample(args.cpu_seconds, threads)
        cpu = {"value": rate, "unit": "cell-updates/s", "cores": threads, "kind": "oracle",
               "sample": desc}
        if ens is not None:
            ens["cpu_oracle"] = _oracle_ensemble_sample(4.0, threads)
        if small is not None:
            small["4096x4096_rho0.20-0.50_seeds1-3_4096steps"]["oracle_1core"] = \
                _oracle_1core_4096(4.0)
        cpu["ladder"] = _cpu_ladder_sample(threads)

    if rank == 0:
        line = {
            "metric": "cell-updates/s", "value": value, "unit": "cell-updates/s",
            "n_gpus": world, "steps": K, "warmup": W, "ms_per_step": ms_max / K,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64 bitplanes" if kernel_id != bml.BML_KERNEL_BYTE else "u8",
            "data": "synthetic",
            "config": {"workload": workload_name(M, N), "M": M, "N": N, "density": DENSITY,
                       "seed": 1, "lattice_steps_per_step": STEPS_PER_BENCH_STEP,
                       "kernel": {0: "auto", 1: "byte", 2: "bitplane", 3: "fused",
                                  4: "tblock"}[kernel_id],
                       "temporal_depth": block_k, "band_rows": band_rows,
                       "lane_words": lane_words,
                       "l2": "inputs larger than L2 (2 x 256 MB bitplanes)",
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "ensemble": ens,
            "model2": m2, "model3": m3, "byte_kernel": byte, "two_phase": two, "one_pass": one,
            "configs": small,
            "mlp": mlp,
            "gpu_launches": gpu_launches, "clocks": clk,
        }
        # the headline figures of every sub-measurement again, last on the
        # line, where a reader that keeps only the end of the output sees them
        line["summary"] = _summary(line)
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def _summary(line):
    """Compact copy of the sub-measurements' headline numbers."""
    def pick(d, *keys):
        return {k: d[k] for k in keys if d is not None and k in d}

    out = {"value": line["value"], "roofline_frac": line["roofline"]["frac"],
           "roofline_kernel": line["roofline"].get("kernel")}
    if line.get("e2e"):
        out["e2e"] = line["e2e"]["value"]
    if line.get("cpu_baseline"):
        out["cpu_baseline"] = line["cpu_baseline"]["value"]
        if line["cpu_baseline"].get("ladder"):
            out["cpu_ladder"] = line["cpu_baseline"]["ladder"]["value_by_form"]
    ens = line.get("ensemble")
    if ens:
        out["ensemble"] = pick(ens, "value", "unit", "steps", "seconds", "temporal_depth",
                               "band_rows", "cell_updates_per_s")
        out["ensemble"]["roofline_frac"] = ens["roofline"]["frac"]
        if ens.get("cpu_oracle"):
            out["ensemble"]["cpu_oracle"] = ens["cpu_oracle"]["value"]
    for key in ("model2", "model3", "byte_kernel", "two_phase", "one_pass"):
        d = line.get(key)
        if d:
            out[key] = {"value": d["value"], "kernel": d.get("kernel"),
                        "roofline_frac": d["roofline"]["frac"]}
    mlp = line.get("mlp")
    if mlp:
        out["mlp"] = {"train_step_us": mlp["train_step_us"],
                      "forward_2624_us": mlp["forward_2624_us"],
                      "gemm_hbm_frac": mlp["gemm"]["roofline"]["frac"]}
    cfg = line.get("configs")
    if cfg:
        a = cfg["256x256_rho0.30_1024steps"]
        b = cfg["4096x4096_rho0.20-0.50_seeds1-3_4096steps"]
        out["configs"] = {"256x256_cell_updates_per_s": a["cell_updates_per_s"],
                          "4096x4096_bitplane_cell_updates_per_s":
                              b["bitplane_cell_updates_per_s"],
                          "4096x4096_byte_cell_updates_per_s": b["byte_cell_updates_per_s"]}
    return out


def _ints(spec):
    return tuple(int(x) for x in spec.split(",")) if spec else None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1250)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kernel", default="auto")
    ap.add_argument("--block-k", type=int, default=0)
    ap.add_argument("--band", type=int, default=None, help="band rows (with --kernel tblock)")
    ap.add_argument("--lane-words", type=int, default=1, help="1 or 2 (with --band)")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-steps", type=int, default=10000)
    ap.add_argument("--ensemble-tiling", default=None,
                    help="K,BAND: explicit ensemble depth and band (default: autotuned)")
    ap.add_argument("--no-model2", action="store_true")
    ap.add_argument("--model2-tiling", default=None,
                    help="K,BAND,LANE_WORDS: explicit Model II tiling (default: autotuned)")
    ap.add_argument("--no-byte", action="store_true")
    ap.add_argument("--byte-steps", type=int, default=16)
    ap.add_argument("--no-configs", action="store_true")
    ap.add_argument("--no-mlp", action="store_true")
    ap.add_argument("--mlp-gemm-rows", type=int, default=1 << 22,
                    help="rows of the GEMM-kernel measurement in the mlp entry")
    ap.add_argument("--no-one-pass", action="store_true")
    ap.add_argument("--no-two-phase", action="store_true")
    ap.add_argument("--two-phase-steps", type=int, default=64)
    ap.add_argument("--one-pass-steps", type=int, default=256)
    ap.add_argument("--model2-steps", type=int, default=1024)
    ap.add_argument("--M", type=int, default=M_ROWS)
    ap.add_argument("--N", type=int, default=N_COLS)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    args = ap.parse_args()
    if args.impl == "ours":
        args.warmup = max(3, args.warmup)  # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
