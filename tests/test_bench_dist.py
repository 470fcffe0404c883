"""Multi-rank logic of bench.py on CPU (gloo, world size 2): barrier, max of
the per-rank times, whole-job rate of weak-scaled replicas, and the
reference arm doing no work on ranks other than 0."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.dist_barrier(world)
        t = bench.dist_max(1.5 + rank, world, device="cpu")
        rate = bench.job_rate(world, 100.0, t)

        class A:
            steps, warmup, gpus = 2, 0, world
        ref = bench.run_reference(A()) if rank == 1 else None
        q.put((rank, t, rate, ref))
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate, ref in res:
        assert t == 2.5                     # max over ranks
        assert rate == pytest.approx(2 * 100.0 / 2.5)
    assert res[1][3] == 0                   # rank 1: reference arm returns without work


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.dist_max(3.0, 1) == 3.0
    assert bench.job_rate(1, 10.0, 2.0) == 5.0


def test_summary_repeats_every_sub_measurement():
    """The line's trailing summary carries the headline number of each
    sub-measurement (a reader keeping only the end of the line sees them)."""
    sys.path.insert(0, ROOT)
    import bench
    rf = {"frac": 0.5}
    line = {"value": 1.0, "roofline": {"frac": 0.6, "kernel": "k"}, "e2e": {"value": 0.9},
            "cpu_baseline": {"value": 1e9},
            "ensemble": {"value": 3.0, "unit": "lattice-steps/s", "steps": 10000,
                         "roofline": rf, "cpu_oracle": {"value": 7.0}},
            "model2": {"value": 2.0, "kernel": "m", "roofline": rf},
            "byte_kernel": {"value": 4.0, "roofline": rf}, "two_phase": None,
            "one_pass": {"value": 5.0, "roofline": rf},
            "mlp": {"train_step_us": 170.0, "forward_2624_us": 60.0,
                    "gemm": {"roofline": {"frac": 0.8}}},
            "configs": {"256x256_rho0.30_1024steps": {"cell_updates_per_s": 1e11},
                        "4096x4096_rho0.20-0.50_seeds1-3_4096steps": {
                            "bitplane_cell_updates_per_s": 7e12,
                            "byte_cell_updates_per_s": 7e11}}}
    s = bench._summary(line)
    assert s["ensemble"]["value"] == 3.0 and s["ensemble"]["cpu_oracle"] == 7.0
    assert s["model2"]["value"] == 2.0 and s["one_pass"]["roofline_frac"] == 0.5
    assert "two_phase" not in s and s["mlp"]["gemm_hbm_frac"] == 0.8
    assert s["configs"]["4096x4096_bitplane_cell_updates_per_s"] == 7e12
