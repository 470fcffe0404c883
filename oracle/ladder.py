"""The paper's CPU implementations (serial with ghost cells, OpenMP, SIMD,
OpenMP+SIMD; and a bit-packed OpenMP form) as timed baselines --
TEST / BASELINE INFRASTRUCTURE (cpu_ladder.c).

    python -m oracle.ladder --fig3 [--reps R] [--out FILE]

runs the paper's Fig. 3 protocol on this host (density 0.3, N x N with N in
1024, 2048, 4096, 1024 steps, mean of R runs per form and size; the serial
form with modulo indexing is the oracle itself) and prints one JSON object.
"""
from __future__ import annotations

import ctypes
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cpu_ladder.c")
_LIB = os.path.join(_HERE, "libcpu_ladder.so")
_lock = threading.Lock()
_lib = None

# form number -> name (the paper's names, Sec. 7; "bitpacked" is beyond it)
FORMS = {1: "serial+halo", 2: "openmp", 3: "simd", 4: "openmp+simd", 5: "bitpacked+openmp"}


def build(force: bool = False) -> str:
    """Compile cpu_ladder.c (-O3, OpenMP; the SIMD loops carry their own
    AVX-512 / AVX2 / baseline clones, chosen at run time)."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=gnu11", "-Wno-psabi",
                    _SRC, "-o", tmp], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64 = ctypes.c_int64
            lib.ladder_run.argtypes = [ctypes.c_int, ctypes.c_void_p, i64, i64, i64,
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
            lib.ladder_run.restype = ctypes.c_int
            _lib = lib
    return _lib


def run(form: int, g: np.ndarray, K: int, threads: int = 1):
    """Advance a copy of g by K steps with the given form; returns (lattice,
    seconds of the K steps alone)."""
    g = np.ascontiguousarray(g, dtype=np.uint8).copy()
    M, N = g.shape
    secs = ctypes.c_double()
    rc = _load().ladder_run(form, g.ctypes.data_as(ctypes.c_void_p), M, N, K, threads,
                            ctypes.byref(secs))
    if rc != 0:
        raise RuntimeError("ladder_run failed (%d)" % rc)
    return g, secs.value


def fig3(sizes=(1024, 2048, 4096), steps=1024, reps=5, threads=None, max_run_s=30.0,
         oracle_max_n=2048):
    """The Fig. 3 protocol: density 0.3 (p_lr = p_tb = 0.15, seeded
    placement, seed 1), N x N, `steps` steps, mean of `reps` runs per form
    and size.  A form whose first run takes longer than max_run_s is not
    repeated at that size (its entry says how many runs it has).  The
    oracle (one core, several minutes per 4096^2 run) runs up to
    oracle_max_n; above, its entry is its rate at the largest size run,
    scaled to the cells (marked "extrapolated"), and the forms there are
    checked against each other (the first form's lattice) instead."""
    import oracle
    threads = threads or os.cpu_count() or 1
    out = {"density": 0.3, "steps": steps, "threads": threads, "seconds": {}}
    for N in sizes:
        g0 = oracle.init(N, N, 1, 0.15, 0.15)
        want = None
        row = {}
        for form in [0] + sorted(FORMS):
            times = []
            if form == 0 and N > oracle_max_n:
                prev = out["seconds"].get(str(max(n for n in sizes if n <= oracle_max_n)))
                if prev:
                    rate = prev["serial (oracle)"]["cell_updates_per_s"]
                    row["serial (oracle)"] = {"mean_s": N * N * steps / rate, "runs": 0,
                                              "cell_updates_per_s": rate,
                                              "extrapolated": True}
                continue
            for r in range(reps):
                if form == 0:  # the oracle: serial, modulo indexing (Sec. 3)
                    t0 = time.perf_counter()
                    got, _, _ = oracle.run(g0, steps, threads=1)
                    times.append(time.perf_counter() - t0)
                else:
                    got, dt = run(form, g0, steps, threads)
                    times.append(dt)
                if want is None:
                    want = got
                elif not np.array_equal(got, want):
                    raise AssertionError("form %d disagrees with the oracle at N=%d" % (form, N))
                if times[0] > max_run_s:
                    break
            name = "serial (oracle)" if form == 0 else FORMS[form]
            row[name] = {"mean_s": float(np.mean(times)), "runs": len(times),
                         "cell_updates_per_s": N * N * steps / float(np.mean(times))}
        out["seconds"][str(N)] = row
    return out


if __name__ == "__main__":
    reps = 5
    if "--reps" in sys.argv:
        reps = int(sys.argv[sys.argv.index("--reps") + 1])
    if "--fig3" in sys.argv:
        res = fig3(reps=reps)
        txt = json.dumps(res)
        if "--out" in sys.argv:
            with open(sys.argv[sys.argv.index("--out") + 1], "w") as fh:
                fh.write(txt + "\n")
        print(txt)
