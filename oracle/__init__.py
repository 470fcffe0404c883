"""CPU oracle for the BML traffic cellular automaton -- TEST INFRASTRUCTURE.

Only the tests, the package smoke check and the benchmark's CPU-baseline /
reference leg may import this package.  The product path (the CUDA library
and its Python binding) never imports, links or executes anything here, and
this package imports nothing from the product.

`bml_oracle.c` is the plain serial byte-per-cell simulator (Marzolla 2018,
Sec. 2 rules, Sec. 3 layout and double buffer, Sec. 4 row-parallel loop for
the threaded mode), with Models II and III (Sec. 2) in `run_model`.  `mlp.py` is the fp64 reference for the surrogate
network.  `features.py` holds the trace features and labels the surrogate
is trained on.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bml_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

EMPTY, LR, TB = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile bml_oracle.c into liboracle.so (plain -O2, OpenMP for the
    threaded mode).  Returns the library path."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".tmp.%d" % os.getpid()
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                    _SRC, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            vp = ctypes.c_void_p
            lib.oracle_splitmix64.argtypes = [u64, u64]
            lib.oracle_splitmix64.restype = u64
            lib.oracle_threshold.argtypes = [dbl]
            lib.oracle_threshold.restype = u64
            lib.oracle_init.argtypes = [vp, i64, i64, u64, dbl, dbl]
            lib.oracle_init.restype = ctypes.c_int
            lib.oracle_init_window.argtypes = [vp, i64, i64, i64, i64, i64, i64, u64, dbl,
                                               dbl]
            lib.oracle_init_window.restype = ctypes.c_int
            lib.oracle_run.argtypes = [vp, i64, i64, i64, vp, vp, ctypes.c_int]
            lib.oracle_run.restype = ctypes.c_int
            lib.oracle_phase.argtypes = [vp, vp, i64, i64, ctypes.c_int]
            lib.oracle_phase.restype = i64
            lib.oracle_run_batch.argtypes = [vp, i64, i64, i64, i64, vp, vp]
            lib.oracle_run_batch.restype = ctypes.c_int
            lib.oracle_run_model.argtypes = [vp, i64, i64, i64, ctypes.c_int, u64, i64,
                                             vp, vp, ctypes.c_int]
            lib.oracle_run_model.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def splitmix64(seed: int, n: int) -> int:
    """n-th SplitMix64 output (n >= 1) from state `seed`."""
    return int(_load().oracle_splitmix64(seed, n))


def threshold(p: float) -> int:
    """floor(p * 2^64) clamped to 2^64 - 1."""
    return int(_load().oracle_threshold(float(p)))


def init(M: int, N: int, seed: int, p_lr: float, p_tb: float) -> np.ndarray:
    """Seeded random lattice, uint8 (M, N) with 0 EMPTY / 1 LR / 2 TB."""
    g = np.empty((M, N), dtype=np.uint8)
    rc = _load().oracle_init(_ptr(g), M, N, seed, p_lr, p_tb)
    if rc != 0:
        raise ValueError("oracle_init rejected its arguments")
    return g


def init_window(i0: int, j0: int, R: int, C: int, M: int, N: int, seed: int, p_lr: float,
                p_tb: float) -> np.ndarray:
    """Rows i0..i0+R-1 and columns j0..j0+C-1 (mod M, N) of the seeded
    placement of an M x N lattice, uint8 (R, C)."""
    w = np.empty((R, C), dtype=np.uint8)
    rc = _load().oracle_init_window(_ptr(w), R, C, i0, j0, M, N, seed, p_lr, p_tb)
    if rc != 0:
        raise ValueError("oracle_init_window rejected its arguments")
    return w


def run(g: np.ndarray, K: int, threads: int = 1):
    """Advance a copy of g by K steps.

    Returns (lattice after K steps, moved_lr[K], moved_tb[K]) as int64."""
    g = np.ascontiguousarray(g, dtype=np.uint8).copy()
    M, N = g.shape
    mlr = np.zeros(K, dtype=np.int64)
    mtb = np.zeros(K, dtype=np.int64)
    rc = _load().oracle_run(_ptr(g), M, N, K, _ptr(mlr), _ptr(mtb), threads)
    if rc != 0:
        raise RuntimeError("oracle_run failed (%d)" % rc)
    return g, mlr, mtb


def run_model(g: np.ndarray, K: int, model: int, tie_seed: int = 0, t0: int = 0,
              threads: int = 1):
    """Advance a copy of g by K steps of Model II (model=2) or Model III
    (model=3; a cell may then hold 3 = one LR and one TB vehicle); the first
    step has index t0 (for Model II it selects the tie-break bits).

    Returns (lattice after K steps, moved_lr[K], moved_tb[K]) as int64."""
    g = np.ascontiguousarray(g, dtype=np.uint8).copy()
    M, N = g.shape
    mlr = np.zeros(K, dtype=np.int64)
    mtb = np.zeros(K, dtype=np.int64)
    rc = _load().oracle_run_model(_ptr(g), M, N, K, model, tie_seed, t0, _ptr(mlr),
                                  _ptr(mtb), threads)
    if rc != 0:
        raise RuntimeError("oracle_run_model failed (%d)" % rc)
    return g, mlr, mtb


def phase(g: np.ndarray, which: int):
    """One phase (0 horizontal, 1 vertical).  Returns (new lattice, moved)."""
    g = np.ascontiguousarray(g, dtype=np.uint8)
    out = np.empty_like(g)
    M, N = g.shape
    moved = _load().oracle_phase(_ptr(g), _ptr(out), M, N, which)
    return out, int(moved)


def run_batch(gs: np.ndarray, K: int):
    """gs: uint8 (count, M, N).  Returns (lattices, moved_lr, moved_tb) with
    counts shaped (count, K)."""
    gs = np.ascontiguousarray(gs, dtype=np.uint8).copy()
    count, M, N = gs.shape
    mlr = np.zeros((count, K), dtype=np.int64)
    mtb = np.zeros((count, K), dtype=np.int64)
    rc = _load().oracle_run_batch(_ptr(gs), count, M, N, K, _ptr(mlr), _ptr(mtb))
    if rc != 0:
        raise RuntimeError("oracle_run_batch failed (%d)" % rc)
    return gs, mlr, mtb
