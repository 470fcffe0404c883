"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module holds none of the automaton's arithmetic: it only draws lattices
and parameters.  The CUDA path's own seeded placement (a SplitMix64 hash per
cell) and the oracle's are separate implementations of one published
generator; this module is for inputs that are handed to both sides.
"""
from __future__ import annotations

import numpy as np

EMPTY, LR, TB = 0, 1, 2


def random_lattice(M: int, N: int, seed: int, p_lr: float, p_tb: float) -> np.ndarray:
    """uint8 (M, N) lattice, each cell LR w.p. p_lr, TB w.p. p_tb, else EMPTY
    (numpy PCG64 stream, not the in-library placement)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.random((M, N))
    g = np.zeros((M, N), dtype=np.uint8)
    g[u < p_lr] = LR
    g[(u >= p_lr) & (u < p_lr + p_tb)] = TB
    return g


def all_lattices(M: int, N: int) -> np.ndarray:
    """Every one of the 3^(M*N) lattices of shape (M, N), as uint8
    (3^(M*N), M, N), enumerated by base-3 digits."""
    n = M * N
    count = 3 ** n
    idx = np.arange(count, dtype=np.int64)
    out = np.empty((count, n), dtype=np.uint8)
    for c in range(n):
        out[:, c] = (idx % 3).astype(np.uint8)
        idx //= 3
    return out.reshape(count, M, N)


def ensemble_params(count: int, seed: int = 1, lo: int = 64, hi: int = 2048,
                    rho_lo: float = 0.1, rho_hi: float = 0.6,
                    f_lo: float = 0.3, f_hi: float = 0.7):
    """Per-lattice parameters of a batched ensemble: M, N uniform on
    {lo..hi}, density rho uniform on [rho_lo, rho_hi], LR fraction f uniform
    on [f_lo, f_hi]; p_lr = rho*f, p_tb = rho*(1-f); seed of lattice l is
    l + 1.  Returns a dict of numpy arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = rng.integers(lo, hi + 1, size=count, dtype=np.int64)
    N = rng.integers(lo, hi + 1, size=count, dtype=np.int64)
    rho = rng.uniform(rho_lo, rho_hi, size=count)
    f = rng.uniform(f_lo, f_hi, size=count)
    seeds = np.arange(1, count + 1, dtype=np.uint64)
    return {"M": M, "N": N, "rho": rho, "f": f,
            "p_lr": rho * f, "p_tb": rho * (1.0 - f), "seed": seeds}


def parse_golden(path: str):
    """Read a worked-example fixture: returns (shape, [(label, moved,
    uint8 lattice)]); moved is the count of a "moved n" state, the pair
    (LR, TB) of an "lr a tb b" state, else None.  '+' marks a cell holding
    one vehicle of each kind (byte 3)."""
    sym = {".": EMPTY, ">": LR, "v": TB, "+": LR | TB}
    shape = None
    blocks = []
    cur = None
    with open(path) as fh:
        for raw in fh:
            line = raw.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            if parts[0] == "shape":
                shape = (int(parts[1]), int(parts[2]))
            elif parts[0] == "state":
                if len(parts) >= 4 and parts[2] == "moved":
                    moved = int(parts[3])
                elif len(parts) >= 6 and parts[2] == "lr" and parts[4] == "tb":
                    moved = (int(parts[3]), int(parts[5]))
                else:
                    moved = None
                cur = [parts[1], moved, []]
                blocks.append(cur)
            else:
                cur[2].append([sym[ch] for ch in line])
    return shape, [(b[0], b[1], np.array(b[2], dtype=np.uint8)) for b in blocks]


def mlp_init_params(in_dim: int, seed: int, hidden: int = 128, n_hidden: int = 3,
                    n_out: int = 2) -> np.ndarray:
    """Initial surrogate-network parameters, flat float64 in the order W1, b1,
    W2, b2, ..., each W row-major [out][in]: He-uniform weights
    (bound sqrt(6 / fan_in)), zero biases, from numpy PCG64(seed)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dims = [in_dim] + [hidden] * n_hidden + [n_out]
    parts = []
    for l in range(len(dims) - 1):
        bound = np.sqrt(6.0 / dims[l])
        parts.append(rng.uniform(-bound, bound, size=(dims[l + 1], dims[l])).ravel())
        parts.append(np.zeros(dims[l + 1]))
    return np.concatenate(parts)
