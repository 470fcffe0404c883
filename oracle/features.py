"""Surrogate inputs and labels from moved-count traces -- TEST INFRASTRUCTURE.

For a lattice with `cars` vehicles (conserved by the dynamics, Sec. 2) and a
moved-count trace m[t] (t = 0 .. T-1, entry t = step t+1):

- velocity at step t: m[t] / cars (cars per step per car; 0 if no car);
- features over steps first .. first+n-1 cut into `points` equal windows:
  [density = cars / (M N), M / 2048, N / 2048, mean velocity of each window];
- labels over the last `window` steps of a run of T steps: steady-state
  velocity = mean velocity over steps T-window .. T-1; jam = 1 if some step
  moved no car (an absorbing fixed point), else 0.
"""
from __future__ import annotations

import numpy as np


def velocity(total: np.ndarray, cars) -> np.ndarray:
    total = np.asarray(total, dtype=np.float64)
    cars = np.asarray(cars, dtype=np.float64)
    with np.errstate(invalid="ignore", divide="ignore"):
        v = total / cars[..., None]
    return np.where(cars[..., None] > 0, v, 0.0)


def features(total: np.ndarray, cars, M, N, first: int, n: int, points: int) -> np.ndarray:
    """total: (count, T) int moved counts.  Returns (count, 3 + points)."""
    assert n % points == 0
    v = velocity(total[:, first:first + n], cars)
    win = v.reshape(v.shape[0], points, n // points).mean(axis=2)
    M = np.asarray(M, dtype=np.float64)
    N = np.asarray(N, dtype=np.float64)
    dens = np.asarray(cars, dtype=np.float64) / (M * N)
    return np.concatenate([dens[:, None], (M / 2048.0)[:, None], (N / 2048.0)[:, None], win],
                          axis=1)


def labels(total: np.ndarray, cars, window: int):
    """Returns (steady-state velocity, jam) over the whole trace length."""
    T = total.shape[1]
    v = velocity(total[:, T - window:], cars).mean(axis=1)
    jam = np.any(np.asarray(total) == 0, axis=1).astype(np.float64)
    return v, jam
