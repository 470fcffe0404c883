"""Pins of the surrogate feature / label oracle (CPU): hand-computed values
on tiny traces, and the rule-184 ring whose velocity is known exactly."""
import numpy as np

import oracle
from oracle import features as F

EMPTY, LR = 0, 1


def test_hand_example():
    total = np.array([[4, 4, 2, 2, 0, 0, 0, 0],
                      [3, 3, 3, 3, 3, 3, 3, 3]])
    cars = np.array([4, 6])
    M, N = np.array([2, 3]), np.array([8, 4])
    f = F.features(total, cars, M, N, first=0, n=8, points=4)
    np.testing.assert_allclose(f[0], [4 / 16, 2 / 2048, 8 / 2048, 1.0, 0.5, 0.0, 0.0])
    np.testing.assert_allclose(f[1], [6 / 12, 3 / 2048, 4 / 2048, 0.5, 0.5, 0.5, 0.5])
    v, jam = F.labels(total, cars, window=4)
    np.testing.assert_allclose(v, [0.0, 0.5])
    np.testing.assert_array_equal(jam, [1.0, 0.0])


def test_no_cars_gives_zero_velocity():
    total = np.zeros((1, 4), dtype=np.int64)
    v, jam = F.labels(total, np.array([0]), window=2)
    assert v[0] == 0.0 and jam[0] == 1.0


def test_rule184_ring_velocity():
    """A single row of LR cars is rule 184: at density n/N <= 1/2 every car
    moves every step after the transient, so the steady velocity is 1; above
    1/2 it is (N - n)/n."""
    for n, N in [(10, 50), (30, 50)]:
        g = np.zeros((1, N), dtype=np.uint8)
        g[0, np.random.Generator(np.random.PCG64(n)).permutation(N)[:n]] = LR
        _, lr, tb = oracle.run(g, 4 * N)
        v, jam = F.labels((lr + tb)[None, :], np.array([n]), window=N)
        assert abs(v[0] - min(1.0, (N - n) / n)) < 1e-12
        assert jam[0] == 0.0
