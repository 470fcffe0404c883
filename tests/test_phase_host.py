"""Host-side parts of the phase-diagram module (no GPU): the PPM writer and
the binomial interval."""
import numpy as np
import pytest


def test_ppm_layout(tmp_path):
    from paper_1804_07981_b300.phase import COLOURS, write_ppm
    g = np.array([[0, 1, 2], [2, 1, 0]], dtype=np.uint8)
    p = tmp_path / "x.ppm"
    write_ppm(str(p), g, scale=2)
    data = p.read_bytes()
    head = b"P6\n6 4\n255\n"
    assert data.startswith(head)
    px = np.frombuffer(data[len(head):], dtype=np.uint8).reshape(4, 6, 3)
    for i in range(4):
        for j in range(6):
            np.testing.assert_array_equal(px[i, j], COLOURS[g[i // 2, j // 2]])
    with pytest.raises(ValueError):
        write_ppm(str(p), np.full((2, 2), 3, dtype=np.uint8))


def test_wilson_interval():
    from paper_1804_07981_b300.phase import wilson
    lo, hi = wilson(0, 10)
    assert lo == 0.0 and 0.25 < hi < 0.35          # 0/10: upper bound ~0.28
    lo, hi = wilson(5, 10)
    assert lo < 0.5 < hi and abs((lo + hi) / 2 - 0.5) < 1e-12
    lo, hi = wilson(10, 10)
    assert hi == 1.0 and 0.65 < lo < 0.75
