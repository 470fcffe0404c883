"""The paper's CPU implementations (oracle/cpu_ladder.c: serial with ghost
cells, OpenMP, SIMD, OpenMP+SIMD, bit-packed OpenMP) reach the oracle's
lattice bit for bit (the Sec. 2 rules, wrap-around, H then V)."""
import numpy as np
import pytest

import oracle
from oracle import ladder
from paper_1804_07981_b300.inputs import random_lattice

SHAPES = [(1, 1), (1, 2), (2, 1), (3, 5), (17, 31), (64, 64), (65, 129), (7, 33), (40, 200),
          (100, 1000), (9, 64 * 3 + 1), (33, 2048)]


@pytest.mark.parametrize("form", sorted(ladder.FORMS))
@pytest.mark.parametrize("M,N", SHAPES)
def test_form_matches_oracle(form, M, N):
    for seed, rho in [(1, 0.3), (2, 0.6)]:
        g0 = random_lattice(M, N, seed * 1000 + M * 7 + N, rho / 2, rho / 2)
        want, _, _ = oracle.run(g0, 23)
        got, secs = ladder.run(form, g0, 23, threads=4)
        np.testing.assert_array_equal(got, want, err_msg=str((ladder.FORMS[form], seed)))
        assert secs >= 0.0


def test_forms_reject_bad_input():
    g = np.zeros((4, 4), dtype=np.uint8)
    g[0, 0] = 3
    with pytest.raises(RuntimeError):
        ladder.run(1, g, 1)
    with pytest.raises(RuntimeError):
        ladder.run(9, np.zeros((4, 4), dtype=np.uint8), 1)


def test_fig3_protocol_small():
    """The Fig. 3 driver on a small size: every form agrees with the oracle
    and reports a time."""
    res = ladder.fig3(sizes=(128,), steps=16, reps=2, threads=2)
    row = res["seconds"]["128"]
    assert set(row) == {"serial (oracle)"} | set(ladder.FORMS.values())
    assert all(v["runs"] == 2 and v["mean_s"] > 0 for v in row.values())
