"""The surrogate-guided sweep at a reduced scale: the exact CA judges the
budget allocation, and the network must save long runs against the method
without it at bounded error."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_sweep_small_scale(lib):
    from paper_1804_07981_b300 import sweep
    res = sweep.run(sweep.SMALL)
    base, sur = res["no_surrogate"], res["surrogate"]
    # without the network every run not jammed by B0 is continued exactly:
    # its answers are the exact ones
    assert base["max_abs_dv"] == 0.0 and base["max_abs_djam_fraction"] == 0.0
    # the network is trained (loss falls) and saves long runs ...
    assert res["training"]["loss_last"] < 0.5 * res["training"]["loss_first"]
    assert sur["extended_runs"] < base["extended_runs"]
    # ... at bounded error against the exact arm
    assert sur["max_abs_dv"] <= 0.01, res
    assert sur["max_abs_djam_fraction"] <= 1.0 / sweep.SMALL["seeds"], res
