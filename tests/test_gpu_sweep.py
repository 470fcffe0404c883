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


def test_network_scores_at_small_scale(lib):
    """The network's own predictions against the exact runs.  Near the
    transition whether a run jams is decided long after the 512-step trace
    the network reads, and the training lattices (M, N drawn independently)
    are rarely square like the sweep's, so its jam probability is far from
    exact there.  Stated bounds: at most 20% of the runs on the wrong side
    of p = 1/2 (the sweep's per-density jam fraction, which no allocator
    knows in advance, would misclassify 8.5%), fewer than the majority class
    would; its velocity error below that of the sweep's global mean
    velocity; and no run the allocator stopped at B0 jams later."""
    from paper_1804_07981_b300 import sweep
    res = sweep.run(sweep.SMALL)
    net = res["network"]
    ref = net["reference_predictors"]
    assert net["runs"] == len(sweep.SMALL["densities"]) * sweep.SMALL["seeds"]
    assert net["jam_p0.5"]["misclassified"] <= 0.20, net
    assert net["jam_p0.5"]["misclassified"] < ref["jam_misclassified_majority"], net
    assert net["v_mae"] < ref["v_mae_global_mean"], net
    assert sum(b["runs"] for b in net["calibration"]) == net["runs"]
    assert net["stopped_at_B0"]["runs"] > 0
    assert net["stopped_at_B0"]["jammed_later"] == 0
    assert net["stopped_at_B0"]["answer_v_mae"] <= 0.01
