"""Host-side scoring of the surrogate network (sweep.network_scores) on
hand-made predictions."""
import numpy as np

from paper_1804_07981_b300 import sweep


def test_network_scores_counts_errors_and_bins():
    rho = np.array([0.25, 0.27, 0.31, 0.36, 0.41, 0.45])
    exact = (np.array([1.0, 1.0, 0.9, 0.0, 0.0, 0.0]), np.array([0, 0, 0, 1, 1, 1.0]))
    pred = {"v_hat": np.array([0.9, 1.0, 0.9, 0.2, 0.0, 0.1]),
            "p_jam": np.array([0.001, 0.2, 0.6, 0.95, 0.4, 0.999]),
            "v_B0": np.array([1.0, 1.0, 0.9, 0.5, 0.5, 0.5]),
            "stopped": np.array([True, False, False, False, False, False])}
    s = sweep.network_scores(pred, exact, rho, tau=0.01)
    assert s["runs"] == 6
    assert np.isclose(s["v_mae"], (0.1 + 0 + 0 + 0.2 + 0 + 0.1) / 6)
    # p >= 0.5: runs 2 (wrong: flows), 3, 5 (right); run 4 (jams, p = 0.4) missed
    assert s["jam_p0.5"] == {"threshold": 0.5, "misclassified": 2 / 6,
                             "false_negatives": 1, "false_positives": 1}
    # p >= tau: every run but the first; the two flowing ones are false positives
    assert s["jam_tau"]["false_negatives"] == 0 and s["jam_tau"]["false_positives"] == 2
    assert [b["runs"] for b in s["calibration"]] == [1, 0, 2, 1, 1, 1]
    assert s["calibration"][2]["jammed"] == 0.5
    bands = s["per_density_band"]
    assert [b["runs"] for b in bands] == [2, 1, 1, 2]
    st = s["stopped_at_B0"]
    assert st["runs"] == 1 and st["answer_v_mae"] == 0.0 and st["jammed_later"] == 0
    assert np.isclose(st["v_hat_mae"], 0.1)
    ref = s["reference_predictors"]
    # per density (each density has one run here) the fraction is 0 or 1
    assert ref["jam_misclassified_per_density_fraction"] == 0.0
    assert ref["jam_misclassified_majority"] == 0.5
    assert ref["v_mae_per_density_mean"] == 0.0
    assert np.isclose(ref["v_mae_global_mean"], np.abs(exact[0] - exact[0].mean()).mean())
