"""Host-side pieces of the learned warm start (no GPU): the starting-radius
calibration from a table of soft-thresholded l1 norms."""
import numpy as np

from paper_1009_1380_gb300 import warmstart as ws


def _soft(x, thresh):
    return np.maximum(np.abs(x) - thresh, 0.0).sum()


def test_calibration_recovers_a_known_radius_rule():
    # slices whose true radius is 2.5 ||soft(x_hat, 0.2 s)||_1 exactly: the
    # calibration picks theta = 0.2 (zero spread) and kappa = 2.5
    rng = np.random.default_rng(0)
    x_hat = rng.standard_normal((12, 16, 16)) * np.linspace(0.5, 2.0, 12)[:, None, None]
    s = x_hat.reshape(12, -1).std(axis=1, ddof=1)
    table = [[_soft(x_hat[i], th * s[i]) for i in range(12)] for th in ws.THETAS]
    tau_star = 2.5 * np.array(table[ws.THETAS.index(0.2)])
    cal = ws.calibrate_table(table, tau_star)
    assert cal["theta"] == 0.2
    assert abs(cal["kappa"] - 2.5) < 1e-9
    assert cal["spread"] < 1e-9


def test_calibration_prefers_the_least_spread():
    # a radius rule with a constant factor at theta = 0 but a varying one at
    # every other theta: theta = 0 wins
    table = [np.array([1.0, 2.0, 4.0])] + [np.array([1.0, 1.0, 1.0])] * (len(ws.THETAS) - 1)
    cal = ws.calibrate_table(table, 3.0 * table[0])
    assert cal["theta"] == ws.THETAS[0] and abs(cal["kappa"] - 3.0) < 1e-12
