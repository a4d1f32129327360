"""Host-side pieces of the learned warm start (torch CPU tensors, no GPU):
the starting-radius calibration and the per-slice scaling."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1009_1380_gb300 import warmstart as ws  # noqa: E402


def test_calibration_recovers_a_known_radius_rule():
    # predictions whose true radius is 2.5 ||soft(x_hat, 0.2 s)||_1 exactly:
    # the calibration picks theta = 0.2 (zero spread) and kappa = 2.5
    g = torch.Generator().manual_seed(0)
    x_hat = torch.randn(12, 16, 16, generator=g) * torch.linspace(0.5, 2.0, 12)[:, None, None]
    s = x_hat.flatten(1).std(dim=1)
    soft = (x_hat.abs().flatten(1) - 0.2 * s[:, None]).clamp_min(0.0).sum(dim=1).double().numpy()
    cal = ws.calibrate(x_hat, 2.5 * soft)
    assert cal["theta"] == 0.2
    assert abs(cal["kappa"] - 2.5) < 1e-9
    assert cal["spread"] < 1e-9


def test_soft_l1_limits():
    x = torch.tensor([[[3.0, -4.0], [0.0, 1.0]]])
    assert ws._soft_l1(x, 0.0)[0] == 8.0
    # a threshold above every magnitude leaves nothing
    assert ws._soft_l1(x, 100.0)[0] == 0.0


def test_scales_are_per_slice_standard_deviations():
    x = torch.stack([torch.zeros(4, 4), torch.ones(4, 4) * torch.arange(4.0)])
    s = ws.scales(x)
    assert s[0].item() == pytest.approx(1e-12)  # clamped away from zero
    assert s[1].item() == pytest.approx(float(np.std(np.repeat(np.arange(4.0), 4), ddof=1)))
