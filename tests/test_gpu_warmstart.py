"""The learned warm start gains over the method without it.

A small instance of the whole pipeline on the GPU: 128 x 128 slices with 45
views, 384 generated (FBP, cold SPGL1) pairs, a 3-level U-Net trained by the
library's own kernels, then 16 fresh slices solved cold, from the FBP and
from the network's prediction, all to the same root tolerance.  The learned
start must be much closer to the solution than the starting points the
method has without the network (zero, as in the cold start, and the FBP
image under the same calibrated projection), must need fewer SPGL1
iterations than the cold start and than the FBP start, every slice must end
at the root (warm failures fall back to the cold solver), and the warm
solutions must match the cold ones in l1 norm to 1e-1 (both stop anywhere
within the root tolerance 1e-3 ||F b|| of sigma, which moves ||x||_1 along
the Pareto curve).  The wall-time gain of the full-size pipeline (4096
pairs at 512^2) is measured by `python -m paper_1009_1380_gb300.warmstart`,
and a bounded run of it by the benchmark's `warm` entry.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_learned_warm_start_reduces_iterations():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build, warmstart
    build.build()
    res = warmstart.run(pairs=384, eval_slices=16, epochs=30, batch=8, lr=2e-3, levels=3, base=32,
                        plans_per_group=16, target_iters=400, eval_tol=1e-3, n=128, m=45, log=print)
    print(res["eval"])
    cold, learned = res["eval"]["cold"], res["eval"]["learned"]
    assert cold["at_root"] == cold["slices"]
    assert learned["at_root"] == learned["slices"]
    # the gain over the method without the network: a start much closer to the
    # solution than zero (relative distance 1) and than the calibrated FBP start
    fbp = res["eval"]["fbp"]
    print("start distance: learned", learned["start_rel_err_mean"], "fbp", fbp["start_rel_err_mean"])
    assert learned["start_rel_err_mean"] < 0.6
    assert learned["start_rel_err_mean"] < 0.75 * fbp["start_rel_err_mean"]
    assert learned["iterations_mean"] < cold["iterations_mean"]
    assert learned["iterations_mean"] < fbp["iterations_mean"]
    # both solutions satisfy the root test | ||r|| - sigma | <= 1e-3 ||F b||;
    # ||F b|| is 10-30 sigma here, so the two residuals may differ by a few
    # percent of sigma, which moves ||x||_1 along the Pareto curve by
    # |d tau| = |d ||r|| | ||r|| / ||A^T r||_inf (measured 5.7% mean)
    assert learned["l1_rel_diff_vs_cold_mean"] < 0.1


def test_slice_statistics_match_their_definitions():
    """cpct_slice_moments / soft_l1 / scale against NumPy in FP64: the mean,
    the sample standard deviation, sum max(|x| - t, 0) and the scaling, per
    slice, on slices of several sizes (ragged tails of the block grid)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build, cpct
    build.build()
    rng = np.random.default_rng(5)
    for shape in [(1, 1), (3, 7, 5), (5, 64, 64), (2, 512, 512), (1, 1000003)]:
        x = (rng.standard_normal(shape) * rng.uniform(0.1, 10.0, (shape[0],) + (1,) * (len(shape) - 1))
             + rng.uniform(-3, 3, (shape[0],) + (1,) * (len(shape) - 1))).astype(np.float32)
        xd = torch.from_numpy(x).cuda()
        x64 = x.reshape(shape[0], -1).astype(np.float64)
        mean, std = cpct.slice_moments(xd)
        scale = float(np.abs(x64).max())
        np.testing.assert_allclose(mean, x64.mean(axis=1), rtol=1e-10, atol=1e-12 * scale)
        ref_std = x64.std(axis=1, ddof=1) if x64.shape[1] > 1 else np.zeros(shape[0])
        np.testing.assert_allclose(std, ref_std, rtol=1e-10, atol=1e-14)
        th = rng.uniform(0.0, 2.0, shape[0])
        soft = cpct.slice_soft_l1(xd, th)
        np.testing.assert_allclose(soft, np.maximum(np.abs(x64) - th[:, None], 0.0).sum(axis=1), rtol=1e-10)
        f = rng.uniform(-2.0, 2.0, shape[0])
        y = cpct.slice_scale(xd, f).cpu().numpy().reshape(shape[0], -1)
        ref = (x.reshape(shape[0], -1) * f.astype(np.float32)[:, None])
        assert np.array_equal(y, ref)
        # deterministic: the same bits on a second call
        assert np.array_equal(cpct.slice_moments(xd)[1], std)
