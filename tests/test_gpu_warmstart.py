"""The learned warm start gains over the method without it.

A small instance of the whole pipeline on the GPU: 128 x 128 slices with 45
views, 192 generated (FBP, cold SPGL1) pairs, a 3-level U-Net trained by the
library's own kernels, then 16 fresh slices solved cold, from the FBP and
from the network's prediction, all to the same root tolerance.  The learned
start must be much closer to the solution than the starting points the
method has without the network (zero, as in the cold start, and the FBP
image under the same calibrated projection), must not cost more than 10%
extra SPGL1 iterations over the cold start, every slice must end at the root
(warm failures fall back to the cold solver), and the warm solutions must
match the cold ones in l1 norm to 1e-2 (both stop anywhere within the root
tolerance 1e-3 ||F b|| of sigma, which moves ||x||_1 along the Pareto
curve).  A network trained this briefly predicts the solution to ~35% (L2);
the iteration and wall-time gain of the full-size pipeline (4096 pairs at
512^2) is measured by `python -m paper_1009_1380_gb300.warmstart`.
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
    assert learned["iterations_mean"] <= 1.1 * cold["iterations_mean"]
    assert learned["iterations_mean"] < fbp["iterations_mean"]
    assert learned["l1_rel_diff_vs_cold_mean"] < 1e-2
