"""Few-view / low-dose sweep (the paper's Conclusions: basis pursuit should
allow fewer views or a lower dose for a similar image quality): at every
point SPGL1's reconstruction of the phase-contrast image is closer to the
true image than the filtered back-projection of the same data, every solve
reaches the root, and the basis-pursuit result with a quarter of the views
is at least as close as the filtered back-projection with all of them.  On
absorption data of the same objects, with the fewest views, the analysis-l1
variant (l1 of the object's horizontal differences) is closer to the object
than the filtered back-projection."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_few_view_sweep():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build, sweep
    build.build()
    pts = sweep.run(n=128, views=(16, 32, 64), noises=(0.01,), count=2, max_iter=400, synth_iters=300, log=print)
    by_m = {p["views"]: p for p in pts}
    for p in pts:
        assert p["spgl1_at_root"] == p["slices"]
        assert p["spgl1_rel_err"] < p["fbp_rel_err"]
    assert by_m[16]["spgl1_rel_err"] <= by_m[64]["fbp_rel_err"]
    assert by_m[16]["analysis_l1_rel_err"] < by_m[16]["absorption_fbp_rel_err"]
