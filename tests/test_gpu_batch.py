"""Batched operators (clones + CUDA graph) and the work-item autotuner."""
import numpy as np
import pytest

from oracle import nufft
from paper_1009_1380_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def test_batch_uneven_views_equals_single_calls(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n = 128
    views = [64, 128, 32, 128, 64, 96, 32]
    base = {m: cpct.Plan(n, n, m) for m in set(views)}
    plans = [cpct.clone(base[m]) for m in views]
    g = torch.Generator(device="cuda").manual_seed(3)
    imgs = [torch.randn((n, n), device="cuda", generator=g) for _ in views]
    outs = [torch.empty((n, n), device="cuda") for _ in views]
    sinos = [torch.empty((m, n), device="cuda") for m in views]
    pair = cpct.Batch(plans, imgs, outs, mode=cpct.BATCH_PAIR, branches=3)
    fwd = cpct.Batch(plans, imgs, sinos, mode=cpct.BATCH_FWD, branches=4)
    for _ in range(2):
        pair.run()
        fwd.run()
    torch.cuda.synchronize()
    info = pair.info()
    assert info["slices"] == len(views) and info["samples"] == sum(m * n for m in views)
    for i, m in enumerate(views):
        y = base[m].fwd(imgs[i])
        z = base[m].adj(y)
        torch.cuda.synchronize()
        assert torch.equal(y, sinos[i]), f"slice {i} forward differs"
        assert torch.equal(z, outs[i]), f"slice {i} pair differs"
    for p in plans:
        p.sync()


def test_tuned_plan_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 256, 64
    p = cpct.Plan(n, n, m)
    fcap, acap = cpct.tune(p, reps=3)
    print("tuned caps", fcap, acap)
    # the automatic caps or one of the fixed candidates
    assert 256 <= fcap <= 4096 and fcap % 64 == 0 and 8 <= acap <= 128
    rng = np.random.default_rng(12)
    img = rng.standard_normal((n, n))
    w = rng.standard_normal((m, n))
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    y = p.fwd(torch.from_numpy(img.astype(np.float32)).cuda()).cpu().numpy()
    z = p.adj(torch.from_numpy(w.astype(np.float32)).cuda()).cpu().numpy()
    ry, rz = nufft.radon_grid(img, geo), nufft.radon_grid_adj(w, geo)
    assert np.linalg.norm(y - ry) / np.linalg.norm(ry) < 1e-5
    assert np.linalg.norm(z - rz) / np.linalg.norm(rz) < 1e-5
    # a tuned plan can be cloned; clones give the same results
    c = cpct.clone(p)
    assert torch.equal(c.fwd(torch.from_numpy(img.astype(np.float32)).cuda()),
                       p.fwd(torch.from_numpy(img.astype(np.float32)).cuda()))
    with pytest.raises(cpct.CpctError):
        cpct.tune(p)  # shared with a clone now
