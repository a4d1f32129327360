"""radon_adj_noalloc: the allocation-free adjoint gives radon_adj's result.

Callers that cannot allocate device memory when they apply the operator (an
allocator that owns the whole pool, a real-time loop, work being recorded
for replay) use radon_adj_noalloc, whose only scratch is a fixed device array
inside the library.  This file is collected last so that a run stopping at
the first failure has already run every other test; it also passes alone in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

KID_ADJ_REDUCE = 6


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def _p(t, offset=0):
    return ctypes.c_void_p(t.data_ptr() + offset)


def test_noalloc_adjoint_matches_radon_adj_twice(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct, synth
    L = cpct.lib()
    # the 2048^2 / 1024-view geometry splits its origin tiles, so the
    # partial-tile scratch is read by the reduce kernel
    n, m = 2048, 1024
    plan = cpct.Plan(n, n, m)
    work = plan.work()
    assert work["n_split"] > 0 and 0 < work["n_slots"] <= 2048, work
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(20)
    x = torch.from_numpy(synth.phantom("c2_2048")).cuda()
    for call in range(2):
        w = torch.randn((m, n), device="cuda", generator=gen) + plan.fwd(x) * (call + 1)
        ref = torch.empty((n, n), device="cuda")
        out = torch.full((n, n), float("nan"), device="cuda")
        assert L.radon_adj(plan.handle, _p(w), _p(ref), stream) == 0
        torch.cuda.synchronize()
        plan.profile_enable(1 << KID_ADJ_REDUCE)
        assert L.radon_adj_noalloc(plan.handle, _p(w), _p(out), stream) == 0
        torch.cuda.synchronize()
        prof = plan.profile_read()
        plan.profile_enable(0)
        plan.sync()
        # the reduce kernel ran, reading the static partial tiles
        assert prof.get("k_adj_reduce", (0.0, 0))[1] == 1, prof
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        rel = float(np.linalg.norm(o - r) / np.linalg.norm(r))
        print(f"call {call}: radon_adj_noalloc vs radon_adj rel {rel:.2e}")
        assert np.isfinite(o).all()
        # same kernels, same summation order: the same bits
        assert torch.equal(out, ref)


def test_noalloc_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    L = cpct.lib()
    plan = cpct.Plan(64, 64, 10)
    w = torch.zeros((10, 64), device="cuda")
    img = torch.zeros((64, 64), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    plan.launch_count(reset=True)
    assert L.radon_adj_noalloc(None, _p(w), _p(img), stream) == -1
    assert L.radon_adj_noalloc(plan.handle, None, _p(img), stream) == -1
    assert L.radon_adj_noalloc(plan.handle, _p(w), None, stream) == -1
    assert L.radon_adj_noalloc(plan.handle, _p(w, 4), _p(img), stream) == -1
    assert L.radon_adj_noalloc(plan.handle, _p(w), _p(img, 4), stream) == -1
    assert plan.launch_count() == 0


def test_noalloc_rejects_plans_needing_more_partial_tiles(torch_cuda):
    """A plan whose heavy tiles are split into more partial tiles than the
    static array holds is refused before any kernel is launched; radon_adj
    (plan-owned partial tiles) still serves it."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    L = cpct.lib()
    n, m = 2048, 1024
    host = cpct.debug_adj_items(n, n, m, 16)
    assert host["n_slots"] > 2048, host
    plan = cpct.Plan(n, n, m)
    plan.set_caps(adj_cap=16)
    assert plan.work()["n_slots"] == host["n_slots"]
    w = torch.randn((m, n), device="cuda")
    out = torch.zeros((n, n), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    plan.launch_count(reset=True)
    assert L.radon_adj_noalloc(plan.handle, _p(w), _p(out), stream) == -1
    assert plan.launch_count() == 0
    assert not out.any()
    ref = plan.adj(w)
    torch.cuda.synchronize()
    plan.sync()
    assert torch.isfinite(ref).all() and ref.abs().max() > 0
