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

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def test_noalloc_adjoint_matches_radon_adj_twice(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct, synth
    L = cpct.lib()
    # the 2048^2 / 1024-view geometry splits its origin tiles, so the
    # partial-tile scratch is exercised
    n, m = 2048, 1024
    plan = cpct.Plan(n, n, m)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    gen = torch.Generator(device="cuda").manual_seed(20)
    x = torch.from_numpy(synth.phantom("c2_2048")).cuda()
    for call in range(2):
        w = torch.randn((m, n), device="cuda", generator=gen) + plan.fwd(x) * (call + 1)
        ref = torch.empty((n, n), device="cuda")
        out = torch.full((n, n), float("nan"), device="cuda")
        assert L.radon_adj(plan.handle, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(ref.data_ptr()), stream) == 0
        assert L.radon_adj_noalloc(plan.handle, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                   stream) == 0
        torch.cuda.synchronize()
        plan.sync()
        r, o = ref.double().cpu().numpy(), out.double().cpu().numpy()
        rel = float(np.linalg.norm(o - r) / np.linalg.norm(r))
        print(f"call {call}: radon_adj_noalloc vs radon_adj rel {rel:.2e}")
        assert np.isfinite(o).all()
        assert rel < TOL


def test_noalloc_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    L = cpct.lib()
    plan = cpct.Plan(64, 64, 10)
    w = torch.zeros((10, 64), device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.radon_adj_noalloc(None, ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(w.data_ptr()), stream) == -1
    assert L.radon_adj_noalloc(plan.handle, None, ctypes.c_void_p(w.data_ptr()), stream) == -1
