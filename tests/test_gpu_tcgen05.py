"""The tensor-core (tcgen05 / tensor memory) MMA sequence against a plain
matrix product of the same bfloat16 values (FP32 accumulation)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n,k", [(64, 32), (64, 128), (32, 64), (128, 96)])
def test_tc_gemm_matches_numpy(n, k):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build, cpct
    build.build()
    g = torch.Generator().manual_seed(n * 1000 + k)
    a = torch.randn((128, k), generator=g).to(torch.bfloat16)
    b = torch.randn((n, k), generator=g).to(torch.bfloat16)
    d = cpct.debug_tc_gemm(a.cuda(), b.cuda()).cpu().numpy().astype(np.float64)
    ref = a.double().numpy() @ b.double().numpy().T
    err = np.abs(d - ref).max() / np.abs(ref).max()
    print(f"n={n} k={k}: max rel err {err:.2e}")
    assert err < 1e-5
