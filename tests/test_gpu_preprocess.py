"""GPU preprocessing front end (cpct_preprocess_pc) against the FP64 oracle:
background normalization of the near and far camera frames, their
difference (the phase-contrast image) and the regrouping into one sinogram
per detector row (section "Introduction", Fig. 1)."""
import numpy as np
import pytest

from oracle import preprocess as pp
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


def _dev(torch, a, dtype):
    if dtype == "raw":
        return torch.from_numpy(np.ascontiguousarray(a.astype(np.uint16).view(np.int16))).cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("m,rows,ns", [(90, 8, 512), (7, 3, 33), (1, 1, 1), (180, 2, 1000)])
def test_preprocess_matches_oracle(torch_cuda, m, rows, ns):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    r = synth.pc_radiographs(m, rows, ns, np.random.default_rng(m + rows + ns), n_spheres=4)
    fl_n, fl_f, dk = (r[k].astype(np.float32) for k in ("flat_near", "flat_far", "dark"))
    out = cpct.preprocess_pc(_dev(torch, r["near"], "raw"), _dev(torch, r["far"], "raw"), _dev(torch, fl_n, "f"),
                             _dev(torch, fl_f, "f"), _dev(torch, dk, "f"))
    torch.cuda.synchronize()
    ref = pp.phase_contrast_sinograms(r["near"], r["far"], fl_n.astype(np.float64), fl_f.astype(np.float64),
                                      dk.astype(np.float64))
    o = out.cpu().numpy().astype(np.float64)
    # each output is a difference of two normalized values of about 1
    # computed in FP32: absolute error a few ulp of 1
    err = float(np.abs(o - ref).max())
    print(f"m={m} rows={rows} ns={ns}: max abs err {err:.2e}, rel L2 "
          f"{np.linalg.norm(o - ref) / max(np.linalg.norm(ref), 1e-30):.2e}")
    assert err <= 1e-6
    # dead reference columns give exactly 0 on both sides
    dead = (fl_n - dk <= 0) & (fl_f - dk <= 0)
    assert np.all(o.transpose(1, 0, 2)[:, dead] == 0.0)


def test_preprocess_rejects_bad_arguments(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    import ctypes
    L = cpct.lib()
    z = torch.zeros(16, device="cuda")
    p = ctypes.c_void_p(z.data_ptr())
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L.cpct_preprocess_pc.argtypes = [ctypes.c_void_p] * 5 + [ctypes.c_int] * 3 + [ctypes.c_void_p] * 2
    assert L.cpct_preprocess_pc(None, p, p, p, p, 1, 1, 1, p, s) == -1
    assert L.cpct_preprocess_pc(p, p, p, p, p, 0, 1, 1, p, s) == -1
    assert L.cpct_preprocess_pc(p, p, p, p, p, 1, 1, 0, p, s) == -1
