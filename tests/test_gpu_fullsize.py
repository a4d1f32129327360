"""Parity at the full sizes of the benchmark configurations (beyond the
2048^2 operator test in test_gpu_radon.py), in the launch configurations the
benchmark and the warm-start pipeline use:

* batched operators (256 x 1024^2 slices, views 64..512): sampled rays of a
  few slices of one graph launch against the FP64 gridding oracle;
* SPGL1 on one 1024^2 / 128-view slice with noise and stuck columns: the
  root condition and ||x||_1 of the device solution re-evaluated with the
  FP64 oracle operator and filter;
* the warm-start denoiser at its full shape (5 levels, 32 base channels) on
  one 512^2 image against the FP64 oracle with the device's operand rounding;
* the largest geometries a plan accepts (32768 views; 2048^2 with 4096
  detector bins): both operators against the FP64 oracle (measured 2.1e-7 ..
  3.1e-7).
"""
import numpy as np
import pytest

from oracle import nufft, ring, unet
from paper_1009_1380_gb300 import synth

pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1009_1380_gb300 import build
    build.build()
    return torch


def test_batched_operator_full_size_sampled(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n = 1024
    views = [64, 512, 128, 256]
    base = {m: cpct.Plan(n, n, m) for m in sorted(set(views))}
    plans = [base[m] for m in views]
    imgs = [synth.phantom("c3_batch1024", slice_index=i) for i in range(len(views))]
    ins = [torch.from_numpy(im).cuda() for im in imgs]
    outs = [torch.empty((m, n), device="cuda") for m in views]
    bt = cpct.Batch(plans, ins, outs, mode=cpct.BATCH_FWD)
    bt.run()
    torch.cuda.synchronize()
    for i, m in enumerate(views):
        geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
        rays = np.array([0, 1, m // 3, m // 2, m - 1])
        ref = nufft.radon_grid(imgs[i].astype(np.float64), geo, rays)
        e = _rel(outs[i].cpu().numpy().astype(np.float64)[rays], ref)
        print(f"slice {i} ({m} views): sampled rays rel {e:.2e}")
        assert e < 1e-5
    bt.close()


def test_batched_adjoint_full_size_against_oracle(torch_cuda):
    """The batched adjoint (one graph launch over slices with uneven view
    counts, 1024^2) element by element: every slice's sinogram is non-zero
    on a few rays (ray 0, ray M/2 and some others), gridded back by the FP64
    oracle and compared with the slice's device result."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n = 1024
    views = [64, 512, 128, 256]
    base = {m: cpct.Plan(n, n, m) for m in sorted(set(views))}
    plans = [base[m] for m in views]
    rng = np.random.default_rng(1024)
    ws, ray_sets = [], []
    for m in views:
        rays = np.unique(np.concatenate([[0, m // 2], rng.choice(m, 6, replace=False)]))
        w = np.zeros((m, n), dtype=np.float32)
        w[rays] = rng.standard_normal((len(rays), n)).astype(np.float32)
        ws.append(w)
        ray_sets.append(rays)
    ins = [torch.from_numpy(w).cuda() for w in ws]
    outs = [torch.empty((n, n), device="cuda") for _ in views]
    bt = cpct.Batch(plans, ins, outs, mode=cpct.BATCH_ADJ)
    bt.run()
    torch.cuda.synchronize()
    for i, m in enumerate(views):
        geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
        G = geo.grid
        rays = ray_sets[i]
        Pt = nufft.ray_idft_adj(ws[i][rays].astype(np.float64))
        ref = nufft.grid_crop_deapod(nufft.ifft2(nufft.grid_spread(Pt, geo, rays)) * (G * G), geo).real
        e = _rel(outs[i].cpu().numpy().astype(np.float64), ref)
        print(f"slice {i} ({m} views, {len(rays)} rays): batched adjoint rel {e:.2e}")
        assert e < 1e-5
    bt.close()


def test_adjoint_full_size_2048_against_oracle(torch_cuda):
    """The 2048^2 / 1024-view adjoint element by element: a sinogram that is
    non-zero on 256 rays (ray 0, ray M/2 and 254 others) is gridded back by
    the FP64 oracle (ray DFT, spread of those rays' samples, inverse 2D FFT,
    crop and deapodize) and by the device, in the benchmark's plan."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 2048, 1024
    rng = np.random.default_rng(2048)
    rays = np.unique(np.concatenate([[0, m // 2], rng.choice(m, 254, replace=False)]))
    w = np.zeros((m, n), dtype=np.float32)
    w[rays] = rng.standard_normal((len(rays), n)).astype(np.float32)
    p = cpct.Plan(n, n, m)
    z = p.adj(torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    p.sync()
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    G = geo.grid
    Pt = nufft.ray_idft_adj(w[rays].astype(np.float64))
    Yh = nufft.grid_spread(Pt, geo, rays)
    ref = nufft.grid_crop_deapod(nufft.ifft2(Yh) * (G * G), geo).real
    zd = z.cpu().numpy().astype(np.float64)
    e = _rel(zd, ref)
    emax = float(np.abs(zd - ref).max() / np.abs(ref).max())
    print(f"2048 adjoint vs oracle on {len(rays)} rays: rel L2 {e:.2e}, max {emax:.2e}")
    assert e < 1e-5


def test_spgl1_full_size_root_by_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    c = synth.CONFIGS["c4_spgl1_1024"]
    n, m = c["n"], c["n_views"]
    p = cpct.Plan(n, n, m)
    x_true = synth.phantom("c4_spgl1_1024", slice_index=0)
    y = p.fwd(torch.from_numpy(x_true).cuda()).cpu().numpy()
    b, std, _ = synth.corrupt_sinogram(y, synth.rng_for(c["index"], 0))
    b32 = b.astype(np.float32)
    sigma = std * np.sqrt(m * n - n + 4)
    x, info = cpct.spgl1(p, torch.from_numpy(b32).cuda(), sigma, opts=cpct.make_opts(max_iter=600))
    print(info)
    assert info["status"] == 1
    xd = x.cpu().numpy().astype(np.float64)
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    bf = ring.ring_filter(b32.astype(np.float64))
    r = ring.ring_filter(nufft.radon_grid(xd, geo)) - bf
    rn = float(np.linalg.norm(r))
    print("oracle ||F(Rx) - F b||", rn, "sigma", sigma, "device", info["rnorm"])
    # the device's root test (opt_tol 1e-4 of ||F b||) re-evaluated in FP64
    assert abs(rn - sigma) <= 2e-4 * np.linalg.norm(bf)
    assert abs(np.abs(xd).sum() - info["xnorm1"]) <= 1e-5 * info["xnorm1"]


def test_denoiser_full_shape_512(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct, warmstart
    levels, base, H = 5, 32, 512
    vec = warmstart.he_init(levels, base, seed=3)
    rng = np.random.default_rng(4)
    vec[-1 - 1:-1] = 0.0
    # a non-zero head so that the output depends on every layer
    specs = unet.layer_specs(levels, base)
    nhead = specs[-1][2]
    vec[-(nhead + 1):-1] = (0.1 * rng.standard_normal(nhead)).astype(np.float32)
    x = rng.standard_normal((1, H, H)).astype(np.float32)
    net = cpct.UNet(levels, base, 1, H, H)
    net.set_params(vec)
    out = net.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    params, o = {}, 0
    for name, co, ci, k in specs:
        nw = co * k * k * ci
        params[name + ".W"] = vec[o:o + nw].astype(np.float64).reshape(co, k, k, ci)
        params[name + ".b"] = vec[o + nw:o + nw + co].astype(np.float64)
        if k == 3:
            params[name + ".W"] = unet.bf16_round(params[name + ".W"])
        o += nw + co
    ref, _ = unet.forward(params, x.astype(np.float64), levels, base, q=unet.bf16_round)
    e = _rel(out - x, ref - x)
    print("512^2 5-level denoiser: correction rel", e)
    assert e < 1e-2


def test_complex_pair_full_size_2048(torch_cuda):
    """The complex pair at 2048^2 / 1024 views: radon_fwd_c on sampled rays
    (ray 0, M/2 and others, the Nyquist imaginary part included) and
    radon_adj_c of a complex sinogram non-zero on a few rays, element by
    element against the FP64 gridding oracle."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 2048, 1024
    img = synth.phantom("c2_2048")
    p = cpct.Plan(n, n, m)
    yc = p.fwd_c(torch.from_numpy(img).cuda())
    rng = np.random.default_rng(4096)
    rays = np.unique(np.concatenate([[0, m // 2], rng.choice(m, 6, replace=False)]))
    w = np.zeros((m, n), dtype=np.complex64)
    w[rays] = (rng.standard_normal((len(rays), n)) + 1j * rng.standard_normal((len(rays), n))).astype(np.complex64)
    z = p.adj_c(torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    p.sync()
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    G = geo.grid
    yc_ref = nufft.radon_grid_c(img.astype(np.float64), geo, rays)
    e_f = _rel(yc.cpu().numpy().astype(np.complex128)[rays], yc_ref)
    Pt = nufft.ray_idft_adj(w[rays].astype(np.complex128))
    z_ref = nufft.grid_crop_deapod(nufft.ifft2(nufft.grid_spread(Pt, geo, rays)) * (G * G), geo).real
    e_a = _rel(z.cpu().numpy().astype(np.float64), z_ref)
    print(f"2048 complex pair: fwd_c sampled rays rel {e_f:.2e}, adj_c on {len(rays)} rays rel {e_a:.2e}")
    assert e_f < 1e-5 and e_a < 1e-5


@pytest.mark.parametrize("n,ns,m", [(64, 64, 32768), (2048, 4096, 256)])
def test_largest_accepted_geometries(torch_cuda, n, ns, m):
    """The limits a plan accepts: the most views (32768, every 16-bit ray
    index of the bin lists in use) and the largest image with the widest
    detector (2048^2, 4096 bins: the 4096-point ray transforms).  Forward and
    adjoint against the FP64 oracle: every ray where the oracle is quick,
    else eight rays including the first and the last (the adjoint of a
    sinogram that is non-zero on those rays only)."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(n + ns + m)
    img = rng.standard_normal((n, n)).astype(np.float32)
    geo = nufft.GridGeometry(n, ns, nufft.default_angles(m))
    G = geo.grid
    rays = np.arange(m) if n <= 64 else np.array([0, 1, 2, 63, 64, 128, 200, m - 1])
    w = np.zeros((m, ns), dtype=np.float32)
    w[rays] = rng.standard_normal((len(rays), ns)).astype(np.float32)
    p = cpct.Plan(n, ns, m)
    y = p.fwd(torch.from_numpy(img).cuda())
    z = p.adj(torch.from_numpy(w).cuda())
    torch.cuda.synchronize()
    p.sync()
    y_ref = nufft.radon_grid(img.astype(np.float64), geo, rays)
    Pt = nufft.ray_idft_adj(w[rays].astype(np.float64))
    Yh = nufft.grid_spread(Pt, geo, rays)
    z_ref = nufft.grid_crop_deapod(nufft.ifft2(Yh) * (G * G), geo).real
    ef = _rel(y.cpu().numpy()[rays].astype(np.float64), y_ref)
    ea = _rel(z.cpu().numpy().astype(np.float64), z_ref)
    print(f"{n}^2, {ns} bins, {m} views: fwd {ef:.2e} on {len(rays)} rays, adj {ea:.2e}")
    assert ef < 1e-5 and ea < 1e-5
