"""GPU ring filter and SPGL1 against the FP64 oracle (through the C ABI).

Pins: the filter matches the oracle projector to FP32 rounding and is
idempotent on the device.  With a single fixed tau (the LASSO problem, whose
solution the mathematics fixes) the device solution matches the oracle's
element by element (relative L2 1e-3) once both duality gaps are small.  The
basis-pursuit denoising solve reaches the root on both sides, and the
solutions agree in misfit and in l1 norm to 1e-3 (the certificate pin).  Its
x is compared at 2e-2 (measured 0.8-1.0%): SPGL1 is an inexact Newton method
whose exit test is the root error alone, with the last LASSO problem's
duality gap still O(1), so x at exit is fixed by the method only to a few
percent -- the FP64 oracle itself ends 2.9% apart (relative L2) between
opt_tol 1e-6 and 1e-7 on this problem, and FP32 operators change
line-search branches.
"""
import numpy as np
import pytest

from oracle import nufft, ring, spgl1
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


def test_ring_filter_parity_and_projector(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    m, ns = 45, 64
    rng = np.random.default_rng(11)
    y = rng.standard_normal((m, ns))
    y[:, [3, 17, 40]] += np.array([0.7, -0.4, 1.1])
    p = cpct.Plan(64, ns, m)
    yd = torch.from_numpy(y.astype(np.float32)).cuda()
    f1 = cpct.ring_filter(p, yd)
    f2 = cpct.ring_filter(p, f1)
    torch.cuda.synchronize()
    ref = ring.ring_filter(y.astype(np.float32).astype(np.float64))
    e = _rel(f1.cpu().numpy(), ref)
    print("ring filter rel", e)
    assert e < 1e-6
    assert _rel(f2.cpu().numpy(), f1.cpu().numpy()) < 1e-6


def _problem(n, m, seed=5):
    rng = np.random.default_rng(seed)
    u, _ = synth.ellipse_phantom(n, 6, rng, axes_range=(200.0, 500.0))
    x_true = synth.laplacian5(u)
    geo = nufft.GridGeometry(n, n, nufft.default_angles(m))
    b, std, _ = synth.corrupt_sinogram(nufft.radon_grid(x_true, geo), rng)
    sigma = std * np.sqrt(m * n - n + 4)
    return geo, x_true, b, sigma


def _ops(n, m, geo):
    A = lambda v: ring.ring_filter(nufft.radon_grid(v.reshape(n, n), geo))
    At = lambda r: nufft.radon_grid_adj(ring.ring_filter(r.reshape(m, n)), geo)
    return A, At


def test_spgl1_matches_oracle(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 64, 64
    geo, x_true, b, sigma = _problem(n, m)
    b32 = b.astype(np.float32)
    bf = ring.ring_filter(b32.astype(np.float64))
    A, At = _ops(n, m, geo)
    tol = 1e-6
    xo, io = spgl1.spgl1(A, At, bf, sigma, opts=spgl1.Options(opt_tol=tol, max_iter=3000))
    p = cpct.Plan(n, n, m)
    xg, ig = cpct.spgl1(p, torch.from_numpy(b32).cuda(), sigma, opts=cpct.make_opts(opt_tol=tol, max_iter=3000))
    xg = xg.cpu().numpy().astype(np.float64)
    rg = np.linalg.norm(A(xg) - bf)
    print("oracle", io.status, io.iterations, io.n_newton, io.rnorm, io.xnorm1, io.rel_gap)
    print("gpu   ", ig)
    print("x rel", _rel(xg, xo), "l1 rel", abs(ig["xnorm1"] - io.xnorm1) / io.xnorm1, "r (oracle op)", rg, sigma)
    assert io.status == spgl1.EXIT_ROOT_FOUND
    assert ig["status"] == 1
    assert abs(ig["rnorm"] - sigma) <= 2 * tol * np.linalg.norm(bf)
    assert abs(rg - io.rnorm) <= 1e-3 * io.rnorm
    assert abs(ig["xnorm1"] - io.xnorm1) <= 1e-3 * io.xnorm1
    # measured 0.8-1.0%; the oracle's own x moves 2.9% between opt_tol 1e-6
    # and 1e-7, so 1e-2 is at the method's own determinacy
    assert _rel(xg, xo) < 2e-2


@pytest.mark.parametrize("n,m,tol", [(64, 64, 1e-3), (128, 90, 1e-3)])
def test_lasso_matches_oracle(torch_cuda, n, m, tol):
    """The LASSO problem min ||F(R x) - F b|| s.t. ||x||_1 <= tau at a fixed
    tau (half the l1 norm of the true image): device and FP64 oracle solutions
    agree element by element.  With a fixed tau the device keeps the residual
    as r - F(R (xt - x)), so its FP32 rounding is relative to the step, not to
    ||R xt||.  The solve runs until the objective stops resolving descent, at
    a duality gap near 1e-3 (the oracle's is 1e-5).  Measured x against the
    oracle: 7.8e-4 at 64^2, 2.1e-4 at 128^2."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    geo, x_true, b, sigma = _problem(n, m)
    b32 = b.astype(np.float32)
    bf = ring.ring_filter(b32.astype(np.float64))
    A, At = _ops(n, m, geo)
    tau = 0.5 * float(np.abs(x_true).sum())
    xo, io = spgl1.lasso(A, At, bf, tau, opts=spgl1.Options(opt_tol=1e-5, max_iter=20000))
    p = cpct.Plan(n, n, m)
    xg, ig = cpct.spgl1(p, torch.from_numpy(b32).cuda(), 0.0,
                        opts=cpct.make_opts(opt_tol=1e-5, max_iter=5000, lasso_tau=tau))
    xg = xg.cpu().numpy().astype(np.float64)
    e = _rel(xg, xo)
    print(f"n={n} m={m} tau={tau:.3f}: oracle status {io.status} it {io.iterations} gap {io.rel_gap:.2e}; "
          f"gpu {ig}; x rel {e:.2e}")
    assert io.status == spgl1.EXIT_OPTIMAL
    # 8: gap <= opt_tol; 4: no descent at the working precision
    assert ig["status"] in (8, 4)
    assert ig["rel_gap"] <= 5e-3
    assert abs(np.abs(xg).sum() - tau) <= 1e-5 * tau
    assert e <= tol


def test_spgl1_batched_equals_single(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 64, 48
    probs = [_problem(n, m, seed=s) for s in (21, 22, 23)]
    plans = [cpct.Plan(n, n, m) for _ in probs]
    bs = [torch.from_numpy(pb[2].astype(np.float32)).cuda() for pb in probs]
    sig = [pb[3] for pb in probs]
    xs, infos = cpct.spgl1_batched(plans, bs, sig)
    for i in range(3):
        x1, i1 = cpct.spgl1(plans[i], bs[i], sig[i])
        assert i1["status"] == infos[i]["status"] and i1["iterations"] == infos[i]["iterations"]
        assert torch.equal(x1, xs[i]), f"slice {i} differs between batched and single solves"


def test_spgl1_with_quadtree_bins(torch_cuda):
    """A solve whose plans use the quadtree bins (several bin sizes, their
    launches forked onto side streams inside the captured tick graph)
    reaches the root, and a batched solve equals the single ones bitwise."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 128, 90
    probs = [_problem(n, m, seed=s) for s in (31, 32)]
    plans = []
    for _ in probs:
        p = cpct.Plan(n, n, m)
        p.set_bins("fwd", "quadtree")
        p.set_bins("adj", "quadtree")
        assert sum(1 for c in p.bins()["adj"][2] if c > 0) > 1
        plans.append(p)
    bs = [torch.from_numpy(pb[2].astype(np.float32)).cuda() for pb in probs]
    sig = [pb[3] for pb in probs]
    xs, infos = cpct.spgl1_batched(plans, bs, sig)
    for i, (geo, x_true, b, sigma) in enumerate(probs):
        x1, i1 = cpct.spgl1(plans[i], bs[i], sig[i])
        print("quadtree solve", i1)
        assert i1["status"] == 1
        assert torch.equal(x1, xs[i])
        A, _ = _ops(n, m, geo)
        bf = ring.ring_filter(b.astype(np.float32).astype(np.float64))
        rg = np.linalg.norm(A(x1.cpu().numpy().astype(np.float64)) - bf)
        assert abs(rg - sigma) <= 2e-4 * np.linalg.norm(bf)


def test_spgl1_warm_start_and_basis_pursuit_flag(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 64, 64
    geo, x_true, b, sigma = _problem(n, m)
    p = cpct.Plan(n, n, m)
    bd = torch.from_numpy(b.astype(np.float32)).cuda()
    x1, i1 = cpct.spgl1(p, bd, sigma)
    x2, i2 = cpct.spgl1(p, bd, sigma, x0=x1)
    print("cold", i1, "warm", i2)
    assert i2["status"] == 1 and i2["iterations"] <= max(5, i1["iterations"] // 5)
    # without the filter the stuck columns enter the misfit: a different problem
    x3, i3 = cpct.spgl1(p, bd, sigma, opts=cpct.make_opts(ring_filter=False, max_iter=50))
    assert i3["status"] in (1, 3)


@pytest.mark.parametrize("where", ["b", "x0"])
def test_spgl1_nonfinite_input(torch_cuda, where):
    """A NaN in the data or in the warm start ends the solve with
    CPCT_ENONFINITE (status 5) instead of iterating on NaNs."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    n, m = 32, 16
    geo, x_true, b, sigma = _problem(n, m, seed=9)
    b32 = b.astype(np.float32)
    x0 = np.zeros((n, n), dtype=np.float32)
    if where == "b":
        b32[3, 5] = np.nan
    else:
        x0[7, 7] = np.nan
    p = cpct.Plan(n, n, m)
    with pytest.raises(cpct.CpctError) as ei:
        cpct.spgl1(p, torch.from_numpy(b32).cuda(), sigma, x0=torch.from_numpy(x0).cuda())
    assert ei.value.status == -5


def _proj_case(case, rng):
    if case == "gauss":
        v = rng.standard_normal(1 << 20)
        return v, 0.1 * np.abs(v).sum()
    if case == "sparse":
        v = rng.standard_normal(1 << 18) * (rng.random(1 << 18) < 0.1)
        return v, 0.02 * np.abs(v).sum()
    if case == "ties":
        v = rng.choice([-3.0, -2.0, -1.0, 1.0, 2.0, 3.0], size=100_003)
        return v, 0.25 * np.abs(v).sum()
    if case == "wide":
        v = np.exp(rng.uniform(-80.0, 20.0, 300_001)) * rng.choice([-1.0, 1.0], 300_001)
        return v, 0.3 * np.abs(v).sum()
    if case == "ragged":
        v = rng.laplace(size=1_000_003)
        return v, 0.5 * np.abs(v).sum()
    if case == "one":
        return np.array([-2.5]), 1.0
    if case == "identity":
        v = rng.standard_normal(4097)
        return v, 1.5 * np.abs(v.astype(np.float32).astype(np.float64)).sum()
    if case == "zero_tau":
        return rng.standard_normal(1000), 0.0
    if case == "zero_v":
        return np.zeros(5000), 3.0
    raise ValueError(case)


@pytest.mark.parametrize("case", ["gauss", "sparse", "ties", "wide", "ragged", "one", "identity", "zero_tau",
                                  "zero_v"])
def test_project_l1_matches_oracle(torch_cuda, case):
    """The device threshold is exact for the FP32 input: the same active set as
    the FP64 sort-based oracle, theta to FP64 rounding, outputs to FP32
    rounding of |v| - theta."""
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(1380)
    v, tau = _proj_case(case, rng)
    v32 = v.astype(np.float32)
    v64 = v32.astype(np.float64)
    ref = spgl1.project_l1(v64, tau)
    vd = torch.from_numpy(v32).cuda()
    out, theta = cpct.project_l1(vd, tau)
    out2, theta2 = cpct.project_l1(vd, tau)
    o = out.cpu().numpy().astype(np.float64)
    assert torch.equal(out, out2) and theta == theta2
    act = ref != 0
    if case in ("identity", "zero_v"):
        assert theta == 0.0 and np.array_equal(o, v64)
        return
    if case == "zero_tau":
        assert not o.any()
        return
    theta_ref = float(np.median(np.abs(v64[act]) - np.abs(ref[act])))
    assert abs(theta - theta_ref) <= 1e-12 * max(theta_ref, 1e-300), (theta, theta_ref)
    # active sets agree except for values within FP32 rounding of theta
    near = np.abs(np.abs(v64) - theta_ref) <= 2 * np.spacing(np.float32(theta_ref))
    assert np.array_equal((o != 0)[~near], act[~near])
    ulp = np.spacing(np.abs(v32)).astype(np.float64)
    assert np.all(np.abs(o - ref) <= ulp + np.spacing(np.float32(theta_ref)))
    assert np.all(np.sign(o[o != 0]) == np.sign(v64[o != 0]))
    # ||out||_1 = tau to FP32 rounding of the outputs
    assert abs(np.abs(o).sum() - tau) <= 1e-6 * tau


def test_project_l1_batched_equals_single(torch_cuda):
    torch = torch_cuda
    from paper_1009_1380_gb300 import cpct
    rng = np.random.default_rng(77)
    vs = [torch.from_numpy(rng.standard_normal(5000).astype(np.float32)).cuda() for _ in range(5)]
    taus = [0.0, 10.0, 100.0, 1e6, 3.5]
    outs, th = cpct.project_l1_batched(vs, taus)
    for v, t, o, h in zip(vs, taus, outs, th):
        o1, h1 = cpct.project_l1(v, t)
        assert torch.equal(o, o1) and h == h1
