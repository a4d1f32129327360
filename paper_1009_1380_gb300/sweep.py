"""Few-view and low-dose sweeps of the reconstruction.

The paper's Conclusions expect the basis-pursuit reconstruction to allow
lower dose or fewer views for a similar image quality.  This module measures
that on synthetic slices: for each number of views M and noise level
(standard deviation as a fraction of the sinogram's maximum; the dose scales
as its inverse square), it reconstructs fresh slices with

* the filtered back-projection of the ring-filtered data (``radon_fbp``, the
  paper's "using a filter" baseline),
* SPGL1 on the L1 problem of section "Introduction" (l1 of the
  phase-contrast image x, constraint ||F(R x - b)|| <= sigma), and
* for absorption data of the same objects (the Conclusions' reference:
  absorption datasets with total-variation regularisation), the filtered
  back-projection and the analysis-l1 variant (l1 of the object's
  horizontal differences, u = C z; ``cpct_synth_dh``),

and reports the relative L2 error of each against the true image (the
phase-contrast image x = lap(u), or the object u for absorption data), with
the SPGL1 iterations and wall time.  Every step runs in the library's
kernels; PyTorch only holds device memory.

Command line: ``python -m paper_1009_1380_gb300.sweep --help``.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import cpct, synth

SWEEP_CONFIG_INDEX = 6  # seeds of the sweep's slices (synth.rng_for)


def _slices(plan, count, noise, first, torch, absorption=False, n_shapes=6):
    """Phase-contrast data of x = lap(u) (or absorption data of u): images,
    device sinograms with noise and stuck columns, misfit bounds."""
    n, m = plan.n, plan.n_views
    imgs, bs, sig = [], [], []
    for i in range(count):
        rng = synth.rng_for(SWEEP_CONFIG_INDEX, first + i)
        u, _ = synth.ellipse_phantom(n, n_shapes, rng, axes_range=(0.1 * n, 0.3 * n))
        img = (u if absorption else synth.laplacian5(u)).astype(np.float32)
        y = plan.fwd(torch.from_numpy(img).cuda()).cpu().numpy()
        b, std, _ = synth.corrupt_sinogram(y, rng, noise_frac=noise)
        imgs.append(img)
        bs.append(torch.from_numpy(b.astype(np.float32)).cuda())
        sig.append(std * np.sqrt(m * n - n + 4))
    return imgs, bs, sig


def _fbp_errors(plan, imgs, bs, torch):
    filt = torch.empty((plan.n_views, plan.n_det), device="cuda", dtype=torch.float32)
    e = []
    for img, b in zip(imgs, bs):
        cpct.ring_filter(plan, b, out=filt)
        e.append(_rel(plan.fbp(filt).cpu().numpy(), img))
    return e


def _rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def run_point(n, m, noise, count, torch, max_iter=400, synth_iters=300):
    """One (views, noise) point: mean relative errors and solver costs."""
    plan0 = cpct.Plan(n, n, m)
    plan0.auto_caps(count)
    plans = [plan0] + [cpct.clone(plan0) for _ in range(count - 1)]
    # phase contrast: FBP and SPGL1 (l1 of x), batched over the slices
    xs, bs, sig = _slices(plan0, count, noise, 0, torch)
    e_fbp = _fbp_errors(plan0, xs, bs, torch)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    xr, inf = cpct.spgl1_batched(plans, bs, sig, opts=cpct.make_opts(max_iter=max_iter))
    torch.cuda.synchronize()
    t_spg = time.perf_counter() - t0
    e_spg = [_rel(xr[i].cpu().numpy(), xs[i]) for i in range(count)]
    # absorption: FBP and the analysis-l1 variant (z = horizontal
    # differences of u, u = C z)
    us, bu, sig_u = _slices(plan0, count, noise, 0, torch, absorption=True)
    e_fbp_u = _fbp_errors(plan0, us, bu, torch)
    t0 = time.perf_counter()
    zr, inf_z = cpct.spgl1_batched(plans, bu, sig_u, opts=cpct.make_opts(max_iter=synth_iters, synth_dh=True))
    torch.cuda.synchronize()
    t_syn = time.perf_counter() - t0
    e_syn = [_rel(cpct.synth_dh(zr[i]).cpu().numpy(), us[i]) for i in range(count)]
    for p in plans:
        p.close()
    return {"n": n, "views": m, "noise": noise, "slices": count,
            "fbp_rel_err": float(np.mean(e_fbp)), "spgl1_rel_err": float(np.mean(e_spg)),
            "spgl1_at_root": sum(1 for f in inf if f["status"] == 1),
            "spgl1_iterations_mean": float(np.mean([f["iterations"] for f in inf])), "spgl1_wall_s": t_spg,
            "absorption_fbp_rel_err": float(np.mean(e_fbp_u)),
            "analysis_l1_rel_err": float(np.mean(e_syn)),
            "analysis_l1_at_root": sum(1 for f in inf_z if f["status"] == 1),
            "analysis_l1_iterations_mean": float(np.mean([f["iterations"] for f in inf_z])),
            "analysis_l1_wall_s": t_syn}


def run(n=256, views=(32, 64, 128, 256), noises=(0.01, 0.04), count=4, max_iter=400, synth_iters=300, log=None):
    import torch
    pts = []
    for m in views:
        for nz in noises:
            r = run_point(n, m, nz, count, torch, max_iter=max_iter, synth_iters=synth_iters)
            if log:
                log(r)
            pts.append(r)
    return pts


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--views", default="32,64,128,256")
    ap.add_argument("--noise", default="0.01,0.04")
    ap.add_argument("--slices", type=int, default=4)
    ap.add_argument("--max-iter", type=int, default=400)
    a = ap.parse_args(argv)
    pts = run(a.n, tuple(int(v) for v in a.views.split(",")), tuple(float(v) for v in a.noise.split(",")), a.slices,
              a.max_iter, log=lambda r: print(json.dumps(r), flush=True))
    print(json.dumps({"sweep": pts}))


if __name__ == "__main__":
    main()
