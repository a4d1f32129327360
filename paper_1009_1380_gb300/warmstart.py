"""Learned warm start for SPGL1 (an extension: the paper has none).

The method generates its own training data: for synthetic slices it computes
the filtered back-projection of the ring-filtered data (radon_fbp) and the
converged cold-start SPGL1 solution of the paper's L1 problem; a U-Net
(cpct_unet_*, trained here with the project's own forward and backward
kernels) learns to map the first to the second.  A new slice then starts
SPGL1 from the prediction projected onto an l1 ball, x0 = P_tau0(net(FBP))
with tau0 an estimate of the root tau* = ||x*||_1: prediction noise spread
over all pixels inflates the l1 norm of a raw prediction, and the number of
SPGL1 iterations from a good x0 grows quickly with the error of tau0 (on a
64^2 problem: 4 iterations from x* itself, 33-40 from x* plus noise with
tau0 within 5% of tau*, 56-82 at 10-20% off, 137 cold).  So
tau0 = kappa ||soft(net(FBP), theta s)||_1, with the noise floor theta and the
factor kappa calibrated on training slices (``calibrate``).  The plain
cold-started solver is the fallback for any slice whose warm solve does not
reach the root, and its root test decides whether a warm solve succeeded
(the residual criterion is unchanged).  The same calibrated projection of
the FBP image itself is the non-learned warm start it is compared with.

Inputs are scaled per slice by s = the standard deviation of the FBP image:
the network sees FBP / s and predicts x / s.

Command line: ``python -m paper_1009_1380_gb300.warmstart --help``.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import cpct, synth

CONFIG = synth.CONFIGS["c5_warm512"]


def layer_shapes(levels, base):
    """(Cout, Cin, k) of every layer in the parameter order of cpct_unet."""
    c = [base << l for l in range(levels)]
    out = []
    for l in range(levels):
        out += [(c[l], 1 if l == 0 else c[l - 1], 3), (c[l], c[l], 3)]
    for l in range(levels - 2, -1, -1):
        out += [(c[l], c[l + 1], 3), (c[l], 2 * c[l], 3), (c[l], c[l], 3)]
    return out + [(1, c[0], 1)]


def he_init(levels, base, seed=0):
    """He-normal 3x3 weights, zero biases and a zero head: the network starts
    as the identity map of its (scaled) input."""
    rng = np.random.default_rng(seed)
    parts = []
    shapes = layer_shapes(levels, base)
    for i, (co, ci, k) in enumerate(shapes):
        if i == len(shapes) - 1:
            parts.append(np.zeros(co * k * k * ci))
        else:
            parts.append(rng.standard_normal(co * k * k * ci) * np.sqrt(2.0 / (ci * k * k)))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def make_slices(plan, count, first_index, torch, n_shapes=None, config_index=None):
    """Synthetic slices: b (count, M, Ns) device, sigma (count,), FBP inputs
    (count, N, N) device.  Slice i uses the seed of slice first_index + i."""
    n, m = plan.n, plan.n_views
    ci = CONFIG["index"] if config_index is None else config_index
    ns = CONFIG["n_shapes"] if n_shapes is None else n_shapes
    b = torch.empty((count, m, plan.n_det), device="cuda", dtype=torch.float32)
    fbp = torch.empty((count, n, n), device="cuda", dtype=torch.float32)
    sigma = np.empty(count)
    filt = torch.empty((m, plan.n_det), device="cuda", dtype=torch.float32)
    for i in range(count):
        rng = synth.rng_for(ci, first_index + i)
        u, _ = synth.ellipse_phantom(n, ns, rng)
        x = torch.from_numpy(synth.laplacian5(u).astype(np.float32)).cuda()
        y = plan.fwd(x).cpu().numpy()
        bi, std, _ = synth.corrupt_sinogram(y, rng)
        b[i].copy_(torch.from_numpy(bi.astype(np.float32)))
        sigma[i] = std * np.sqrt(m * plan.n_det - plan.n_det + 4)
        cpct.ring_filter(plan, b[i], out=filt)
        plan.fbp(filt, out=fbp[i])
    return b, sigma, fbp


def solve(plans, b, sigma, opts, x0=None):
    """Batched SPGL1 over all slices in groups of len(plans); returns
    (x (count, N, N), infos, wall seconds)."""
    torch = plans[0]._torch
    count, P = b.shape[0], len(plans)
    xs = torch.empty((count, plans[0].n, plans[0].n), device=b.device, dtype=torch.float32)
    infos = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for g in range(0, count, P):
        k = min(P, count - g)
        x0s = None if x0 is None else [x0[g + i] for i in range(k)]
        out, inf = cpct.spgl1_batched(plans[:k], [b[g + i] for i in range(k)], list(sigma[g:g + k]), x0s=x0s,
                                      opts=opts)
        for i in range(k):
            xs[g + i].copy_(out[i])
        infos.extend(inf)
    torch.cuda.synchronize()
    return xs, infos, time.perf_counter() - t0


def scales(fbp):
    """Per-slice standard deviations (host float64), kept away from zero."""
    return np.maximum(cpct.slice_moments(fbp)[1], 1e-12)


CLIP_FACTOR = 2.0      # clip at twice the median of the recent gradient norms
CLIP_WINDOW = 50
DIVERGE_FACTOR = 1.5   # an epoch loss this far above the best restores the best weights


def train(net, fbp, target, epochs, batch, lr, seed=0, log=None):
    """Adam on (FBP / s, x / s) pairs; returns the per-epoch mean losses.

    Safeguards for a network without normalisation layers: cosine decay of
    the learning rate to 5% over all steps; gradients clipped to twice the
    median norm of the last 50 steps (after 20 steps); the weights of the best
    epoch are kept, and an epoch whose loss exceeds 1.5x the best restores
    them and halves the learning rate."""
    torch = net._torch
    inv = 1.0 / scales(fbp)
    inp, tgt = cpct.slice_scale(fbp, inv), cpct.slice_scale(target, inv)
    rng = np.random.default_rng(seed)
    count = fbp.shape[0]
    steps_per_epoch = max(1, count // batch)
    total = epochs * steps_per_epoch
    losses, norms = [], []
    best_loss, best_params = float("inf"), None
    scale_lr = 1.0
    step = 0
    for ep in range(epochs):
        perm = rng.permutation(count)
        tot, nb = 0.0, 0
        for g in range(0, count - batch + 1, batch):
            idx = torch.from_numpy(perm[g:g + batch]).cuda()
            xb, tb = inp.index_select(0, idx).contiguous(), tgt.index_select(0, idx).contiguous()
            tot += net.backward(xb, tb)
            lr_t = scale_lr * lr * (0.05 + 0.95 * 0.5 * (1.0 + np.cos(np.pi * step / total)))
            clip = CLIP_FACTOR * float(np.median(norms[-CLIP_WINDOW:])) if len(norms) >= 20 else 0.0
            norms.append(net.adam_step(lr_t, max_grad_norm=clip, return_norm=True))
            nb += 1
            step += 1
        net.sync()  # raises if a bounded device wait of the epoch's passes expired
        losses.append(tot / max(nb, 1))
        if log:
            log(f"epoch {ep}: loss {losses[-1]:.4e}")
        if losses[-1] < best_loss:
            best_loss, best_params = losses[-1], net.get_params()
        elif losses[-1] > DIVERGE_FACTOR * best_loss and best_params is not None:
            net.set_params(best_params)
            scale_lr *= 0.5
            if log:
                log(f"epoch {ep}: loss above {DIVERGE_FACTOR}x the best, weights restored, learning rate halved")
    if best_params is not None and losses[-1] > best_loss:
        net.set_params(best_params)
    return losses


def predict(net, fbp, batch):
    torch = net._torch
    s = scales(fbp)
    inp = cpct.slice_scale(fbp, 1.0 / s)
    out = torch.empty_like(inp)
    for g in range(0, fbp.shape[0], batch):
        k = min(batch, fbp.shape[0] - g)
        net.forward(inp[g:g + k], out=out[g:g + k])
    net.sync()  # raises if a bounded device wait of a forward pass expired
    return cpct.slice_scale(out, s, out=out)


# candidate noise floors (in units of the prediction's per-slice standard
# deviation) of the starting-radius estimate
THETAS = (0.0, 0.02, 0.05, 0.1, 0.2, 0.3, 0.5, 0.75, 1.0)


def _soft_l1(x_hat, theta, s=None):
    """Per slice ||soft(x_hat, theta s)||_1, s the slice's standard deviation
    (cpct_slice_moments and cpct_slice_soft_l1)."""
    s = cpct.slice_moments(x_hat)[1] if s is None else s
    return cpct.slice_soft_l1(x_hat, theta * s)


def calibrate_table(soft, tau_star):
    """The calibration from soft[t][i] = ||soft(x_hat_i, THETAS[t] s_i)||_1:
    theta minimises the spread of log(tau* / ||soft||_1) over the slices,
    kappa is the median ratio at that theta."""
    tau_star = np.asarray(tau_star, dtype=np.float64)
    best = None
    for th, col in zip(THETAS, soft):
        r = tau_star / np.maximum(np.asarray(col, dtype=np.float64), 1e-30)
        spread = float(np.std(np.log(r)))
        if best is None or spread < best["spread"]:
            best = {"theta": th, "kappa": float(np.median(r)), "spread": spread}
    return best


def calibrate(x_hat, tau_star):
    """Starting-radius estimate tau0 = kappa ||soft(x_hat, theta s)||_1 with
    theta and kappa fitted on the given slices (calibrate_table)."""
    s = cpct.slice_moments(x_hat)[1]
    return calibrate_table([_soft_l1(x_hat, th, s) for th in THETAS], tau_star)


def project_start(x_hat, cal):
    """x0 = P_tau0(x_hat), tau0 = kappa ||soft(x_hat, theta s)||_1 (exact
    projection per slice)."""
    x0 = torch_empty_like(x_hat)
    tau0 = cal["kappa"] * _soft_l1(x_hat, cal["theta"])
    cpct.project_l1_batched([x_hat[i] for i in range(x_hat.shape[0])], tau0,
                            outs=[x0[i] for i in range(x_hat.shape[0])])
    return x0


def torch_empty_like(t):
    return t.new_empty(t.shape)


def evaluate(net, plans, b, sigma, fbp, opts, batch, kappa):
    """Cold start, FBP warm start and learned warm start on the same slices.

    ``kappa`` = {"fbp": cal, "learned": cal} from ``calibrate``.  A warm solve
    that does not reach the root is redone cold (the fallback); its time
    counts against the warm start."""
    torch = plans[0]._torch
    res = {}
    x_cold, inf_cold, t_cold = solve(plans, b, sigma, opts)
    res["cold"] = _summary(inf_cold, t_cold, 0.0)
    for name in ("fbp", "learned"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x_hat = fbp if name == "fbp" else predict(net, fbp, batch)
        torch.cuda.synchronize()
        t_pred = time.perf_counter() - t0
        x0 = project_start(x_hat, kappa[name])
        torch.cuda.synchronize()
        t_net = time.perf_counter() - t0
        x, inf, t = solve(plans, b, sigma, opts, x0=x0)
        bad = [i for i, f in enumerate(inf) if f["status"] != 1]
        t_fb = 0.0
        if bad:
            idx = torch.tensor(bad, device=b.device)
            _, inf_fb, t_fb = solve(plans, b.index_select(0, idx).contiguous(), sigma[bad], opts)
            for j, i in enumerate(bad):
                inf[i] = dict(inf_fb[j], fallback=True)
        r = _summary(inf, t + t_fb + t_net, t_net)
        r["predict_s"] = t_pred
        r["fallbacks"] = len(bad)
        # quality of the start: relative L2 distance to the cold solution
        d0 = (x0 - x_cold).flatten(1).norm(dim=1) / x_cold.flatten(1).norm(dim=1).clamp_min(1e-30)
        dh = (x_hat - x_cold).flatten(1).norm(dim=1) / x_cold.flatten(1).norm(dim=1).clamp_min(1e-30)
        r["start_rel_err_mean"] = float(d0.mean().item())
        r["prediction_rel_err_mean"] = float(dh.mean().item())
        # the warm and the cold solution of each slice: l1 norms
        l1w = np.array([f["xnorm1"] for f in inf])
        l1c = np.array([f["xnorm1"] for f in inf_cold])
        r["l1_rel_diff_vs_cold_mean"] = float(np.mean(np.abs(l1w - l1c) / l1c))
        res[name] = r
    # the learned start with the network overlapped with the solves
    x_p, inf_p, t_p, t_pnet = solve_pipelined(net, plans, b, sigma, fbp, opts, batch, kappa["learned"])
    bad = [i for i, f in enumerate(inf_p) if f["status"] != 1]
    t_fb = 0.0
    if bad:
        idx = torch.tensor(bad, device=b.device)
        _, inf_fb, t_fb = solve(plans, b.index_select(0, idx).contiguous(), sigma[bad], opts)
        for j, i in enumerate(bad):
            inf_p[i] = dict(inf_fb[j], fallback=True)
    r = _summary(inf_p, t_p + t_fb, t_pnet)
    r["fallbacks"] = len(bad)
    res["learned_pipelined"] = r
    return res


def solve_pipelined(net, plans, b, sigma, fbp, opts, batch, cal):
    """Learned warm start with the network off the critical path: a host
    thread predicts and projects the starts of slice group g+1 on its own
    stream while group g is solved (groups of len(plans) slices).  Returns
    (x, infos, wall seconds, seconds spent in the network thread)."""
    import queue
    import threading
    torch = plans[0]._torch
    count, P = b.shape[0], len(plans)
    groups = [(g, min(count, g + P)) for g in range(0, count, P)]
    q = queue.Queue(maxsize=2)
    t_net = [0.0]
    err = []

    def producer():
        try:
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                for g0, g1 in groups:
                    t0 = time.perf_counter()
                    x0 = project_start(predict(net, fbp[g0:g1], batch), cal)
                    stream.synchronize()
                    t_net[0] += time.perf_counter() - t0
                    q.put(x0)
        except Exception as e:  # surfaced in the consumer
            err.append(e)
            q.put(None)

    xs = torch.empty((count, plans[0].n, plans[0].n), device=b.device, dtype=torch.float32)
    infos = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    th = threading.Thread(target=producer, daemon=True)
    th.start()
    for g0, g1 in groups:
        x0 = q.get()
        if x0 is None:
            th.join()
            raise err[0]
        k = g1 - g0
        out, inf = cpct.spgl1_batched(plans[:k], [b[g0 + i] for i in range(k)], list(sigma[g0:g1]),
                                      x0s=[x0[i] for i in range(k)], opts=opts)
        for i in range(k):
            xs[g0 + i].copy_(out[i])
        infos.extend(inf)
    th.join()
    torch.cuda.synchronize()
    return xs, infos, time.perf_counter() - t0, t_net[0]


def _summary(infos, wall, t_net):
    its = np.array([f["iterations"] for f in infos])
    roots = sum(1 for f in infos if f["status"] == 1)
    return {"slices": len(infos), "at_root": roots, "wall_s": wall, "net_s": t_net,
            "slices_per_s": roots / wall if wall > 0 else None, "iterations_mean": float(its.mean()),
            "iterations_median": float(np.median(its)), "iterations_max": int(its.max()),
            "ticks_mean": float(np.mean([f["ticks"] for f in infos])),
            "ticks_max": int(max(f["ticks"] for f in infos)),
            # line-search trials (accepted or not); ticks - trials are the
            # bookkeeping ticks (the first, and one or two per Newton update)
            "trials_mean": float(np.mean([f["trials"] for f in infos]))}


INFER_BATCH = 32  # images per forward call at inference (deep levels fill the GPU)


def run(pairs, eval_slices, epochs, batch, lr, levels, base, plans_per_group, target_iters, eval_tol, n=None, m=None,
        log=print):
    import torch
    n = CONFIG["n"] if n is None else n
    m = CONFIG["n_views"] if m is None else m
    out = {"config": {"n": n, "views": m, "pairs": pairs, "eval_slices": eval_slices, "epochs": epochs,
                      "batch": batch, "lr": lr, "levels": levels, "base": base, "target_max_iter": target_iters,
                      "eval_opt_tol": eval_tol}}
    plan0 = cpct.Plan(n, n, m)
    plan0.auto_caps(plans_per_group)  # work items for a group of slices at once
    plans = [plan0] + [cpct.clone(plan0) for _ in range(plans_per_group - 1)]
    t0 = time.perf_counter()
    b, sigma, fbp = make_slices(plan0, pairs, 0, torch)
    out["gen_inputs_s"] = time.perf_counter() - t0
    x_t, inf_t, t_sol = solve(plans, b, sigma, cpct.make_opts(max_iter=target_iters))
    out["targets"] = _summary(inf_t, t_sol, 0.0)
    log(f"targets: {out['targets']}")
    net = cpct.UNet(levels, base, batch, n, n)
    net.set_params(he_init(levels, base, seed=7))
    t0 = time.perf_counter()
    losses = train(net, fbp, x_t, epochs, batch, lr, log=log)
    torch.cuda.synchronize()
    out["train_s"] = time.perf_counter() - t0
    out["train_loss"] = losses
    # calibration of the starting radius on (up to 256) training slices
    k = min(pairs, 256)
    tau_star = [f["xnorm1"] for f in inf_t[:k]]
    kappa = {"fbp": calibrate(fbp[:k], tau_star), "learned": calibrate(predict(net, fbp[:k], batch), tau_star)}
    out["kappa"] = kappa
    log(f"kappa {kappa}")
    del b, fbp, x_t
    # inference copy of the trained weights with a larger batch
    infer_batch = min(INFER_BATCH, eval_slices)
    net_inf = cpct.UNet(levels, base, infer_batch, n, n)
    net_inf.set_params(net.get_params())
    net.close()
    be, se, fe = make_slices(plan0, eval_slices, pairs, torch)
    out["eval"] = evaluate(net_inf, plans, be, se, fe, cpct.make_opts(opt_tol=eval_tol, max_iter=target_iters),
                           infer_batch, kappa)
    c, w = out["eval"]["cold"], out["eval"]["learned"]
    out["speedup_wall"] = c["wall_s"] / w["wall_s"] if w["wall_s"] > 0 else None
    wp = out["eval"]["learned_pipelined"]
    out["speedup_wall_pipelined"] = c["wall_s"] / wp["wall_s"] if wp["wall_s"] > 0 else None
    out["iterations_ratio"] = w["iterations_mean"] / c["iterations_mean"] if c["iterations_mean"] > 0 else None
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--pairs", type=int, default=4096)
    ap.add_argument("--eval", type=int, default=512)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--levels", type=int, default=5)
    ap.add_argument("--base", type=int, default=32)
    ap.add_argument("--group", type=int, default=64, help="slices per batched SPGL1 solve")
    ap.add_argument("--target-iters", type=int, default=500)
    ap.add_argument("--eval-tol", type=float, default=1e-3)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--views", type=int, default=None)
    ap.add_argument("--out", default=None, help="write the JSON summary here")
    a = ap.parse_args(argv)
    res = run(a.pairs, a.eval, a.epochs, a.batch, a.lr, a.levels, a.base, a.group, a.target_iters, a.eval_tol,
              n=a.n, m=a.views)
    line = json.dumps(res)
    print(line)
    if a.out:
        with open(a.out, "w") as fh:
            fh.write(line + "\n")


if __name__ == "__main__":
    main()
