"""SPGL1 basis-pursuit denoising, FP64 reference (oracle).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

Section "Introduction": the reconstruction is the L1 problem

    minimize ||x||_1  subject to  ||filter(Radon{x} - data)||_2 < eps,

solved with SPGL1 (van den Berg and Friedlander, SIAM J. Sci. Comput. 31(2),
2008), which only needs the operator and its adjoint.  Because the filter F
is an orthogonal projector, filter(Radon{x} - data) = (F R) x - F data, so the
solver is applied to A = F R with right-hand side F data and sigma = eps.

The published method, restated:

* the Pareto curve phi(tau) = ||b - A x_tau||_2, where x_tau solves the LASSO
  problem  min ||A x - b||_2  s.t. ||x||_1 <= tau, is convex, decreasing and
  differentiable with phi'(tau) = -||A^T r_tau||_inf / ||r_tau||_2;
* the root phi(tau) = sigma is found by Newton's method,
  tau <- tau + (||r|| - sigma) ||r|| / ||A^T r||_inf, each LASSO problem being
  solved only as accurately as the current root error requires (duality gap);
* each LASSO problem is solved by the spectral projected gradient method:
  x <- P_tau(x - alpha g) with g = -A^T r, Barzilai-Borwein step lengths
  alpha = s^T s / s^T y, and a non-monotone backtracking search along the
  projection arc against the maximum of the last few objective values;
* P_tau is the Euclidean projection onto the l1 ball of radius tau.

Inexact Newton and termination (readings): the LASSO problem for the current
tau counts as solved when its relative duality gap is <= max(opt_tol,
relative error in f) or when it stagnates (relative decrease of f in the last
step <= dec_tol = 1e-4 while ||r|| > 2 sigma, <= 0.1 |(||r|| - sigma)| /
||r|| otherwise); the tau Newton step is then taken, and the root is accepted
when | ||r|| - sigma | <= opt_tol max(1, ||b||) at such a point (root error
measured relative to the data).

Constants (the paper gives none; readings): memory of 3 objective values,
sufficient-decrease gamma = 1e-4, step lengths clamped to [1e-16, 1e5],
a flat projection arc is detected when two consecutive trial displacements
have the same norm to 1e-6 (the step then jumps to half the displacement's
scale), after every Newton update of tau the step restarts from the projected
gradient,
opt_tol = 1e-4, bp_tol = 1e-6, at most 30 halvings per line search.

Parity pins (tests/test_oracle_spgl1.py): the l1 projection is pinned by its
optimality conditions and by an independent bisection; the solver with
sigma = 0 is pinned against a linear-programming solve of basis pursuit and
with sigma > 0 by the optimality certificate (root error and duality gap).
Exact iterate-by-iterate parity with the GPU solver is NOT pinned: FP32
operator rounding can flip line-search branches ("parity unpinned" for the
iterate sequence; final-point parity is pinned by the certificate).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------------------
# Euclidean projection onto the l1 ball
# ---------------------------------------------------------------------------
def project_l1(v: np.ndarray, tau: float) -> np.ndarray:
    """argmin_x ||x - v||_2 s.t. ||x||_1 <= tau (sort-based threshold search).

    The solution is soft thresholding x = sign(v) max(|v| - theta, 0) with the
    smallest theta >= 0 for which ||x||_1 <= tau.  Sorting |v| in decreasing
    order u_1 >= u_2 >= ..., theta = (sum_{i<=rho} u_i - tau) / rho where rho
    is the largest j with u_j > (sum_{i<=j} u_i - tau) / j.
    """
    v = np.asarray(v, dtype=np.float64)
    if tau <= 0:
        return np.zeros_like(v)
    a = np.abs(v).ravel()
    if a.sum() <= tau:
        return v.copy()
    u = np.sort(a)[::-1]
    cs = np.cumsum(u)
    j = np.arange(1, u.size + 1)
    cond = u - (cs - tau) / j > 0
    rho = np.nonzero(cond)[0][-1]
    theta = (cs[rho] - tau) / (rho + 1)
    return np.sign(v) * np.maximum(np.abs(v) - theta, 0.0)


def project_l1_bisect(v: np.ndarray, tau: float, iters: int = 200) -> np.ndarray:
    """The same projection by bisection on theta (independent check)."""
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    if tau <= 0:
        return np.zeros_like(v)
    if a.sum() <= tau:
        return v.copy()
    lo, hi = 0.0, float(a.max())
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if np.maximum(a - mid, 0.0).sum() > tau:
            lo = mid
        else:
            hi = mid
    return np.sign(v) * np.maximum(a - hi, 0.0)


# ---------------------------------------------------------------------------
# solver
# ---------------------------------------------------------------------------
EXIT_ROOT_FOUND = 1
EXIT_BP_FOUND = 2
EXIT_ITERATIONS = 3
EXIT_LINE_ERROR = 4


@dataclass
class Options:
    max_iter: int = 300
    opt_tol: float = 1e-4
    bp_tol: float = 1e-6
    memory: int = 3
    gamma: float = 1e-4
    step_min: float = 1e-16
    step_max: float = 1e5
    max_line: int = 30
    dec_tol: float = 1e-4
    restart_step: bool = True


@dataclass
class Info:
    status: int = 0
    iterations: int = 0
    n_prod_A: int = 0
    n_prod_At: int = 0
    tau: float = 0.0
    rnorm: float = 0.0
    xnorm1: float = 0.0
    rel_gap: float = 0.0
    history: list = field(default_factory=list)


def spgl1(A, At, b, sigma, x0=None, tau0=None, opts: Options | None = None):
    """Solve min ||x||_1 s.t. ||A x - b||_2 <= sigma.

    ``A`` and ``At`` are callables (real arrays in, real arrays out).  Returns
    (x, Info).  ``x0`` warm-starts the iterate; ``tau0`` defaults to 0 for a
    cold start and to ||x0||_1 for a warm start.
    """
    o = opts or Options()
    info = Info()
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))

    def Ax(x):
        info.n_prod_A += 1
        return A(x)

    def Atr(r):
        info.n_prod_At += 1
        return At(r)

    if x0 is None:
        x = None
        tau = 0.0 if tau0 is None else float(tau0)
    else:
        x = np.asarray(x0, dtype=np.float64)
        tau = float(np.abs(x).sum()) if tau0 is None else float(tau0)
    if x is None:
        xshape = Atr(b).shape
        x = np.zeros(xshape)
    x = project_l1(x, tau)
    r = b - Ax(x)
    g = -Atr(r)
    f = 0.5 * float(r.ravel() @ r.ravel())

    def pg_step(x, g, tau):
        # step length 1 / ||P_tau(x - g) - x||_inf from the projected gradient
        dx = project_l1(x - g, tau) - x
        dxn = float(np.abs(dx).max()) if dx.size else 0.0
        return o.step_max if dxn < 1.0 / o.step_max else min(o.step_max, max(o.step_min, 1.0 / dxn))

    alpha = pg_step(x, g, tau)

    fhist = [f]
    it = 0
    f_old = None
    n_stationary = 0
    while True:
        rnorm = float(np.linalg.norm(r))
        gnorm = float(np.abs(g).max())
        # duality gap of the current LASSO problem, in the scale of f
        gap = float(r.ravel() @ (r - b).ravel()) + tau * gnorm
        rel_gap = abs(gap) / max(1.0, f)
        err_root = abs(rnorm - sigma) / max(1.0, bnorm)
        err_f = abs(f - 0.5 * sigma ** 2) / max(1.0, f)
        info.history.append((it, tau, rnorm, rel_gap))

        status = 0
        # the current LASSO problem is solved as accurately as the distance
        # to the root requires: certified by its duality gap, or stagnant
        # (objective decrease below 1e-4 relative far from the root, below a
        # tenth of the relative root error near it)
        solved_sub = rel_gap <= max(o.opt_tol, err_f)
        if f_old is not None and f > 0:
            dec = abs(f - f_old) / f
            if rnorm > 2 * sigma:
                solved_sub = solved_sub or dec <= o.dec_tol
            else:
                solved_sub = solved_sub or dec <= 0.1 * abs(rnorm - sigma) / max(rnorm, 1e-300)
        if solved_sub:
            if err_root <= o.opt_tol:
                status = EXIT_ROOT_FOUND
            elif gnorm <= o.bp_tol * rnorm or rnorm <= o.bp_tol * bnorm:
                status = EXIT_BP_FOUND
        if status == 0 and it >= o.max_iter:
            status = EXIT_ITERATIONS
        if status:
            break

        if solved_sub and gnorm > 0:
            # Newton step on the Pareto curve
            tau_new = max(0.0, tau + (rnorm - sigma) * rnorm / gnorm)
            if tau_new < tau:
                # the ball shrank: project x onto it and bring the residual,
                # objective and gradient up to date with the projected x
                x = project_l1(x, tau_new)
                r = b - Ax(x)
                g = -Atr(r)
                f = 0.5 * float(r.ravel() @ r.ravel())
            tau_was_zero = tau == 0.0
            tau = tau_new
            if tau_was_zero or o.restart_step:
                # leaving tau = 0 (x = 0, no step history yet): restart the
                # step length from the projected gradient on the new ball
                alpha = pg_step(x, g, tau)

        # spectral projected gradient step, non-monotone arc search
        it += 1
        x_old, g_old, f_old = x, g, f
        fmax = max(fhist[-o.memory:])
        step = alpha
        accepted = False
        dn_prev = None
        gn = float(np.linalg.norm(g_old))
        for _ in range(o.max_line + 1):
            xt = project_l1(x_old - step * g_old, tau)
            rt = b - Ax(xt)
            ft = 0.5 * float(rt.ravel() @ rt.ravel())
            d = (xt - x_old).ravel()
            gtd = float(g_old.ravel() @ d)
            if gtd >= 0:
                break  # no descent along the arc: x is stationary for this tau
            if ft < fmax + o.gamma * gtd:
                accepted = True
                break
            dn = float(np.linalg.norm(d))
            if dn_prev is not None and abs(dn - dn_prev) <= 1e-6 * dn and gn > 0:
                # the arc is flat here (the projection saturates for long
                # steps): jump to the step whose gradient move is half the
                # current displacement
                step = min(0.5 * step, 0.5 * dn / gn)
            else:
                step *= 0.5
            dn_prev = dn
        if not accepted and gtd < 0 and ft < f_old:
            accepted = True  # halvings exhausted, but f decreased
        if not accepted:
            # no descent along the arc, or no measurable decrease after every
            # halving: x is stationary for the current LASSO problem to the
            # working precision, which is then solved (f unchanged registers
            # as stagnation at the next check); only repeated stationarity
            # without progress is a failure
            n_stationary += 1
            if n_stationary > 3:
                info.status = EXIT_LINE_ERROR
                break
            continue
        n_stationary = 0
        x, r, f = xt, rt, ft
        g = -Atr(r)
        s = (x - x_old).ravel()
        yv = (g - g_old).ravel()
        sts = float(s @ s)
        sty = float(s @ yv)
        alpha = o.step_max if sty <= 0 else min(o.step_max, max(o.step_min, sts / sty))
        if f > 0.5 * sigma ** 2:
            fhist.append(f)

    if info.status == 0:
        info.status = status
    info.iterations = it
    info.tau = tau
    info.rnorm = float(np.linalg.norm(r))
    info.xnorm1 = float(np.abs(x).sum())
    gnorm = float(np.abs(g).max())
    gap = float(r.ravel() @ (r - b).ravel()) + tau * gnorm
    info.rel_gap = abs(gap) / max(1.0, 0.5 * info.rnorm ** 2)
    return x, info
