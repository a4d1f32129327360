"""SPGL1 basis-pursuit denoising, FP64 reference (oracle).

TEST INFRASTRUCTURE ONLY -- never imported by the product path.

Section "Introduction": the reconstruction is the L1 problem

    minimize ||x||_1  subject to  ||filter(Radon{x} - data)||_2 < eps,

solved with SPGL1 (van den Berg and Friedlander, SIAM J. Sci. Comput. 31(2),
2008), which only needs the operator and its adjoint.  Because the filter F
is an orthogonal projector, filter(Radon{x} - data) = (F R) x - F data, so the
solver is applied to A = F R with right-hand side F data and sigma = eps.

The published method, restated (paper and its public reference code):

* Pareto curve phi(tau) = ||b - A x_tau||_2, x_tau a solution of the LASSO
  problem  min ||A x - b||_2  s.t. ||x||_1 <= tau; phi is convex, decreasing
  and differentiable, phi'(tau) = -||A^T r_tau||_inf / ||r_tau||_2;
* the root phi(tau) = sigma is found by Newton's method,
  tau <- tau + (||r|| - sigma) ||r|| / ||A^T r||_inf, each LASSO problem
  solved only roughly: tau is updated when the objective f = ||r||^2 / 2
  stops decreasing (relative change <= dec_tol while ||r|| > 2 sigma, and
  below a tenth of the root error once ||r|| <= 2 sigma), never two
  iterations in a row; the Barzilai-Borwein step is kept across updates;
  when tau decreases, x is projected onto the smaller ball;
* exit tests at the top of every iteration, in this order: least-squares
  solution (||g||_inf <= ls_tol ||r||); and, when the duality gap is small
  (|r^T (r - b) + tau ||g||_inf| / max(1, f) <= max(opt_tol, |f - sigma^2/2|
  / max(1, f))) or the root error is <= opt_tol: suboptimal BP (||r|| <=
  sigma), overridden by root found (root error <= opt_tol), overridden by
  BP solution (||r|| <= bp_tol ||b||); with
  a single fixed tau (the LASSO problem alone): optimal when the gap is <=
  opt_tol or ||r|| < opt_tol ||b||;
* each iteration is a spectral projected-gradient step: a non-monotone
  search along the projection arc x(s) = P_tau(x - s g), starting at the
  Barzilai-Borwein step s = gstep (s^T s / s^T y of the last step, clamped
  to [step_min, step_max]), halving it, against the largest of the last
  `memory` objective values (values with f <= sigma^2/2 are not recorded);
  if two consecutive rejected trials move x by displacements of the same
  norm (to 1e-6), the arc is flat and the gradient is rescaled so that the
  next displacement is a fraction 2^-k of the last one (k = 0, 1, ... per
  rescaling within the search);
* if the arc search fails (no sufficient decrease within max_line halvings,
  or a trial with no descent), a backtracking search along the fixed
  feasible direction d = P_tau(x - gstep g) - x follows (safeguarded
  quadratic interpolation of the step, else halving); if that fails too, x
  is kept, step_max is divided by 10 (at most max_line_errors times, then
  the solve stops with a line-search error) and gstep = min(step_max,
  gstep);
* P_tau is the Euclidean projection onto the l1 ball of radius tau.

Readings where the published method leaves a choice:

* root error |(||r|| - sigma)| / max(1, ||b||): the root certificate
  |(||r|| - sigma)| <= opt_tol max(1, ||b||) of the L1 problem's solution
  (the published code divides by max(1, ||r||), which is 10-30x stricter on
  the tomography problems here, where ||b|| >> sigma);
* the stagnation threshold near the root is 0.1 |(||r|| - sigma)| / ||r||,
  a relative root error: the published 0.1 |(||r|| - sigma)| compares a
  relative change of f with an absolute residual difference, so it depends
  on the scale of the data (scaling A and b by c leaves the relative change
  of f unchanged and multiplies |(||r|| - sigma)| by c); for data with
  ||r|| ~ 1 the two agree;

* sufficient decrease as in the paper's Algorithm 1: f(x_trial) <
  f_max + gamma g^T (x_trial - x) on the arc, and f_max + gamma t g^T d at
  step t along the feasible direction;
* a first arc trial without descent (g^T (P(x - gstep g) - x) >= 0) at a
  point the exit tests did not certify: for x in the ball this happens only
  when the displacement is at the level of rounding -- the projection then
  mostly pulls x back onto the ball's surface, which x misses by the
  rounding of its l1 norm -- i.e. the Barzilai-Borwein step is too short
  for the working precision.  The iteration ends with x unchanged (which
  counts as stagnation for the tau update) and the next one restarts from
  the projected-gradient step 1 / ||P(x - g) - x||_inf, the solver's
  initial step; no fallback search or step-max damping (the fallback
  direction is that same rounding-level displacement).  With a fixed tau,
  three such iterations in a row end the solve as a line-search failure
  (no descent at the working precision);
* the fallback search starts at t = 1/2 (interpolated from the first arc
  trial): its t = 1 point is the first arc trial, already rejected by the
  same test;
* after a failed fallback search x, f and r are all restored;
* after the projection onto a smaller ball, r, f and g are recomputed at
  the projected x and the non-monotone history restarts from its f: values
  recorded on the larger ball can lie below every objective value the
  smaller ball attains, and a search against them cannot succeed (with a
  superoptimal warm start every search then failed until the line-error
  limit stopped the solve);
* a cold start has tau = 0 and x = 0; a warm start x0 has tau =
  ||x0||_1 unless tau0 is given.

Constants: memory 3, gamma 1e-4, step lengths clamped to [1e-16, 1e5],
opt_tol 1e-4, bp_tol = ls_tol = 1e-6, dec_tol 1e-4, max_line 10 (at most 11
trials per search), max_line_errors 10.

Parity pins (tests/test_oracle_spgl1.py): the l1 projection is pinned by its
optimality conditions and by an independent bisection; the solver with
sigma = 0 is pinned against a linear-programming solve of basis pursuit,
with sigma > 0 by the optimality certificate and an independent SLSQP
solve, and the fixed-tau LASSO solution by its duality gap and an
independent projected-gradient solve.  Exact iterate-by-iterate parity with
the GPU solver is NOT pinned: FP32 operator rounding can flip line-search
branches ("parity unpinned" for the iterate sequence; final-point parity is
pinned by the certificate).
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
EXIT_LEAST_SQUARES = 6
EXIT_SUBOPTIMAL_BP = 7
EXIT_OPTIMAL = 8


@dataclass
class Options:
    max_iter: int = 300
    opt_tol: float = 1e-4
    bp_tol: float = 1e-6
    ls_tol: float = 1e-6
    dec_tol: float = 1e-4
    memory: int = 3
    gamma: float = 1e-4
    step_min: float = 1e-16
    step_max: float = 1e5
    max_line: int = 10
    max_line_errors: int = 10


@dataclass
class Info:
    status: int = 0
    iterations: int = 0
    n_prod_A: int = 0
    n_prod_At: int = 0
    n_newton: int = 0
    n_line_errors: int = 0
    n_safeguard: int = 0
    n_stationary: int = 0
    tau: float = 0.0
    rnorm: float = 0.0
    xnorm1: float = 0.0
    rel_gap: float = 0.0
    history: list = field(default_factory=list)


def _clamp_step(v, o, step_max):
    return min(step_max, max(o.step_min, v))


def spgl1(A, At, b, sigma, x0=None, tau0=None, opts: Options | None = None, single_tau=False):
    """Solve min ||x||_1 s.t. ||A x - b||_2 <= sigma (Pareto root finding), or,
    with ``single_tau``, the LASSO problem min ||A x - b||_2 s.t. ||x||_1 <=
    tau0 alone (sigma ignored).

    ``A`` and ``At`` are callables (real arrays in, real arrays out).  Returns
    (x, Info).  ``x0`` warm-starts the iterate; ``tau0`` defaults to 0 for a
    cold start and to ||x0||_1 for a warm start.
    """
    o = opts or Options()
    info = Info()
    b = np.asarray(b, dtype=np.float64)
    bnorm = float(np.linalg.norm(b))
    if single_tau:
        if tau0 is None:
            raise ValueError("a single-tau (LASSO) solve needs tau0")
        sigma = 0.0

    def Ax(x):
        info.n_prod_A += 1
        return A(x)

    def Atr(r):
        info.n_prod_At += 1
        return At(r)

    def f_of(r):
        return 0.5 * float(r.ravel() @ r.ravel())

    if x0 is None:
        x = np.zeros(Atr(b).shape)
        info.n_prod_At -= 1  # shape query only
        tau = 0.0 if tau0 is None else float(tau0)
    else:
        x = np.asarray(x0, dtype=np.float64)
        tau = float(np.abs(x).sum()) if tau0 is None else float(tau0)
    step_max = o.step_max
    line_errors_left = o.max_line_errors

    x = project_l1(x, tau)
    r = b - Ax(x)
    g = -Atr(r)
    f = f_of(r)
    fhist = [-np.inf] * o.memory
    fhist[0] = f
    f_old = f
    dx = project_l1(x - g, tau) - x
    dxn = float(np.abs(dx).max()) if dx.size else 0.0
    gstep = step_max if dxn < 1.0 / step_max else _clamp_step(1.0 / dxn, o, step_max)

    it = 0
    n_nodescent = 0
    upd_last = False
    status = 0
    while True:
        # ---- exit tests and Newton update of tau (top of the iteration) ----
        gnorm = float(np.abs(g).max())
        rnorm = float(np.linalg.norm(r))
        gap = float(r.ravel() @ (r - b).ravel()) + tau * gnorm
        rel_gap = abs(gap) / max(1.0, f)
        aerr1 = rnorm - sigma
        rerr1 = abs(aerr1) / max(1.0, bnorm)
        rerr2 = abs(f - 0.5 * sigma ** 2) / max(1.0, f)
        info.history.append((it, tau, rnorm, rel_gap))
        if single_tau:
            if rel_gap <= o.opt_tol or rnorm < o.opt_tol * bnorm:
                status = EXIT_OPTIMAL
        else:
            if gnorm <= o.ls_tol * rnorm:
                status = EXIT_LEAST_SQUARES
            if rel_gap <= max(o.opt_tol, rerr2) or rerr1 <= o.opt_tol:
                if rnorm <= sigma:
                    status = EXIT_SUBOPTIMAL_BP
                if rerr1 <= o.opt_tol:
                    status = EXIT_ROOT_FOUND
                if rnorm <= o.bp_tol * bnorm:
                    status = EXIT_BP_FOUND
            change = abs(f - f_old)
            near = 0.1 * abs(rnorm - sigma) / max(rnorm, 1e-300)
            stagnant = (change <= o.dec_tol * f and rnorm > 2 * sigma) or (change <= near * f and rnorm <= 2 * sigma)
            upd = stagnant and not status and not upd_last
            upd_last = upd
            if upd:
                tau_old = tau
                tau = max(0.0, tau + rnorm * aerr1 / gnorm)
                info.n_newton += 1
                shrink = tau < tau_old
                if shrink:
                    # the ball shrank: x is projected onto it, and the
                    # residual, objective, gradient and the non-monotone
                    # history restart at the projected point (objective
                    # values recorded on the larger ball are below what the
                    # smaller one can attain)
                    x = project_l1(x, tau)
                    r = b - Ax(x)
                    g = -Atr(r)
                    f = f_of(r)
                    fhist = [-np.inf] * o.memory
                    fhist[0] = f
        if not status and it >= o.max_iter:
            status = EXIT_ITERATIONS
        if status:
            break

        # ---- one spectral projected-gradient iteration ----
        it += 1
        x_old, f_old, g_old, r_old = x, f, g, r
        fmax = max(fhist)
        # non-monotone search along the projection arc
        step, scale, n_safe, sn = 1.0, 1.0, 0, 0.0
        gn = float(np.linalg.norm(g))
        accepted = stationary = False
        d1 = f1 = gtd1 = None
        for trial in range(o.max_line + 1):
            xt = project_l1(x - step * scale * gstep * g, tau)
            rt = b - Ax(xt)
            ft = f_of(rt)
            s = (xt - x).ravel()
            gts = float(g.ravel() @ s)
            if trial == 0:
                d1, f1, gtd1 = s.reshape(x.shape), ft, gts
            if gts >= 0:
                stationary = trial == 0
                break
            if ft < fmax + o.gamma * gts:
                accepted = True
                break
            step *= 0.5
            sn_old, sn = sn, float(np.linalg.norm(s))
            if abs(sn - sn_old) <= 1e-6 * sn and gn > 0:
                # flat arc: rescale so that the next displacement is
                # step * |s| / 2^n_safe
                scale = sn / (gstep * gn) / 2.0 ** n_safe
                n_safe += 1
                info.n_safeguard += 1
        if not accepted and not stationary:
            # feasible-direction search along d1 (its t = 1 point is the
            # first arc trial, already rejected)
            t, fnew = 1.0, f1
            for _ in range(o.max_line):
                if t <= 0.1:
                    t *= 0.5
                else:
                    den = 2.0 * (fnew - f - t * gtd1)
                    tmp = (-gtd1 * t * t) / den if den != 0 else np.nan
                    t = tmp if (np.isfinite(tmp) and 0.1 <= tmp <= 0.9 * t) else 0.5 * t
                xt = x + t * d1
                rt = b - Ax(xt)
                fnew = ft = f_of(rt)
                if ft < fmax + o.gamma * t * gtd1:
                    accepted = True
                    break
        if not stationary:
            n_nodescent = 0
        if accepted:
            x, r, f = xt, rt, ft
            g = -Atr(r)
            s = (x - x_old).ravel()
            yv = (g - g_old).ravel()
            sts, sty = float(s @ s), float(s @ yv)
            gstep = step_max if sty <= 0 else _clamp_step(sts / sty, o, step_max)
        elif stationary:
            # the projected-gradient step from the BB length does not move x
            # downhill.  Unless the duality gap already certifies x (the exit
            # tests would have stopped), the step is too short for the
            # working precision: the next iteration restarts from the
            # projected-gradient step length 1 / ||P(x - g) - x||_inf, the
            # solver's initial step.  x is unchanged, which registers as
            # stagnation of f for the tau update.
            n_nodescent += 1
            info.n_stationary += 1
            if single_tau and n_nodescent > 2:
                status = EXIT_LINE_ERROR
                break
            dx = project_l1(x - g, tau) - x
            dxn = float(np.abs(dx).max()) if dx.size else 0.0
            gstep = step_max if dxn < 1.0 / step_max else _clamp_step(1.0 / dxn, o, step_max)
        else:
            x, f, g, r = x_old, f_old, g_old, r_old
            info.n_line_errors += 1
            if line_errors_left <= 0:
                status = EXIT_LINE_ERROR
                break
            step_max /= 10.0
            line_errors_left -= 1
            gstep = min(step_max, gstep)
        if single_tau or f > 0.5 * sigma ** 2:
            fhist[it % o.memory] = f

    info.status = status
    info.iterations = it
    info.tau = tau
    info.rnorm = float(np.linalg.norm(r))
    info.xnorm1 = float(np.abs(x).sum())
    gnorm = float(np.abs(g).max())
    gap = float(r.ravel() @ (r - b).ravel()) + tau * gnorm
    info.rel_gap = abs(gap) / max(1.0, 0.5 * info.rnorm ** 2)
    return x, info


def lasso(A, At, b, tau, x0=None, opts: Options | None = None):
    """The LASSO problem min ||A x - b||_2 s.t. ||x||_1 <= tau by the same
    spectral projected gradient (SPGL1 with a single fixed tau)."""
    return spgl1(A, At, b, 0.0, x0=x0, tau0=tau, opts=opts, single_tau=True)
