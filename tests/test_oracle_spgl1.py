"""Pins of the SPGL1 oracle: l1-ball projection and basis-pursuit solutions."""
import numpy as np
import pytest
from scipy.optimize import NonlinearConstraint, linprog, minimize

from oracle import nufft, ring, spgl1


def test_project_l1_kkt_and_bisection():
    rng = np.random.default_rng(0)
    for n, tau in [(10, 1.0), (200, 5.0), (1000, 0.3)]:
        v = rng.standard_normal(n) * 2
        x = spgl1.project_l1(v, tau)
        assert abs(np.abs(x).sum() - tau) < 1e-10
        # KKT: v - x = theta sign(x) on the support, |v| <= theta off it
        sup = x != 0
        theta = (v - x)[sup] * np.sign(x[sup])
        assert np.ptp(theta) < 1e-10 and theta.min() > 0
        assert np.all(np.abs(v[~sup]) <= theta[0] + 1e-12)
        np.testing.assert_allclose(x, spgl1.project_l1_bisect(v, tau), atol=1e-10)
        # variational inequality <v - x, z - x> <= 0 for feasible z
        for _ in range(20):
            z = rng.standard_normal(n)
            z *= tau / np.abs(z).sum() * rng.uniform()
            assert (v - x) @ (z - x) <= 1e-10
    # inside the ball: identity
    v = np.array([0.1, -0.2])
    np.testing.assert_array_equal(spgl1.project_l1(v, 1.0), v)


def _dense_radon(n, ns, m):
    th = nufft.default_angles(m)
    E = np.eye(n * n)
    return np.stack([nufft.radon_exact(E[i].reshape(n, n), ns, th).ravel() for i in range(n * n)], axis=1)


def _bp_lp(A, b, weights=None):
    """min sum_i w_i |x_i| s.t. A x = b as an LP in (x, t): min w.t, -t <= x <= t."""
    m, n = A.shape
    c = np.concatenate([np.zeros(n), np.ones(n) if weights is None else weights])
    I = np.eye(n)
    A_ub = np.block([[I, -I], [-I, -I]])
    b_ub = np.zeros(2 * n)
    A_eq = np.hstack([A, np.zeros((m, n))])
    res = linprog(c, A_ub=A_ub, b_ub=b_ub, A_eq=A_eq, b_eq=b, bounds=[(None, None)] * n + [(0, None)] * n,
                  method="highs")
    assert res.status == 0
    return res.x[:n], res.fun


def test_basis_pursuit_matches_lp():
    n, ns, m = 16, 16, 8
    R = _dense_radon(n, ns, m)
    rng = np.random.default_rng(3)
    x_true = np.zeros(n * n)
    idx = rng.choice(n * n, size=12, replace=False)
    x_true[idx] = rng.standard_normal(12)
    b = R @ x_true
    x_lp, obj = _bp_lp(R, b)
    opts = spgl1.Options(max_iter=20000, opt_tol=1e-9, bp_tol=1e-9)
    x, info = spgl1.spgl1(lambda v: R @ v, lambda r: R.T @ r, b, 0.0, opts=opts)
    assert info.status in (spgl1.EXIT_ROOT_FOUND, spgl1.EXIT_BP_FOUND), info.status
    assert abs(np.abs(x).sum() - obj) / obj < 1e-6
    assert np.linalg.norm(R @ x - b) / np.linalg.norm(b) < 1e-6
    # uniqueness of the LP optimum: re-solve with a slightly perturbed cost;
    # an isolated vertex does not move
    x_lp2, _ = _bp_lp(R, b, 1.0 + 1e-7 * rng.uniform(size=n * n))
    assert np.linalg.norm(x_lp - x_lp2) < 1e-8 * np.linalg.norm(x_lp)
    assert np.linalg.norm(x - x_lp) / np.linalg.norm(x_lp) < 1e-6


def test_bpdn_certificate_with_ring_filter():
    n, ns, m = 16, 16, 12
    R = _dense_radon(n, ns, m)
    F = ring.ring_filter_matrix(m, ns)
    A = F @ R
    rng = np.random.default_rng(4)
    x_true = np.zeros(n * n)
    x_true[rng.choice(n * n, size=10, replace=False)] = 1.0
    y = R @ x_true
    noise = 0.01 * np.abs(y).max()
    b = y + rng.normal(0, noise, y.shape)
    b = b.reshape(m, ns)
    b[:, 3] += 0.5  # stuck column
    bf = F @ b.ravel()
    sigma = noise * np.sqrt(m * ns - ns + 4)
    x, info = spgl1.spgl1(lambda v: A @ v, lambda r: A.T @ r, bf, sigma)
    assert info.status == spgl1.EXIT_ROOT_FOUND
    assert abs(info.rnorm - sigma) <= 1e-4 * max(1.0, np.linalg.norm(bf))
    # the misfit is measured after the filter: the stuck column does not enter
    r = np.linalg.norm(F @ (R @ x) - bf)
    assert abs(r - sigma) <= 1e-4 * np.linalg.norm(bf)
    assert abs(np.abs(x).sum() - info.tau) <= 1e-6 * info.tau + 1e-12
    # independent optimum: the same problem as a smooth program in (x+, x-)
    # >= 0 with one quadratic constraint, solved by SLSQP from the
    # minimum-norm least-squares point
    N = n * n
    M = np.hstack([A, -A])
    x_ls = np.linalg.lstsq(A, bf, rcond=None)[0]
    z0 = np.concatenate([np.maximum(x_ls, 0), np.maximum(-x_ls, 0)])
    cons = NonlinearConstraint(lambda z: sigma ** 2 - np.sum((M @ z - bf) ** 2), 0, np.inf,
                               jac=lambda z: (-2 * (M.T @ (M @ z - bf)))[None, :])
    res = minimize(lambda z: z.sum(), z0, jac=lambda z: np.ones_like(z), bounds=[(0, None)] * (2 * N),
                   constraints=[cons], method="SLSQP", options=dict(maxiter=3000, ftol=1e-12))
    assert np.sum((M @ res.x - bf) ** 2) ** 0.5 <= sigma * (1 + 1e-6)
    assert abs(np.abs(x).sum() - res.fun) <= 1e-3 * res.fun, (np.abs(x).sum(), res.fun)


def _bpdn_problem(seed=4):
    n, ns, m = 16, 16, 12
    R = _dense_radon(n, ns, m)
    F = ring.ring_filter_matrix(m, ns)
    A = F @ R
    rng = np.random.default_rng(seed)
    x_true = np.zeros(n * n)
    x_true[rng.choice(n * n, size=10, replace=False)] = 1.0
    y = R @ x_true
    noise = 0.01 * np.abs(y).max()
    b = (y + rng.normal(0, noise, y.shape)).reshape(m, ns)
    b[:, 3] += 0.5
    bf = F @ b.ravel()
    sigma = noise * np.sqrt(m * ns - ns + 4)
    return A, bf, sigma


def test_warm_start_at_the_solution_stays_there():
    """Started at its own solution (tau0 = its l1 norm), the solver finds the
    root at once and does not move the point."""
    A, bf, sigma = _bpdn_problem()
    op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
    x, info = spgl1.spgl1(op, opT, bf, sigma)
    assert info.status == spgl1.EXIT_ROOT_FOUND
    x2, info2 = spgl1.spgl1(op, opT, bf, sigma, x0=x)
    assert info2.status == spgl1.EXIT_ROOT_FOUND
    assert info2.iterations <= 3
    assert np.linalg.norm(x2 - x) <= 1e-3 * np.linalg.norm(x)


def test_lasso_fixed_tau_matches_independent_qp():
    """With a single fixed tau the solver returns the LASSO solution
    min ||A x - b|| s.t. ||x||_1 <= tau: checked against the same problem as a
    smooth program in (x+, x-) >= 0 solved by SLSQP, and by its duality gap."""
    A, bf, sigma = _bpdn_problem()
    op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
    x_bp, info_bp = spgl1.spgl1(op, opT, bf, sigma)
    tau = 0.8 * info_bp.tau  # strictly inside the Pareto curve's root
    # the gap certifies x to first order while f is resolved to FP64 rounding
    # (second order): a relative gap of 1e-7 is within reach, 1e-10 is not
    x, info = spgl1.lasso(op, opT, bf, tau, opts=spgl1.Options(opt_tol=1e-7, max_iter=20000))
    assert info.status == spgl1.EXIT_OPTIMAL, info.status
    assert abs(np.abs(x).sum() - tau) <= 1e-9 * tau
    N = A.shape[1]
    M = np.hstack([A, -A])
    res = minimize(lambda z: 0.5 * np.sum((M @ z - bf) ** 2), np.full(2 * N, tau / (2 * N)),
                   jac=lambda z: M.T @ (M @ z - bf), bounds=[(0, None)] * (2 * N),
                   constraints=[{"type": "ineq", "fun": lambda z: tau - z.sum(), "jac": lambda z: -np.ones_like(z)}],
                   method="SLSQP", options=dict(maxiter=5000, ftol=1e-14))
    x_qp = res.x[:N] - res.x[N:]
    f_sp = 0.5 * np.sum((A @ x - bf) ** 2)
    f_qp = 0.5 * np.sum((A @ x_qp - bf) ** 2)
    assert f_sp <= f_qp * (1 + 1e-9)
    assert np.linalg.norm(x - x_qp) <= 1e-3 * np.linalg.norm(x_qp), np.linalg.norm(x - x_qp) / np.linalg.norm(x_qp)
    # duality gap of the returned point
    r = bf - A @ x
    gap = r @ (r - bf) + tau * np.abs(A.T @ r).max()
    assert abs(gap) <= 1e-7 * max(1.0, 0.5 * r @ r)


def test_flat_arc_safeguard_rescales_the_step():
    """A Barzilai-Borwein step far too long for the ball makes consecutive
    arc trials project to the same point; the safeguard then shrinks the
    displacement geometrically, and the search still finds a decrease."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((30, 60))
    b = rng.standard_normal(30)
    op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
    x, info = spgl1.lasso(op, opT, b, 0.5, opts=spgl1.Options(opt_tol=1e-7, max_iter=5000, step_min=1e5))
    # step_min = step_max: every iteration starts at a step of 1e5
    assert info.status == spgl1.EXIT_OPTIMAL, info.status
    assert info.n_safeguard > 0
    x_ref, _ = spgl1.lasso(op, opT, b, 0.5, opts=spgl1.Options(opt_tol=1e-7, max_iter=5000))
    assert np.linalg.norm(x - x_ref) <= 1e-4 * np.linalg.norm(x_ref)


def test_warm_start_near_the_solution_saves_iterations():
    """A warm start close to the solution (x* plus 1% noise, projected onto the
    ball of the final radius, tau = its l1 norm) reaches the same root in
    fewer iterations than the cold start; so does the superoptimal start x*
    plus noise without the projection (tau above the root)."""
    for seed in (4, 5, 6):
        A, bf, sigma = _bpdn_problem(seed)
        op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
        x, info = spgl1.spgl1(op, opT, bf, sigma)
        rng = np.random.default_rng(12)
        xn = x + 0.01 * np.linalg.norm(x) / np.sqrt(x.size) * rng.standard_normal(x.size)
        for x0 in (spgl1.project_l1(xn, info.tau), xn):
            x2, info2 = spgl1.spgl1(op, opT, bf, sigma, x0=x0)
            assert info2.status == spgl1.EXIT_ROOT_FOUND
            assert info2.n_line_errors == 0
            assert info2.iterations < info.iterations
            assert abs(info2.xnorm1 - info.xnorm1) <= 1e-3 * info.xnorm1


@pytest.mark.parametrize("mistake", ["theta_next_rho", "no_clip", "unsigned", "scaled"])
def test_planted_projection_mistakes_fail_the_pin(monkeypatch, mistake):
    """A plausible mistake planted in the l1-ball projection (on the CPU)
    fails the optimality pin above: the threshold taken with one term too
    many, soft thresholding without the clip at zero, the signs dropped,
    and a rescaling of v onto the sphere instead of a projection."""
    right = spgl1.project_l1

    def wrong(v, tau):
        v = np.asarray(v, dtype=np.float64)
        if np.abs(v).sum() <= tau:
            return v.copy()
        u = np.sort(np.abs(v))[::-1]
        cs = np.cumsum(u)
        j = np.arange(1, u.size + 1)
        rho = int(np.nonzero(u > (cs - tau) / j)[0][-1])
        if mistake == "theta_next_rho":
            rho = min(rho + 1, u.size - 1)
        theta = (cs[rho] - tau) / (rho + 1)
        if mistake == "no_clip":
            return np.sign(v) * (np.abs(v) - theta)
        if mistake == "unsigned":
            return np.maximum(np.abs(v) - theta, 0.0)
        if mistake == "scaled":
            return v * tau / np.abs(v).sum()
        return np.sign(v) * np.maximum(np.abs(v) - theta, 0.0)

    monkeypatch.setattr(spgl1, "project_l1", wrong)
    with pytest.raises(AssertionError):
        test_project_l1_kkt_and_bisection()
    monkeypatch.setattr(spgl1, "project_l1", right)
    test_project_l1_kkt_and_bisection()
