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


def test_step_restart_readings_reach_the_same_root():
    """Both step-length readings (restart from the projected gradient after a
    Newton update of tau, or keep the Barzilai-Borwein step) satisfy the root
    certificate and agree on ||x||_1 to the inexactness of the Newton method
    (opt_tol 1e-6 here)."""
    A, bf, sigma = _bpdn_problem()
    op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
    res = []
    for restart in (True, False):
        x, info = spgl1.spgl1(op, opT, bf, sigma, opts=spgl1.Options(opt_tol=1e-6, restart_step=restart))
        assert info.status == spgl1.EXIT_ROOT_FOUND
        assert abs(info.rnorm - sigma) <= 1e-6 * max(1.0, np.linalg.norm(bf))
        res.append(np.abs(x).sum())
    assert abs(res[0] - res[1]) <= 1e-3 * res[0]


def test_tau0_at_the_root_saves_iterations():
    """Starting from x = 0 with tau0 = the final radius skips the Newton
    steps of the cold start: fewer iterations, the same root."""
    A, bf, sigma = _bpdn_problem()
    op, opT = (lambda v: A @ v), (lambda r: A.T @ r)
    x, info = spgl1.spgl1(op, opT, bf, sigma)
    x2, info2 = spgl1.spgl1(op, opT, bf, sigma, tau0=info.tau)
    assert info2.status == spgl1.EXIT_ROOT_FOUND
    assert info2.iterations < info.iterations
    assert abs(info2.xnorm1 - info.xnorm1) <= 1e-3 * info.xnorm1
