"""Pins for the oracle's objective, gradient and optimisers (Sec. 2, Eqs. 5-6, 10-11).

The quadratic special case (p = q = 2) makes the whole problem linear; its minimiser
is then the solution of a dense linear system built here from the explicit
non-uniform DFT matrix and the graph Laplacian of the neighbour weights, solved by
numpy.linalg.solve.
"""
import itertools

import numpy as np

import synth
from test_oracle_radon import nudft_forward


def small_problem(orc, N=10, nd=12, na=7, S=1, seed=21):
    rng = np.random.default_rng(seed)
    th = synth.angles(na)
    x_true = rng.uniform(0, 1, (S, N, N))
    g = np.stack([orc.forward(s, th, nd) for s in x_true]) + rng.normal(0, 0.05, (S, na, nd))
    K = orc.kernel(N, th, nd)
    atg = orc.adjoint(g, N, th)
    return th, g, K, atg, float(np.sum(g * g))


def test_toeplitz_objective_equals_eq5(orc):
    pr = orc.Prior()
    th, g, K, atg, gtg = small_problem(orc, S=2)
    rng = np.random.default_rng(22)
    for _ in range(3):
        x = rng.normal(0.5, 0.2, atg.shape)
        assert abs(orc.objective(x, atg, gtg, K, pr) - orc.objective_direct(x, g, th, pr)) < 1e-10 * orc.objective_direct(x, g, th, pr)


def test_gradient_is_derivative_of_eq5(orc):
    pr = orc.Prior()
    th, g, K, atg, gtg = small_problem(orc, S=2)
    x = np.random.default_rng(23).normal(0.5, 0.2, atg.shape)
    G = orc.gradient(x, atg, K, pr)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 4, 7), (0, 9, 3), (1, 5, 5)]:
        xp = x.copy()
        xp[idx] += h
        xm = x.copy()
        xm[idx] -= h
        fd = (orc.objective_direct(xp, g, th, pr) - orc.objective_direct(xm, g, th, pr)) / (2 * h)
        assert abs(G[idx] - fd) < 1e-5 * max(1.0, abs(fd))


def test_power_iteration_bounds_largest_eigenvalue(orc):
    N, nd = 8, 10
    th = synth.angles(9)
    K = orc.kernel(N, th, nd)
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    lmax = np.linalg.eigvalsh(A.T @ A).max()
    est = orc.power_lambda_max(K, N)
    assert est <= lmax * (1 + 1e-12) and est >= 0.995 * lmax


def gaussian_mrf_laplacian(orc, S, N):
    """Hessian of Phi for p = q = 2 (rho = D^2 / (2 sigma^2)) times sigma^2: weighted graph Laplacian."""
    n = S * N * N
    H = np.zeros((n, n))
    idx = lambda z, r, c: (z * N + r) * N + c
    for z, r, c in itertools.product(range(S), range(N), range(N)):
        for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
            if (dz, dy, dx) == (0, 0, 0):
                continue
            z2, r2, c2 = z + dz, r + dy, c + dx
            if 0 <= z2 < S and 0 <= r2 < N and 0 <= c2 < N:
                b = orc.neighbour_weight(dz, dy, dx)
                H[idx(z, r, c), idx(z, r, c)] += b
                H[idx(z, r, c), idx(z2, r2, c2)] -= b
    return H


def test_quadratic_case_reaches_linear_solve(orc):
    S, N, nd, na = 2, 6, 8, 5
    pr = orc.Prior(p=2.0, q=2.0, sigma=0.5, lam=0.3)
    rng = np.random.default_rng(24)
    th = synth.angles(na)
    g = rng.uniform(0, 1, (S, na, nd))
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    H = np.kron(np.eye(S), A.T @ A) + pr.lam / pr.sigma ** 2 * gaussian_mrf_laplacian(orc, S, N)
    rhs = np.concatenate([A.T @ g[s].ravel() for s in range(S)])
    x_star = np.linalg.solve(H, rhs).reshape(S, N, N)
    K = orc.kernel(N, th, nd)
    atg = orc.adjoint(g, N, th)
    L = orc.lipschitz(K, N, pr)
    x = orc.nesterov(np.zeros((S, N, N)), atg, float(np.sum(g * g)), K, pr, L, 3000)
    assert np.linalg.norm(x - x_star) < 1e-6 * np.linalg.norm(x_star)
    xg = orc.gradient_descent(np.zeros((S, N, N)), atg, K, pr, L, 200)
    # plain descent is slower than the accelerated method from the same start
    assert np.linalg.norm(xg - x_star) > np.linalg.norm(orc.nesterov(np.zeros((S, N, N)), atg, float(np.sum(g * g)), K, pr, L, 200) - x_star)


def test_projected_method_reaches_the_bounded_least_squares_solution(orc):
    # the quadratic case again, with data whose unconstrained minimiser has negative entries:
    # the projected fast gradient method (x_{k+1} = max(y - G/L, 0)) reaches the minimiser over
    # x >= 0, computed independently by non-negative least squares on a Cholesky factor of the
    # dense system (|| R x - d ||^2 = x.H x - 2 rhs.x + const with H = R^T R, R^T d = rhs)
    from scipy.linalg import cholesky, solve_triangular
    from scipy.optimize import nnls

    S, N, nd, na = 2, 6, 8, 5
    pr = orc.Prior(p=2.0, q=2.0, sigma=0.5, lam=0.3)
    rng = np.random.default_rng(25)
    th = synth.angles(na)
    g = rng.uniform(-1, 1, (S, na, nd))
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    H = np.kron(np.eye(S), A.T @ A) + pr.lam / pr.sigma ** 2 * gaussian_mrf_laplacian(orc, S, N)
    rhs = np.concatenate([A.T @ g[s].ravel() for s in range(S)])
    assert np.min(np.linalg.solve(H, rhs)) < -1e-2  # the bound is active
    R = cholesky(H)  # upper: H = R^T R
    x_star, _ = nnls(R, solve_triangular(R, rhs, trans="T"), maxiter=10000)
    x_star = x_star.reshape(S, N, N)
    K = orc.kernel(N, th, nd)
    atg = orc.adjoint(g, N, th)
    L = orc.lipschitz(K, N, pr)
    x = orc.nesterov(np.zeros((S, N, N)), atg, float(np.sum(g * g)), K, pr, L, 5000, nonneg=True)
    assert np.min(x) >= 0.0
    assert np.linalg.norm(x - x_star) < 1e-6 * np.linalg.norm(x_star)


def test_descent_is_monotone_and_nesterov_reaches_same_minimum(orc):
    pr = orc.Prior()
    th, g, K, atg, gtg = small_problem(orc, N=10, S=2)
    N = 10
    L = orc.lipschitz(K, N, pr)
    x = np.zeros_like(atg)
    F = [orc.objective(x, atg, gtg, K, pr)]
    for _ in range(30):
        x = orc.gradient_descent(x, atg, K, pr, L, 1)
        F.append(orc.objective(x, atg, gtg, K, pr))
    assert all(b <= a + 1e-12 * abs(a) for a, b in zip(F, F[1:]))
    xa = orc.nesterov(np.zeros_like(atg), atg, gtg, K, pr, L, 4000)
    xb = orc.gradient_descent(xa, atg, K, pr, L, 2000)
    Fa, Fb = orc.objective(xa, atg, gtg, K, pr), orc.objective(xb, atg, gtg, K, pr)
    assert Fa - Fb < 1e-8 * abs(Fb)


def test_restart_log(orc):
    pr = orc.Prior()
    th, g, K, atg, gtg = small_problem(orc, N=10, S=1)
    L = orc.lipschitz(K, 10, pr)
    log = []
    orc.nesterov(np.zeros_like(atg), atg, gtg, K, pr, L, 60, log=log)
    assert len(log) == 60
    # F(y_0) at y_0 = x_0 = 0 is 1/2 g.g
    assert abs(log[0][0] - 0.5 * gtg) < 1e-12 * gtg
    assert all((d > 0) == r for _, d, r in log)
    assert log[-1][0] < 0.5 * log[0][0]


def test_restart_modes(orc):
    # every restart mode reaches the minimiser of the quadratic case (a dense linear solve)
    S, N, nd, na = 1, 6, 8, 5
    pr = orc.Prior(p=2.0, q=2.0, sigma=0.5, lam=0.3)
    rng = np.random.default_rng(25)
    th = synth.angles(na)
    g = rng.uniform(0, 1, (S, na, nd))
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    H = A.T @ A + pr.lam / pr.sigma ** 2 * gaussian_mrf_laplacian(orc, S, N)
    x_star = np.linalg.solve(H, A.T @ g[0].ravel()).reshape(S, N, N)
    K = orc.kernel(N, th, nd)
    atg = orc.adjoint(g, N, th)
    L = orc.lipschitz(K, N, pr)
    gtg = float(np.sum(g * g))
    logs = {}
    for mode in ("gradient", "function", "none"):
        logs[mode] = []
        x = orc.nesterov(np.zeros((S, N, N)), atg, gtg, K, pr, L, 3000, log=logs[mode], restart=mode)
        assert np.linalg.norm(x - x_star) < 1e-6 * np.linalg.norm(x_star), mode
    # the function test restarts exactly when the objective at y went up
    lf = logs["function"]
    assert all(r == (k > 0 and lf[k][0] > lf[k - 1][0]) for k, (_, _, r) in enumerate(lf))
    assert not any(r for _, _, r in logs["none"])
    # without restart the first steps are the plain accelerated sequence, so all modes agree
    # until the first restart of a mode
    first = min(k for k, (_, _, r) in enumerate(logs["gradient"]) if r)
    assert all(abs(a[0] - b[0]) <= 1e-12 * abs(b[0]) for a, b in zip(logs["gradient"][:first + 1], logs["none"][:first + 1]))


def test_accelerated_rate_without_restart(orc):
    # the fast gradient method's guarantee (Nesterov; Beck and Teboulle's bound): without restart
    # F(x_k) - F* <= 2 L |x_0 - x*|^2 / (k + 1)^2 on the quadratic case, whose minimiser x* is a
    # dense linear solve; a broken momentum sequence loses this rate
    S, N, nd, na = 1, 6, 8, 5
    pr = orc.Prior(p=2.0, q=2.0, sigma=0.5, lam=0.3)
    rng = np.random.default_rng(26)
    th = synth.angles(na)
    g = rng.uniform(0, 1, (S, na, nd))
    A = np.stack([nudft_forward(e.reshape(N, N), th, nd).ravel() for e in np.eye(N * N)], axis=1)
    H = A.T @ A + pr.lam / pr.sigma ** 2 * gaussian_mrf_laplacian(orc, S, N)
    x_star = np.linalg.solve(H, A.T @ g[0].ravel()).reshape(S, N, N)
    K = orc.kernel(N, th, nd)
    atg = orc.adjoint(g, N, th)
    gtg = float(np.sum(g * g))
    L = orc.lipschitz(K, N, pr)
    F_star = orc.objective(x_star, atg, gtg, K, pr)
    x0 = np.zeros((S, N, N))
    r0 = float(np.sum((x0 - x_star) ** 2))
    for k in (1, 2, 3, 5, 8, 13, 21, 34, 55):
        xk = orc.nesterov(x0, atg, gtg, K, pr, L, k, restart="none")
        gap = orc.objective(xk, atg, gtg, K, pr) - F_star
        assert -1e-9 * abs(F_star) <= gap <= 2 * L * r0 / (k + 1) ** 2, k
