"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these compare the oracle with itself: each checks a closed form, an
eigen-relation of the discrete operator, an explicitly assembled matrix, the
exact solution of the all-at-once system, a hand-derived iterate set, or a
structural property (finite termination, parareal exactness).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import (OracleProblem, block_dot, chebyshev_ie_propagator, dense_rk4_propagator_matrix,
                    implicit_euler_propagator, matrix_propagator, norm_N_inf, parareal, pitsbicg,
                    rk4_propagator, rk4_step_matrix, spatial_operator)
from paper_2203_10148_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- steppers

@pytest.mark.parametrize("a,dT,m", [(-2.0, 0.3, 7), (-0.5, 1.0, 100), (1.3, 0.1, 3)])
def test_ie_scalar_closed_form(a, dT, m):
    """m implicit-Euler steps of y' = a y: factor (1 - a dT/m)^{-m}."""
    F = implicit_euler_propagator(np.array([[a]]), dT, m)
    got = F(np.array([[1.0]]))[0, 0]
    assert got == pytest.approx((1.0 - a * dT / m) ** (-m), rel=1e-14)


@pytest.mark.parametrize("a,dT,m", [(-2.0, 0.3, 7), (-40.0, 0.05, 3), (0.7, 1.0, 200)])
def test_rk4_scalar_closed_form(a, dT, m):
    """m RK4 steps of y' = a y: factor (1 + z + z^2/2 + z^3/6 + z^4/24)^m, z = a dT/m."""
    z = a * dT / m
    expect = (1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24) ** m
    F = rk4_propagator(np.array([[a]]), dT, m)
    assert F(np.array([[1.0]]))[0, 0] == pytest.approx(expect, rel=1e-13)
    Phi = dense_rk4_propagator_matrix(np.array([[a]]), dT, m)
    assert Phi[0, 0] == pytest.approx(expect, rel=1e-13)


def _mu(k, n):
    h = 1.0 / (n + 1)
    return -4.0 / (h * h) * math.sin(k * math.pi * h / 2.0) ** 2


def test_heat1d_sine_modes_are_eigenvectors():
    """sin(k pi x_j) is an eigenvector of D2 with mu_k = -(4/h^2) sin^2(k pi h/2)."""
    M, nu = 63, 0.1
    L = spatial_operator("heat1d", M, 1, nu)
    x = np.arange(1, M + 1) / (M + 1.0)
    for k in (1, 3, 17, 63):
        v = np.sin(k * math.pi * x)
        np.testing.assert_allclose(L @ v, nu * _mu(k, M) * v, rtol=0, atol=1e-10 * abs(nu * _mu(k, M)))


def test_heat1d_ie_trajectory_closed_form():
    """Noise-free heat1d workload: the fine trajectory is
    sum_k a_k (1 - dt nu mu_k)^{-m n} sin(k pi x)."""
    M, nu, T, N, m = 63, 0.1, 1.0, 16, 100
    x = np.arange(1, M + 1) / (M + 1.0)
    y0 = np.sin(math.pi * x) + 0.5 * np.sin(3 * math.pi * x)
    L = spatial_operator("heat1d", M, 1, nu)
    dT = T / N
    prob = OracleProblem(implicit_euler_propagator(L, dT, m), implicit_euler_propagator(L, dT, 1), y0, N)
    lam = prob.serial_fine()
    dt = dT / m
    for n in (0, 1, 5, 16):
        expect = sum(a * (1 - dt * nu * _mu(k, M)) ** (-m * n) * np.sin(k * math.pi * x)
                     for k, a in ((1, 1.0), (3, 0.5)))
        np.testing.assert_allclose(lam[n], expect, rtol=0, atol=1e-12)


def test_heat2d_rk4_sine_modes():
    """2D Dirichlet: sin(k pi x) sin(l pi y) is an eigenvector of the 5-point
    Laplacian with mu_k + mu_l; RK4 multiplies it by R(dt nu (mu_k + mu_l))^m,
    and one IE step divides it by 1 - dT nu (mu_k + mu_l)."""
    n, nu, dT, m = 12, 0.05, 0.01, 9
    L = spatial_operator("heat2d", n, n, nu)
    xs = np.arange(1, n + 1) / (n + 1.0)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    for (k, l) in ((1, 1), (2, 5), (12, 3)):
        v = (np.sin(k * math.pi * X) * np.sin(l * math.pi * Y)).reshape(-1)
        lam = nu * (_mu(k, n) + _mu(l, n))
        np.testing.assert_allclose(L @ v, lam * v, atol=1e-9 * abs(lam))
        z = lam * dT / m
        R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
        got = rk4_propagator(L, dT, m)(v[None, :])[0]
        np.testing.assert_allclose(got, R ** m * v, atol=1e-13)
        got = implicit_euler_propagator(L, dT, 1)(v[None, :])[0]
        np.testing.assert_allclose(got, v / (1 - dT * lam), atol=1e-13)


def test_heat2d_index_orientation():
    """x varies fastest (index j*nx + i): a mode with different x and y
    wavenumbers on a rectangular grid must use hx = 1/(nx+1) along i."""
    nx, ny, nu = 7, 5, 1.0
    L = spatial_operator("heat2d", nx, ny, nu)
    xs = np.arange(1, nx + 1) / (nx + 1.0)
    ys = np.arange(1, ny + 1) / (ny + 1.0)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    v = (np.sin(2 * math.pi * X) * np.sin(1 * math.pi * Y)).reshape(-1)
    lam = _mu(2, nx) + _mu(1, ny)
    np.testing.assert_allclose(L @ v, lam * v, atol=1e-10 * abs(lam))


@pytest.mark.parametrize("vx,vy", [(0.7, -0.3), (-0.4, 0.9)])
def test_advdiff_fourier_modes_constant_velocity(vx, vy):
    """Periodic grid, constant velocity: exp(2 pi i (kx x + ky y)) is an
    eigenvector; upwind differences give -(v/h)(1 - e^{-i theta}) for v >= 0
    and -(v/h)(e^{i theta} - 1) for v < 0; central diffusion gives
    nu (2 cos theta - 2)/h^2 per axis."""
    n, nu = 16, 0.01
    h = 1.0 / n
    L = spatial_operator("advdiff2d", n, n, nu, np.full(n * n, vx), np.full(n * n, vy))
    xs = np.arange(n) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    for kx, ky in ((1, 0), (3, -2), (-5, 7)):
        tx, ty = 2 * math.pi * kx * h, 2 * math.pi * ky * h
        e = np.exp(2j * math.pi * (kx * X + ky * Y)).reshape(-1)
        lam = nu * (2 * math.cos(tx) - 2 + 2 * math.cos(ty) - 2) / h ** 2
        lam -= vx * (1 - np.exp(-1j * tx)) / h if vx >= 0 else vx * (np.exp(1j * tx) - 1) / h
        lam -= vy * (1 - np.exp(-1j * ty)) / h if vy >= 0 else vy * (np.exp(1j * ty) - 1) / h
        np.testing.assert_allclose(L @ e, lam * e, atol=1e-9 * abs(lam))


def _chebyshev_T(K, z):
    """Chebyshev polynomial of the first kind, T_K(z) = cosh(K arccosh z),
    evaluated directly at a complex point (not by the three-term recurrence)."""
    return np.cosh(K * np.arccosh(complex(z)))


@pytest.mark.parametrize("vx,vy", [(0.6, 0.3), (-0.5, 0.8)])
@pytest.mark.parametrize("K", [1, 2, 5, 8, 13])
def test_chebyshev_ie_step_is_the_chebyshev_polynomial_on_fourier_modes(vx, vy, K):
    """Constant velocity on the periodic grid: the diagonal of I - dT L is one
    number D, every Fourier mode b is an eigenvector of I - dT L with
    eigenvalue mu (from the difference symbols), and the scaled eigenvalue is
    lambda = mu / D.  K steps of Chebyshev acceleration on [1 - rho, 1 + rho]
    from w = b leave the residual b - (I - dT L) w_K = P_K(lambda)(1 - mu) b
    with the residual polynomial P_K(lambda) = T_K((1 - lambda)/rho) / T_K(1/rho)
    (Saad, Sec. 12.3).  Modes up to the grid's Nyquist frequency, where the
    advection symbol puts lambda off the real interval."""
    n, nu, dT = 16, 0.02, 0.2
    h = 1.0 / n
    L = spatial_operator("advdiff2d", n, n, nu, np.full(n * n, vx), np.full(n * n, vy))
    D = 1.0 + dT * (4 * nu / h ** 2 + abs(vx) / h + abs(vy) / h)
    rho = (D - 1.0) / D
    assert 0.8 < rho < 0.95                 # the stiff regime of the 512^2 workload
    G = chebyshev_ie_propagator(L, dT, 1, K)
    xs = np.arange(n) / n
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    for kx, ky in ((0, 0), (1, 0), (2, -3), (4, 4), (-7, 5), (8, 8)):
        tx, ty = 2 * math.pi * kx * h, 2 * math.pi * ky * h
        b = np.exp(2j * math.pi * (kx * X + ky * Y)).reshape(-1)
        ell = nu * (2 * math.cos(tx) - 2 + 2 * math.cos(ty) - 2) / h ** 2
        ell -= vx * (1 - np.exp(-1j * tx)) / h if vx >= 0 else vx * (np.exp(1j * tx) - 1) / h
        ell -= vy * (1 - np.exp(-1j * ty)) / h if vy >= 0 else vy * (np.exp(1j * ty) - 1) / h
        mu = 1.0 - dT * ell
        lam = mu / D
        P = _chebyshev_T(K, (1.0 - lam) / rho) / _chebyshev_T(K, 1.0 / rho)
        w = G(b[None, :])[0]
        resid = b - (w - dT * (L @ w))
        np.testing.assert_allclose(resid, P * (1.0 - mu) * b, rtol=0,
                                   atol=1e-12 * max(1.0, abs(1.0 - mu)))


def test_chebyshev_ie_step_tends_to_the_implicit_euler_step():
    """With many steps the Chebyshev coarse step converges to the exact
    implicit-Euler step (sparse LU) on the variable-velocity workload field,
    in the regime of the 512^2 workload: diffusion-dominated (cell Peclet
    number |v| h / nu about 0.4, so the scaled spectrum hugs the real
    interval) and stiff (nu dT / h^2 about 2.6, rho about 0.9); K = 48, the
    workloads' count, solves the system to better than 1e-6.  With K = 8 it
    is still far from it on rough data, which is why the coarse step is
    defined by K."""
    w = inputs.advdiff2d(n=32, nu=0.08, N=1, T=0.0312)
    L = spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy)
    exact = implicit_euler_propagator(L, w.T, 1)
    b = inputs.SeededStream(5).normal(2 * w.M).reshape(2, w.M)
    b[1] = w.y0[0]
    ref = exact(b)
    got = chebyshev_ie_propagator(L, w.T, 1, 160)(b)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    rough8 = chebyshev_ie_propagator(L, w.T, 1, 8)(b[:1])
    assert np.abs(rough8 - ref[:1]).max() > 1e-3 * np.abs(ref[:1]).max()
    A = np.eye(w.M) - w.T * L.toarray()
    x48 = chebyshev_ie_propagator(L, w.T, 1, 48)(b)
    for j in range(2):
        assert np.linalg.norm(b[j] - A @ x48[j]) <= 1e-6 * np.linalg.norm(b[j])


def test_chebyshev_ie_step_with_one_step_is_scaled_richardson():
    """K = 1: w_1 = b + D^{-1}(b - (I - dT L) b) (theta = 1), a closed form."""
    w = inputs.advdiff2d(n=16, N=1, T=0.1)
    L = spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy)
    A = (np.eye(w.M) - w.T * L.toarray())
    b = w.y0[0]
    expect = b + (b - A @ b) / np.diag(A)
    np.testing.assert_allclose(chebyshev_ie_propagator(L, w.T, 1, 1)(b[None])[0], expect,
                               rtol=0, atol=1e-13 * np.abs(expect).max())


def test_advdiff_workload_coarse_step_is_the_chebyshev_step():
    """The advection-diffusion workloads name their coarse step's Chebyshev
    count, and the oracle problem applies that operator (K = 0: exact IE)."""
    w = inputs.advdiff2d(n=16, N=2, T=0.05)
    assert w.coarse_inner == 48
    L = spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy)
    b = w.y0
    np.testing.assert_array_equal(OracleProblem.from_workload(w).G(b),
                                  chebyshev_ie_propagator(L, w.dT, 1, 48)(b))
    w.coarse_inner = 0
    np.testing.assert_array_equal(OracleProblem.from_workload(w).G(b),
                                  implicit_euler_propagator(L, w.dT, 1)(b))


def test_advdiff_workload_energy_does_not_grow():
    """Divergence-free velocity, upwind advection and diffusion dissipate:
    the discrete L2 energy does not grow over a fine slice."""
    w = inputs.advdiff2d(n=32, N=8, T=0.5)
    prob = OracleProblem.from_workload(w)
    u = prob.y0
    for _ in range(4):
        v = prob.F(u[None, :])[0]
        assert np.linalg.norm(v) <= np.linalg.norm(u) * (1 + 1e-12)
        u = v


def test_dense_propagator_vs_stepping_and_expm():
    """Phi_F by binary powering equals explicit RK4 stepping (brute force) and
    approximates expm(dT A) within RK4's O(dt^4) error."""
    w = inputs.dense(M=24, N=8, T=1.0, fine_steps=37)
    A = w.A
    dT = w.T / w.N
    Phi = dense_rk4_propagator_matrix(A, dT, 37)
    V = inputs.SeededStream(5).normal(3 * 24).reshape(3, 24)
    stepped = rk4_propagator(A, dT, 37)(V)
    np.testing.assert_allclose(V @ Phi.T, stepped, rtol=0, atol=1e-13 * np.abs(stepped).max())
    E = sla.expm(dT * A)
    dt = dT / 37
    err = np.abs(Phi - E).max()
    assert err < 1e-9 and err < 10 * dT * (np.linalg.norm(A, 2) * dt) ** 4


# ------------------------------------------------------- block operators

def _tiny_problem(N=3, M=2, seed=11):
    s = inputs.SeededStream(seed)
    PhiF = 0.5 * s.normal(M * M).reshape(M, M)
    PhiG = 0.5 * s.normal(M * M).reshape(M, M)
    y0 = s.normal(M)
    return OracleProblem.from_propagators(PhiF, PhiG, y0, N), PhiF, PhiG, y0


def test_block_operator_matches_assembled_eq4():
    """apply_F equals the assembled block lower-bidiagonal matrix of eq. (4)
    (identity on the diagonal, -F on the subdiagonal, N+1 blocks)."""
    N, M = 3, 2
    prob, PhiF, PhiG, y0 = _tiny_problem(N, M)
    Fbig = np.eye((N + 1) * M)
    for n in range(1, N + 1):
        Fbig[n * M:(n + 1) * M, (n - 1) * M:n * M] = -PhiF
    X = inputs.SeededStream(3).normal((N + 1) * M).reshape(N + 1, M)
    np.testing.assert_allclose(prob.apply_F(X).reshape(-1), Fbig @ X.reshape(-1), atol=1e-14)


def test_sweep_matches_assembled_eq7():
    """sweep_Ginv equals the explicit block matrix of eq. (7), right
    (blocks G^{i-j} below the diagonal); the serial trajectory equals
    F^{-1} B with the blocks F^{i-j} of eq. (7), left."""
    N, M = 4, 2
    prob, PhiF, PhiG, y0 = _tiny_problem(N, M)
    Ginv = np.zeros(((N + 1) * M, (N + 1) * M))
    Finv = np.zeros_like(Ginv)
    for i in range(N + 1):
        for j in range(i + 1):
            Ginv[i * M:(i + 1) * M, j * M:(j + 1) * M] = np.linalg.matrix_power(PhiG, i - j)
            Finv[i * M:(i + 1) * M, j * M:(j + 1) * M] = np.linalg.matrix_power(PhiF, i - j)
    Q = inputs.SeededStream(4).normal((N + 1) * M).reshape(N + 1, M)
    np.testing.assert_allclose(prob.sweep_Ginv(Q).reshape(-1), Ginv @ Q.reshape(-1), atol=1e-13)
    np.testing.assert_allclose(prob.serial_fine().reshape(-1), Finv @ prob.rhs().reshape(-1), atol=1e-13)


def test_serial_trajectory_solves_all_at_once_system():
    """The serial fine trajectory is the exact solution of eq. (4): B - F Lam = 0."""
    w = inputs.heat1d()
    prob = OracleProblem.from_workload(w)
    lam = prob.serial_fine()
    res = prob.rhs() - prob.apply_F(lam)
    assert np.abs(res).max() <= 1e-14 * np.abs(lam).max()


# ------------------------------------------------------------ Algorithm 1

def _frac(v):
    return float(Fraction(v))


def test_algorithm1_hand_derived_iterates():
    """Exact rational iterates of Algorithm 1 for M = 1, N = 2 (tests/golden)."""
    g = json.load(open(os.path.join(GOLDEN, "bicgstab_scalar_N2.json")))
    f, gg, y0 = _frac(g["f"]), _frac(g["g"]), _frac(g["y0"])
    prob = OracleProblem.from_propagators(np.array([[f]]), np.array([[gg]]), [y0], g["N"])
    X0 = prob.coarse_prediction()
    np.testing.assert_allclose(X0[:, 0], [_frac(v) for v in g["X0"]], atol=1e-15)
    np.testing.assert_allclose(prob.residual(X0)[:, 0], [_frac(v) for v in g["R0"]], atol=1e-15)
    X1, info1 = pitsbicg(prob, tol=0.0, max_iter=1, eps0=0.0)
    s0 = info1.scalars[0]
    assert s0["rho"] == pytest.approx(_frac(g["rho0"]), rel=1e-14)
    assert s0["alpha"] == pytest.approx(_frac(g["alpha0"]), rel=1e-14)
    assert s0["omega"] == pytest.approx(_frac(g["omega0"]), rel=1e-14)
    assert s0["beta"] == pytest.approx(_frac(g["beta0"]), rel=1e-13)
    np.testing.assert_allclose(X1[:, 0], [_frac(v) for v in g["X1"]], atol=1e-15)
    np.testing.assert_allclose(info1.R[:, 0], [_frac(v) for v in g["R1"]], atol=1e-15)
    X2, info2 = pitsbicg(prob, tol=1e-12)
    assert info2.iterations == g["iterations"]
    assert info2.scalars[1]["alpha"] == pytest.approx(_frac(g["alpha1"]), rel=1e-13)
    np.testing.assert_allclose(X2[:, 0], [_frac(v) for v in g["X2"]], atol=1e-15)


def test_pitsbicg_converges_to_serial_heat1d():
    """PiTSBiCG on the 1D heat workload reaches the serial fine trajectory."""
    w = inputs.heat1d()
    prob = OracleProblem.from_workload(w)
    X, info = pitsbicg(prob, tol=1e-10)
    assert info.status == "ok"
    lam = prob.serial_fine()
    assert np.linalg.norm(X - lam) / np.linalg.norm(lam) < 1e-9
    assert info.matvecs <= 2 * info.iterations + 1


@pytest.mark.parametrize("N,M,seed", [(2, 1, 1), (3, 2, 2), (4, 3, 3), (4, 4, 4), (3, 4, 5)])
def test_finite_termination_tiny(N, M, seed):
    """G^{-1}F = I + nilpotent (degree <= N+1 minimal polynomial): BiCGStab
    reaches the exact solution within N+1 iterations on tiny systems."""
    s = inputs.SeededStream(100 + seed)
    PhiF = np.eye(M) * 0.6 + 0.2 * s.normal(M * M).reshape(M, M)
    PhiG = PhiF + 0.1 * s.normal(M * M).reshape(M, M)
    prob = OracleProblem.from_propagators(PhiF, PhiG, s.normal(M), N)
    X, info = pitsbicg(prob, tol=1e-13)
    lam = prob.serial_fine()
    assert info.iterations <= N + 1
    assert np.abs(X - lam).max() <= 1e-11 * np.abs(lam).max()


def test_recursive_residual_tracks_true_residual():
    """After k iterations the recursive R^k equals G^{-1}(B - F X^k) to rounding."""
    w = inputs.heat1d(M=31, N=8, fine_steps=20)
    prob = OracleProblem.from_workload(w)
    for k in (1, 2, 3):
        X, info = pitsbicg(prob, tol=0.0, max_iter=k)
        true_R = prob.residual(X)
        # the gap is a rounding-level multiple of the data scale, ||B|| = ||y0||
        assert np.abs(info.R - true_R).max() <= 1e-13 * np.linalg.norm(prob.y0)
        assert norm_N_inf(true_R) < 0.5 * info.r0


def test_coarse_equal_fine_exits_at_first_half_step():
    """G = F gives G^{-1}F = I: S^0 = R^0 - D^0 = 0 and X^1 is exact."""
    M, N = 3, 5
    s = inputs.SeededStream(9)
    Phi = 0.5 * np.eye(M) + 0.1 * s.normal(M * M).reshape(M, M)
    prob = OracleProblem.from_propagators(Phi, Phi, s.normal(M), N)
    X, info = pitsbicg(prob, tol=1e-14, x0="zero")
    assert info.iterations == 1 and info.matvecs == 2
    assert info.scalars[0]["alpha"] == pytest.approx(1.0, rel=1e-14)
    np.testing.assert_allclose(X, prob.serial_fine(), atol=1e-14)


def test_forced_restart_keeps_solution():
    """eps0 = 1 forces the restart branch every iteration; the solution is unchanged."""
    w = inputs.heat1d(M=15, N=6, fine_steps=10)
    prob = OracleProblem.from_workload(w)
    X, info = pitsbicg(prob, tol=1e-12, eps0=1.0, max_iter=200)
    assert info.restarts >= 1 and info.status == "ok"
    lam = prob.serial_fine()
    assert np.linalg.norm(X - lam) / np.linalg.norm(lam) < 1e-10


def test_solution_independent_of_coarse_propagator():
    """Lam* solves F Lam = B whatever G is; only the iteration count changes."""
    w = inputs.heat1d(M=31, N=8, fine_steps=40)
    p1 = OracleProblem.from_workload(w)
    p2 = OracleProblem(p1.F, implicit_euler_propagator(p1.L, w.T / w.N, 2), p1.y0, w.N)
    X1, _ = pitsbicg(p1, tol=1e-12)
    X2, _ = pitsbicg(p2, tol=1e-12)
    np.testing.assert_allclose(X1, X2, atol=1e-11 * np.abs(X1).max())


def test_block_inner_product_scale_invariance():
    """A positive weight on the inner product (an h^d mesh factor) cancels in
    alpha, omega and beta: scaling every block vector leaves the iterates fixed."""
    w = inputs.heat1d(M=15, N=6, fine_steps=10)
    prob = OracleProblem.from_workload(w)
    X1, i1 = pitsbicg(prob, tol=0.0, max_iter=3)
    w2 = inputs.heat1d(M=15, N=6, fine_steps=10)
    w2.y0 = w2.y0 * 1024.0
    X2, i2 = pitsbicg(OracleProblem.from_workload(w2), tol=0.0, max_iter=3)
    np.testing.assert_allclose(X2 / 1024.0, X1, rtol=1e-12, atol=1e-15)
    for a, b in zip(i1.scalars, i2.scalars):
        assert a["alpha"] == pytest.approx(b["alpha"], rel=1e-12)
        assert a["omega"] == pytest.approx(b["omega"], rel=1e-12)


# --------------------------------------------------------------- parareal

def test_parareal_exact_after_k_iterations():
    """Parareal (eq. (6)) reproduces lam_0..lam_k exactly after k iterations,
    and the whole fine trajectory at k = N."""
    w = inputs.heat1d(M=31, N=8, fine_steps=20)
    prob = OracleProblem.from_workload(w)
    lam = prob.serial_fine()
    for k in (1, 3, 8):
        X, info = parareal(prob, kmax=k)
        assert info.iterations == k
        np.testing.assert_allclose(X[:k + 1], lam[:k + 1], atol=1e-13 * np.abs(lam).max())
    assert np.abs(X - lam).max() <= 1e-13 * np.abs(lam).max()


def test_parareal_matches_predictor_corrector_eq5():
    """Eq. (6) equals the predictor-corrector lam_{n+1}^{k+1} =
    G(lam_n^{k+1}) + F(lam_n^k) - G(lam_n^k) row by row."""
    w = inputs.heat1d(M=15, N=6, fine_steps=10)
    prob = OracleProblem.from_workload(w)
    prev = prob.coarse_prediction()
    for k in range(3):
        nxt = np.empty_like(prev)
        nxt[0] = prob.y0
        for n in range(prob.N):
            nxt[n + 1] = (prob.G(nxt[n][None])[0] + prob.F(prev[n][None])[0] - prob.G(prev[n][None])[0])
        X, _ = parareal(prob, kmax=k + 1)
        np.testing.assert_allclose(X, nxt, atol=1e-13)
        prev = nxt


# ------------------------------------------------------------ sources (f != 0)
def test_forced_scalar_closed_forms():
    """y' = a y + b from 0 over one slice: implicit Euler gives
    y* (1 - (1 - a dt)^(-m)) and RK4 gives y* (1 - R(a dt)^m), y* = -b/a
    (both methods keep the steady state y* exactly)."""
    from oracle.operators import implicit_euler_propagator, rk4_propagator
    a, b, dT, m = -3.0, 0.7, 0.4, 9
    dt = dT / m
    ys = -b / a
    L = np.array([[a]])
    c_ie = implicit_euler_propagator(L, dT, m, source=[b])(np.zeros((1, 1)))[0, 0]
    assert c_ie == pytest.approx(ys * (1 - (1 - a * dt) ** (-m)), rel=1e-13)
    z = a * dt
    R = 1 + z + z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    c_rk = rk4_propagator(L, dT, m, source=[b])(np.zeros((1, 1)))[0, 0]
    assert c_rk == pytest.approx(ys * (1 - R ** m), rel=1e-12)
    # the steady state is a fixed point of both
    assert implicit_euler_propagator(L, dT, m, source=[b])(np.array([[ys]]))[0, 0] == pytest.approx(ys, rel=1e-14)
    assert rk4_propagator(L, dT, m, source=[b])(np.array([[ys]]))[0, 0] == pytest.approx(ys, rel=1e-14)


@pytest.mark.parametrize("fine", [("ie", 7), ("rk4", 5)])
def test_forced_system_solution_is_forced_serial_trajectory(fine):
    """With a source, the solution of F Lambda = B (B = (y0, c, ..., c)),
    solved densely, is the serial trajectory of the affine fine propagator,
    and parareal reaches it after N corrections."""
    w = inputs.with_source(inputs.heat1d(M=9, N=6, fine_steps=fine[1]))
    w.fine = fine
    o = OracleProblem.from_workload(w)
    lam = o.serial_fine()
    n = (w.N + 1) * w.M
    E = np.eye(n)
    Fm = np.stack([o.apply_F(E[i].reshape(w.N + 1, w.M)).ravel() for i in range(n)], axis=1)
    X = np.linalg.solve(Fm, o.rhs().ravel()).reshape(w.N + 1, w.M)
    assert np.abs(X - lam).max() <= 1e-12 * np.abs(lam).max()
    Xp, _ = parareal(o, kmax=w.N)
    assert np.abs(Xp - lam).max() <= 1e-12 * np.abs(lam).max()
    Xb, info = pitsbicg(o, tol=1e-13)
    assert np.abs(Xb - lam).max() <= 1e-10 * np.abs(lam).max()


def test_fem_backward_euler_is_the_mass_matrix_step():
    """Sec. 4 (FEM, backward Euler): with A = -Mm^{-1}(mu K + C) - r I the
    oracle's implicit Euler step (I - dt A)^{-1} is the mass-matrix step
    (Mm + dt (mu K + C + r Mm)) y+ = Mm y, solved here directly from the
    assembled matrices, and the fine propagator is its m-th power."""
    from oracle.operators import implicit_euler_propagator
    n, dt, m = 7, 1e-3, 5
    for pde in inputs.PAPER_PDES:
        mu, r, adv = inputs.PAPER_PDES[pde]
        w = inputs.paper_pde(pde, n=n, N=4, T=4 * m * dt, dt=dt, discretization="fem")
        assert w.fine == ("ie", m)
        Mm, K, C = inputs.fem_p1_matrices(n, adv)
        S = Mm + dt * (mu * K + C + r * Mm)
        y = w.y0[0]
        for _ in range(m):
            y = np.linalg.solve(S, Mm @ y)
        got = implicit_euler_propagator(w.A, w.T / w.N, m)(w.y0)[0]
        np.testing.assert_allclose(got, y, rtol=1e-11, atol=1e-14)
