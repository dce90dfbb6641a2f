"""FP64 oracle: propagators and block operators of PiTSBiCG.

TEST INFRASTRUCTURE ONLY.  This module is the plain, slow, CPU statement of
what the CUDA path computes.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / reference leg of ``bench.py`` may import it; the
product path never calls it.  It shares no code with the CUDA library.

Every function names the passage of Riahi, "PiTSBiCG: Parallel in Time Stable
Bi-Conjugate Gradient Algorithm" (arXiv 2203.10148) it follows:

* Sec. 2, eq. (1): the Cauchy problem y' = A y + f on [0, T] (f a
  time-independent source, 0 unless given);
* Sec. 2, eq. (2): N equal slices, each started from lambda_n;
* Sec. 2, eq. (3): continuity lambda_{n+1} = F(lambda_n);
* Sec. 2, eq. (4): the all-at-once block bidiagonal system  F Lambda = B;
* Sec. 3, eq. (7): the inverses of the block operators; G^{-1} is applied
  by forward substitution (a sequential sweep, Sec. 3 text after Alg. 1).

Readings of points the paper leaves open:

* Lambda has N+1 blocks lambda_0..lambda_N (eq. (7) shows F^N in the
  bottom-left corner and the text after Algorithm 1 places the iterates in
  (L^2)^{N+1}); the block operator then holds exactly N fine propagations.
* B = (y0, 0, ..., 0): every row n >= 1 of eq. (4) is lambda_n - F(lambda_{n-1}) = 0.
* The fine and coarse solvers are fixed linear time steppers of the
  semi-discrete problem: implicit Euler (IE) or classical RK4 (stage form).
  The periodic advection-diffusion coarse step is IE with its linear solve
  replaced by a fixed number K of Chebyshev steps (``chebyshev_ie_propagator``),
  a fixed linear operator like the others; K = 0 in a workload means the
  exact IE solve.
* The block inner product sums the Euclidean products of all N+1 blocks
  (no mesh weight; it cancels in alpha, beta and omega).
* ||.||_{N,inf} is the largest Euclidean norm over the blocks.

Layout: a block vector is an (N+1, M) float64 array, row n = lambda_n; 2D
states are row-major with index j*nx + i (j the y index).

Parity pins live in tests/test_oracle_pins.py.
"""
from __future__ import annotations

import math
from typing import Callable, Optional

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

Propagator = Callable[[np.ndarray], np.ndarray]


# --------------------------------------------------------------------------
# Spatial operators (the linear differential operator of eq. (1), discretised)
# --------------------------------------------------------------------------

def second_difference(n: int, h: float) -> sp.csr_matrix:
    """Dirichlet-0 second difference (u_{i-1} - 2 u_i + u_{i+1}) / h^2, n points."""
    e = np.ones(n)
    return sp.diags([e[:-1], -2.0 * e, e[:-1]], [-1, 0, 1], format="csr") / (h * h)


def periodic_shift(n: int, s: int) -> sp.csr_matrix:
    """(S u)_i = u_{(i + s) mod n}."""
    rows = np.arange(n)
    return sp.csr_matrix((np.ones(n), (rows, (rows + s) % n)), shape=(n, n))


def spatial_operator(kind: str, nx: int, ny: int, nu: float,
                     vx: Optional[np.ndarray] = None, vy: Optional[np.ndarray] = None,
                     A: Optional[np.ndarray] = None):
    """The operator L of y' = L y for each workload family (eq. (1), f = 0).

    heat1d:    nu * D2, M = nx interior points, h = 1/(nx+1).
    heat2d:    nu * (D2_x + D2_y), 5-point, Dirichlet 0, h = 1/(n+1) per axis.
    advdiff2d: nu * periodic 5-point Laplacian - vx * Dx_up - vy * Dy_up on
               the periodic grid x_i = i/nx; Dx_up is the upwind one-sided
               difference (backward where vx >= 0, forward where vx < 0).
    dense:     the given matrix A.
    Returns a scipy sparse matrix, or a dense ndarray for ``dense``.
    """
    if kind == "heat1d":
        return (nu * second_difference(nx, 1.0 / (nx + 1))).tocsr()
    if kind == "heat2d":
        Ix, Iy = sp.identity(nx), sp.identity(ny)
        Dx = second_difference(nx, 1.0 / (nx + 1))
        Dy = second_difference(ny, 1.0 / (ny + 1))
        # index j*nx + i: x varies fastest, so x acts on the second Kronecker factor
        return (nu * (sp.kron(Iy, Dx) + sp.kron(Dy, Ix))).tocsr()
    if kind == "advdiff2d":
        hx, hy = 1.0 / nx, 1.0 / ny
        Ix, Iy = sp.identity(nx), sp.identity(ny)
        Sxp, Sxm = periodic_shift(nx, +1), periodic_shift(nx, -1)
        Syp, Sym = periodic_shift(ny, +1), periodic_shift(ny, -1)
        lap_x = (Sxp - 2.0 * sp.identity(nx) + Sxm) / (hx * hx)
        lap_y = (Syp - 2.0 * sp.identity(ny) + Sym) / (hy * hy)
        lap = sp.kron(Iy, lap_x) + sp.kron(lap_y, Ix)
        back_x = sp.kron(Iy, (sp.identity(nx) - Sxm) / hx)   # (u_i - u_{i-1}) / h
        fwd_x = sp.kron(Iy, (Sxp - sp.identity(nx)) / hx)    # (u_{i+1} - u_i) / h
        back_y = sp.kron((sp.identity(ny) - Sym) / hy, Ix)
        fwd_y = sp.kron((Syp - sp.identity(ny)) / hy, Ix)
        vxp, vxm = np.maximum(vx, 0.0), np.minimum(vx, 0.0)
        vyp, vym = np.maximum(vy, 0.0), np.minimum(vy, 0.0)
        adv = (sp.diags(vxp) @ back_x + sp.diags(vxm) @ fwd_x
               + sp.diags(vyp) @ back_y + sp.diags(vym) @ fwd_y)
        return (nu * lap - adv).tocsr()
    if kind == "dense":
        return np.array(A, dtype=np.float64)
    raise ValueError(f"unknown operator kind {kind!r}")


# --------------------------------------------------------------------------
# Time steppers over one slice (the fine solver F and coarse solver G)
# --------------------------------------------------------------------------

def _identity_like(L):
    n = L.shape[0]
    return sp.identity(n, format="csc") if sp.issparse(L) else np.eye(n)


def implicit_euler_propagator(L, dT: float, steps: int, source=None) -> Propagator:
    """u <- (I - dt L)^{-1} (u + dt f), repeated ``steps`` times with dt = dT/steps
    (f = 0 without a source: the linear propagator).

    Acts on the rows of a (k, M) array.  The linear solve uses a direct LU
    factorisation (SuperLU for sparse L, LAPACK for dense L).
    """
    dt = dT / steps
    Msys = _identity_like(L) - dt * L
    if sp.issparse(Msys):
        lu = spla.splu(sp.csc_matrix(Msys))
        solve = lu.solve
    else:
        fac = sla.lu_factor(Msys)
        solve = lambda rhs: sla.lu_solve(fac, rhs)

    f = None if source is None else np.asarray(source, dtype=np.float64).reshape(-1, 1)

    def apply(X: np.ndarray) -> np.ndarray:
        U = np.array(X, dtype=np.float64).T.copy()    # (M, k): one state per column
        for _ in range(steps):
            U = solve(U if f is None else U + dt * f)
        return U.T.copy()

    return apply


def chebyshev_ie_propagator(L, dT: float, steps: int, K: int) -> Propagator:
    """Implicit Euler with each linear solve replaced by K steps of Chebyshev
    acceleration: the coarse propagator of the periodic advection-diffusion
    problem, whose implicit-Euler system has variable coefficients and is not
    symmetric.

    One step of dt = dT/steps maps b to the K-th iterate of Chebyshev
    acceleration (Saad, Iterative Methods for Sparse Linear Systems, 2nd ed.,
    Sec. 12.3, Algorithm 12.1) for the Jacobi-scaled implicit-Euler system
    D^{-1} (I - dt L) w = D^{-1} b, D = diag(I - dt L), started from w = b,
    with the eigenvalue interval [1 - rho, 1 + rho], rho = max_p (D_p - 1)/D_p:
    the Gershgorin discs of D^{-1}(I - dt L) all lie in |z - 1| <= rho (the
    off-diagonal row sums of I - dt L equal D_p - 1).  K and the interval are
    fixed, so the step is a fixed polynomial in D^{-1}(I - dt L): a linear
    operator, as eq. (7) requires of G, that tends to the exact implicit-Euler
    step as K grows.  Works on real or complex rows.
    """
    dt = dT / steps
    A = (_identity_like(L) - dt * L)
    A = sp.csr_matrix(A) if sp.issparse(A) else np.asarray(A)
    diag = np.asarray(A.diagonal(), dtype=np.float64)
    rho = float(np.max((diag - 1.0) / diag))
    theta, delta = 1.0, rho          # centre and half-width of [1 - rho, 1 + rho]

    def scaled(V):                   # D^{-1} A V, column by column
        return (A @ V) / diag[:, None]

    def solve(B):
        if delta == 0.0:             # A = I: w = b is the exact solution
            return B.copy()
        X = B.copy()
        R = B / diag[:, None] - scaled(X)          # r_0 of the scaled system
        sigma1 = theta / delta
        rho_k = 1.0 / sigma1
        Dk = R / theta
        for k in range(K):
            X = X + Dk
            if k == K - 1:
                break
            R = R - scaled(Dk)
            rho_next = 1.0 / (2.0 * sigma1 - rho_k)
            Dk = (rho_next * rho_k) * Dk + (2.0 * rho_next / delta) * R
            rho_k = rho_next
        return X

    def apply(X: np.ndarray) -> np.ndarray:
        Xa = np.asarray(X)
        U = np.array(Xa, dtype=np.result_type(Xa.dtype, np.float64)).T.copy()
        for _ in range(steps):
            U = solve(U)
        return U.T.copy()

    return apply


def rk4_propagator(L, dT: float, steps: int, source=None) -> Propagator:
    """Classical four-stage Runge-Kutta (stage form) for u' = L u + f, dt = dT/steps
    (f = 0 without a source)."""
    dt = dT / steps
    f = 0.0 if source is None else np.asarray(source, dtype=np.float64).reshape(-1, 1)

    def apply(X: np.ndarray) -> np.ndarray:
        U = np.array(X, dtype=np.float64).T.copy()
        for _ in range(steps):
            k1 = L @ U + f
            k2 = L @ (U + 0.5 * dt * k1) + f
            k3 = L @ (U + 0.5 * dt * k2) + f
            k4 = L @ (U + dt * k3) + f
            U = U + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        return U.T.copy()

    return apply


def rk4_step_matrix(A: np.ndarray, dt: float) -> np.ndarray:
    """The RK4 one-step matrix R(dt A) = I + Z + Z^2/2 + Z^3/6 + Z^4/24, Z = dt A."""
    Z = dt * np.asarray(A, dtype=np.float64)
    I = np.eye(Z.shape[0])
    Z2 = Z @ Z
    Z3 = Z2 @ Z
    Z4 = Z3 @ Z
    return I + Z + Z2 / 2.0 + Z3 / 6.0 + Z4 / 24.0


def matrix_power_binary(R: np.ndarray, m: int) -> np.ndarray:
    """R^m by repeated squaring (plain binary powering)."""
    result = np.eye(R.shape[0])
    base = R.copy()
    while m > 0:
        if m & 1:
            result = result @ base
        m >>= 1
        if m:
            base = base @ base
    return result


def dense_rk4_propagator_matrix(A: np.ndarray, dT: float, steps: int) -> np.ndarray:
    """Phi_F = R(dt A)^steps, the dense fine propagator of one slice, dt = dT/steps."""
    return matrix_power_binary(rk4_step_matrix(A, dT / steps), steps)


def matrix_propagator(Phi: np.ndarray) -> Propagator:
    """u <- Phi u for each row of X."""
    Phi = np.asarray(Phi, dtype=np.float64)
    return lambda X: np.asarray(X, dtype=np.float64) @ Phi.T


# --------------------------------------------------------------------------
# The problem: L, F, G and y0
# --------------------------------------------------------------------------

class OracleProblem:
    """One PiT problem: operator, fine propagator F and coarse propagator G.

    Built from a workload description (fields kind, nx, ny, nu, vx, vy, A,
    T, N, fine, coarse, y0), or directly from two propagators for algebraic
    tests (``from_propagators``).
    """

    def __init__(self, fine: Propagator, coarse: Propagator, y0: np.ndarray, N: int,
                 T: float = 1.0, L=None, fine_forced: Optional[Propagator] = None):
        self.F = fine
        self.G = coarse
        self.y0 = np.asarray(y0, dtype=np.float64).reshape(-1)
        self.N = int(N)
        self.T = float(T)
        self.M = self.y0.size
        # A source f (eq. (1)) makes the fine propagator affine,
        # F_f(lam) = F(lam) + c with c = F_f(0), the same for every slice of a
        # time-independent source; the rows n >= 1 of eq. (4) then read
        # lam_n - F(lam_{n-1}) = c.
        self.F_forced = fine_forced
        self.c = None if fine_forced is None else fine_forced(np.zeros((1, self.M)))[0]
        self.L = L

    @classmethod
    def from_workload(cls, w, member: int = 0) -> "OracleProblem":
        L = spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy, w.A)
        dT = w.T / w.N
        fk, fm = w.fine
        ck, cm = w.coarse
        if fk == "ie":
            F = implicit_euler_propagator(L, dT, fm)
        elif fk == "rk4" and w.kind == "dense":
            F = matrix_propagator(dense_rk4_propagator_matrix(L, dT, fm))
        elif fk == "rk4":
            F = rk4_propagator(L, dT, fm)
        else:
            raise ValueError(fk)
        if ck == "ie" and w.kind == "advdiff2d" and getattr(w, "coarse_inner", 0) > 0:
            G = chebyshev_ie_propagator(L, dT, cm, w.coarse_inner)
        elif ck == "ie":
            G = implicit_euler_propagator(L, dT, cm)
        elif ck == "rk4":
            G = rk4_propagator(L, dT, cm)
        else:
            raise ValueError(ck)
        y0 = np.asarray(w.y0)
        y0 = y0[member] if y0.ndim == 2 else y0
        Ff = None
        src = getattr(w, "f", None)
        if src is not None:
            src = np.asarray(src)
            src = src[member] if src.ndim == 2 else src
            if fk == "ie":
                Ff = implicit_euler_propagator(L, dT, fm, source=src)
            else:
                Ff = rk4_propagator(L, dT, fm, source=src)
        return cls(F, G, y0, w.N, w.T, L, fine_forced=Ff)

    @classmethod
    def from_propagators(cls, Phi_F: np.ndarray, Phi_G: np.ndarray, y0, N: int) -> "OracleProblem":
        return cls(matrix_propagator(Phi_F), matrix_propagator(Phi_G), y0, N)

    # ---- block vectors --------------------------------------------------
    def zeros(self) -> np.ndarray:
        return np.zeros((self.N + 1, self.M))

    def rhs(self) -> np.ndarray:
        """B = (y0, 0, ..., 0), the right-hand side of eq. (4); with a source
        B = (y0, c, ..., c)."""
        B = self.zeros()
        B[0] = self.y0
        if self.c is not None:
            B[1:] = self.c
        return B

    def apply_F(self, Lam: np.ndarray) -> np.ndarray:
        """Block operator of eq. (4): (F Lam)_0 = lam_0, (F Lam)_n = lam_n - F(lam_{n-1}).

        The N fine propagations F(lam_0..lam_{N-1}) are independent (eq. (2)).
        """
        Lam = np.asarray(Lam, dtype=np.float64)
        Y = Lam.copy()
        Y[1:] -= self.F(Lam[:-1])
        return Y

    def sweep_Ginv(self, Q: np.ndarray) -> np.ndarray:
        """G^{-1} Q by forward substitution (eq. (7), right): z_0 = q_0,
        z_n = q_n + G(z_{n-1}), one coarse step after the other."""
        Q = np.asarray(Q, dtype=np.float64)
        Z = np.empty_like(Q)
        Z[0] = Q[0]
        for n in range(1, self.N + 1):
            Z[n] = Q[n] + self.G(Z[n - 1][None, :])[0]
        return Z

    def apply_GinvF(self, Lam: np.ndarray) -> np.ndarray:
        """The preconditioned operator G^{-1} F of eq. (8), applied matrix-free."""
        return self.sweep_Ginv(self.apply_F(Lam))

    def residual(self, X: np.ndarray) -> np.ndarray:
        """Preconditioned residual G^{-1}(B - F X) (Algorithm 1, first line)."""
        return self.sweep_Ginv(self.rhs() - self.apply_F(X))

    def serial_fine(self) -> np.ndarray:
        """lam_0 = y0, lam_n = F(lam_{n-1}): the serial fine trajectory, which is
        F^{-1} B by the forward substitution of eq. (7), left.  With a source
        the affine fine propagator itself is stepped (not F + c)."""
        F = self.F if self.F_forced is None else self.F_forced
        Lam = self.zeros()
        Lam[0] = self.y0
        for n in range(1, self.N + 1):
            Lam[n] = F(Lam[n - 1][None, :])[0]
        return Lam

    def coarse_prediction(self) -> np.ndarray:
        """G^{-1} B: lam_n = G^n y0, the parareal predictor at k = 0 (eq. (6))."""
        return self.sweep_Ginv(self.rhs())


# --------------------------------------------------------------------------
# Block inner product and norm (Sec. 3, text after Algorithm 1)
# --------------------------------------------------------------------------

def block_dot(U: np.ndarray, V: np.ndarray) -> float:
    """<U, V> = sum over the blocks of the Euclidean product of the states."""
    return float(np.sum(np.asarray(U, dtype=np.float64) * np.asarray(V, dtype=np.float64)))


def block_norms(U: np.ndarray) -> np.ndarray:
    """Euclidean norm of each block lambda_n."""
    return np.sqrt(np.sum(np.asarray(U, dtype=np.float64) ** 2, axis=1))


def norm_N_inf(U: np.ndarray) -> float:
    """||U||_{N,inf} = max_n ||U_n||_2 (Algorithm 1, the while test)."""
    return float(np.max(block_norms(U)))


def norm2(U: np.ndarray) -> float:
    return math.sqrt(block_dot(U, U))
