"""Seeded synthetic workloads for PiTSBiCG (Riahi, arXiv 2203.10148).

This module only *builds inputs*: grids, coefficients, initial values and the
serving request stream.  It holds none of the method's arithmetic (no
propagator, no block operator, no Krylov step), so both the CUDA path and the
FP64 oracle can consume the same arrays without sharing any code that computes
the method.

Random numbers come from a counter-based SplitMix64 stream (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): output
``i`` of a stream with key ``k`` is ``mix64(k + (i+1) * 0x9E3779B97F4A7C15)``.
Uniforms take the top 53 bits; normals use the Box-Muller transform.  The
generator is plain integer arithmetic, so it gives identical arrays on x86 and
Arm hosts and across numpy versions.

Workload recipes (the paper's experiments are FEM runs in FreeFem++ on
problems of the form of eq. (9), Sec. 4; those are not reproducible here, so
seeded finite-difference workloads of the same family stand in for them):

* ``heat1d``   -- u_t = nu u_xx on (0,1), Dirichlet 0, M interior points,
                  h = 1/(M+1); fine = implicit Euler (IE) m steps per slice,
                  coarse = IE 1 step per slice; u0 = sin(pi x) + 0.5 sin(3 pi x)
                  + N(0, sigma^2) noise.
* ``heat2d``   -- u_t = nu (u_xx + u_yy) on the unit square, Dirichlet 0,
                  n x n interior points, h = 1/(n+1); fine = RK4 m steps per
                  slice, coarse = IE 1 step; u0 = sum of Gaussian bumps.
* ``advdiff2d``-- u_t = nu Lap u - v . grad u on the periodic unit square,
                  n x n points x_i = i/n; v = curl of a random stream function
                  (8 Fourier modes) scaled to max |v| = 1; upwind advection,
                  central diffusion; fine = RK4 with
                  dt = min(0.4 h/|v|max, 0.2 h^2/nu); coarse = IE 1 step
                  whose linear solve is ``coarse_inner`` Chebyshev steps.
* ``dense``    -- y' = A y, A = -(S S^T/M + 0.1 I) + 0.5 (K - K^T)/sqrt(M);
                  fine = RK4 with ``steps`` steps per slice (applied as one
                  precomputed dense propagator), coarse = IE 1 step.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Default seeds of the named workloads (one per configuration family).
SEED_HEAT1D = 0x50495400
SEED_HEAT2D = 0x50495401
SEED_ADVDIFF2D = 0x50495402
SEED_SERVING = 0x50495300
SEED_DENSE = 0x50495404


def _mix64(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


class SeededStream:
    """Counter-based SplitMix64 stream; ``draws`` advance a 64-bit counter."""

    def __init__(self, seed: int):
        self.key = np.uint64(int(seed) & 0xFFFFFFFFFFFFFFFF)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        idx = np.arange(self.counter + 1, self.counter + n + 1, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            z = self.key + idx * _GAMMA
        return _mix64(z)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return lo + (hi - lo) * u

    def normal(self, n: int, sigma: float = 1.0) -> np.ndarray:
        m = (n + 1) // 2
        u1 = 1.0 - self.uniform(m)          # (0, 1]
        u2 = self.uniform(m)
        r = np.sqrt(-2.0 * np.log(u1))
        z = np.concatenate([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)])
        return sigma * z[:n]

    def integers(self, lo: int, hi: int, n: int) -> np.ndarray:
        """Uniform integers in the closed range [lo, hi]."""
        u = self.uniform(n)
        return (lo + np.floor(u * (hi - lo + 1))).astype(np.int64).clip(lo, hi)


@dataclasses.dataclass
class Workload:
    """One PiT problem (or a batch of problems sharing one operator).

    ``y0`` has shape (batch, M); ``M = nx * ny`` with row-major 2D states
    (index j * nx + i, j the y index).  ``fine`` and ``coarse`` are
    (stepper, steps per slice) with stepper in {"ie", "rk4"}.
    """

    name: str
    kind: str
    nx: int
    ny: int
    nu: float
    T: float
    N: int
    fine: Tuple[str, int]
    coarse: Tuple[str, int]
    y0: np.ndarray
    vx: Optional[np.ndarray] = None
    vy: Optional[np.ndarray] = None
    A: Optional[np.ndarray] = None
    tol: float = 1e-6
    precision: str = "fp64"
    arrival: float = 0.0
    f: Optional[np.ndarray] = None     # time-independent source (batch, M) of y' = L y + f
    # advdiff2d: Chebyshev steps replacing each implicit-Euler solve of the
    # coarse step (0: the library's default)
    coarse_inner: int = 0

    @property
    def M(self) -> int:
        return self.nx * self.ny

    @property
    def batch(self) -> int:
        return self.y0.shape[0]

    @property
    def dT(self) -> float:
        return self.T / self.N

    def member(self, b: int) -> "Workload":
        return dataclasses.replace(self, y0=self.y0[b:b + 1].copy(),
                                   f=None if self.f is None else self.f[b:b + 1].copy())

    def describe(self) -> dict:
        return {"workload": self.name, "kind": self.kind, "grid": [self.nx, self.ny],
                "M": self.M, "N": self.N, "batch": self.batch, "T": self.T, "nu": self.nu,
                "fine": list(self.fine), "coarse": list(self.coarse), "tol": self.tol,
                **({"coarse_inner": self.coarse_inner} if self.coarse_inner else {}),
                "precision": self.precision}


def heat1d(M: int = 63, nu: float = 0.1, T: float = 1.0, N: int = 16,
           fine_steps: int = 100, coarse_steps: int = 1, noise: float = 1e-3,
           batch: int = 1, seed: int = SEED_HEAT1D, tol: float = 1e-10) -> Workload:
    s = SeededStream(seed)
    x = np.arange(1, M + 1) / (M + 1.0)
    base = np.sin(np.pi * x) + 0.5 * np.sin(3.0 * np.pi * x)
    y0 = np.stack([base + s.normal(M, noise) for _ in range(batch)])
    return Workload(f"heat1d_M{M}_N{N}", "heat1d", M, 1, nu, T, N, ("ie", fine_steps),
                    ("ie", coarse_steps), y0, tol=tol, precision="fp64")


def gaussian_bumps(s: SeededStream, n: int, count: int) -> np.ndarray:
    """Sum of ``count`` Gaussian bumps on the n x n interior grid, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    xs = np.arange(1, n + 1) * h
    X, Y = np.meshgrid(xs, xs, indexing="xy")      # X varies along columns (i)
    a = s.uniform(count)
    w = s.uniform(count, 0.03, 0.1)
    c = s.uniform(2 * count, 0.2, 0.8).reshape(count, 2)
    u = np.zeros((n, n))
    for j in range(count):
        r2 = (X - c[j, 0]) ** 2 + (Y - c[j, 1]) ** 2
        u += a[j] * np.exp(-r2 / (2.0 * w[j] ** 2))
    return u.reshape(-1)


def heat2d(n: int = 128, nu: float = 1e-2, T: float = 1.0, N: int = 512,
           fine_steps: int = 50, coarse_steps: int = 1, bumps: int = 8,
           batch: int = 1, seed: int = SEED_HEAT2D, tol: float = 1e-6,
           precision: str = "mixed") -> Workload:
    s = SeededStream(seed)
    y0 = np.stack([gaussian_bumps(s, n, bumps) for _ in range(batch)])
    return Workload(f"heat2d_{n}x{n}_N{N}", "heat2d", n, n, nu, T, N, ("rk4", fine_steps),
                    ("ie", coarse_steps), y0, tol=tol, precision=precision)


def _integer_modes(s: SeededStream, count: int, kmax: int) -> np.ndarray:
    out = []
    while len(out) < count:
        k = s.integers(-kmax, kmax, 2)
        if k[0] != 0 or k[1] != 0:
            out.append(k)
    return np.array(out, dtype=np.float64)


def advdiff2d_rk4_steps(n: int, nu: float, dT: float, vmax: float = 1.0) -> int:
    """RK4 steps per slice: dt = min(0.4 h/|v|max, 0.2 h^2/nu), h = 1/n."""
    h = 1.0 / n
    dt = min(0.4 * h / vmax, 0.2 * h * h / nu)
    return int(math.ceil(dT / dt - 1e-12))


def advdiff2d(n: int = 512, nu: float = 5e-3, T: float = 0.5, N: int = 256,
              fine_steps: Optional[int] = None, coarse_steps: int = 1, coarse_inner: int = 48,
              psi_modes: int = 8, u_modes: int = 16, batch: int = 1,
              seed: int = SEED_ADVDIFF2D, tol: float = 1e-6,
              precision: str = "mixed") -> Workload:
    s = SeededStream(seed)
    xs = np.arange(n) / float(n)
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    k = _integer_modes(s, psi_modes, 4)
    a = s.normal(psi_modes)
    phi = s.uniform(psi_modes, 0.0, 2.0 * np.pi)
    dpsi_dx = np.zeros((n, n))
    dpsi_dy = np.zeros((n, n))
    for j in range(psi_modes):
        arg = 2.0 * np.pi * (k[j, 0] * X + k[j, 1] * Y) + phi[j]
        dpsi_dx += a[j] * 2.0 * np.pi * k[j, 0] * np.cos(arg)
        dpsi_dy += a[j] * 2.0 * np.pi * k[j, 1] * np.cos(arg)
    vx, vy = dpsi_dy, -dpsi_dx
    scale = 1.0 / np.max(np.sqrt(vx * vx + vy * vy))
    # the velocity field sampled as FP32 values (every coefficient v / h of a
    # power-of-two grid is then exact in FP32); both sides read these arrays
    vx = (vx * scale).astype(np.float32).astype(np.float64)
    vy = (vy * scale).astype(np.float32).astype(np.float64)
    y0s = []
    for _ in range(batch):
        kk = _integer_modes(s, u_modes, 4)
        b = s.normal(u_modes)
        th = s.uniform(u_modes, 0.0, 2.0 * np.pi)
        u = np.zeros((n, n))
        for j in range(u_modes):
            u += b[j] * np.cos(2.0 * np.pi * (kk[j, 0] * X + kk[j, 1] * Y) + th[j]) / np.hypot(*kk[j])
        y0s.append(u.reshape(-1))
    if fine_steps is None:
        fine_steps = advdiff2d_rk4_steps(n, nu, T / N)
    return Workload(f"advdiff2d_{n}x{n}_N{N}", "advdiff2d", n, n, nu, T, N, ("rk4", fine_steps),
                    ("ie", coarse_steps), np.stack(y0s), vx=vx.reshape(-1).copy(),
                    vy=vy.reshape(-1).copy(), tol=tol, precision=precision,
                    coarse_inner=coarse_inner)


def dense(M: int = 1024, T: float = 10.0, N: int = 4096, fine_steps: int = 200,
          coarse_steps: int = 1, batch: int = 1, seed: int = SEED_DENSE,
          tol: float = 1e-6, precision: str = "mixed") -> Workload:
    s = SeededStream(seed)
    S = s.normal(M * M).reshape(M, M)
    K = s.normal(M * M).reshape(M, M)
    A = -(S @ S.T / M + 0.1 * np.eye(M)) + 0.5 * (K - K.T) / math.sqrt(M)
    y0 = np.stack([s.normal(M) for _ in range(batch)])
    return Workload(f"dense_M{M}_N{N}", "dense", M, 1, 0.0, T, N, ("rk4", fine_steps),
                    ("ie", coarse_steps), y0, A=A, tol=tol, precision=precision)


def with_source(w: Workload, seed: int = 0x50495405, amplitude: float = 1.0) -> Workload:
    """The workload with a seeded smooth time-independent source f (one per
    member): a few products of sine modes for grids, normal values scaled by
    1/sqrt(M) for dense operators."""
    s = SeededStream(seed)
    if w.kind in ("heat2d", "advdiff2d"):
        n = w.nx
        xs = np.arange(1, n + 1) / (n + 1.0)
        fs = []
        for _ in range(w.batch):
            kx = s.integers(1, 5, 3)
            ky = s.integers(1, 5, 3)
            a = s.normal(3)
            g = sum(a[i] * np.outer(np.sin(ky[i] * np.pi * xs), np.sin(kx[i] * np.pi * xs))
                    for i in range(3))
            fs.append(g.ravel())
        f = np.stack(fs)
    elif w.kind == "heat1d":
        xs = np.arange(1, w.M + 1) / (w.M + 1.0)
        f = np.stack([sum(s.normal(1)[0] * np.sin(k * np.pi * xs) for k in (1, 2, 5))
                      for _ in range(w.batch)])
    else:
        f = s.normal(w.batch * w.M).reshape(w.batch, w.M) / math.sqrt(w.M)
    return dataclasses.replace(w, f=amplitude * f, name=w.name + "_forced")


# The three test problems of Sec. 4 (eq. (9), read as
# y_t + u . grad y - div(mu grad y) + r y = 0 with y = 0 on the boundary):
# (mu, r, advection by the rotation u = (-y, x)).
PAPER_PDES = {
    "diffusion": (1.0, 0.0, False),
    "diffusion_reaction": (1.0, 1.5, False),
    "advection_diffusion_reaction": (0.1, 0.5, True),
}


def fem_p1_matrices(n: int, velocity: bool):
    """P1 finite elements on the centred unit square: n x n interior nodes of a
    uniform grid (h = 1/(n+1)), every cell cut along its diagonal from
    (x_i, y_j) to (x_i + h, y_j + h).  Returns the mass matrix Mm, the
    stiffness matrix K and the convection matrix C (C_ij = int phi_i u . grad
    phi_j with u = (-y, x), three-midpoint quadrature, exact here), all on the
    interior nodes (Dirichlet 0), dense, row-major node order j * n + i."""
    h = 1.0 / (n + 1)
    nn = n + 2                                   # nodes per side with the boundary
    xs = -0.5 + h * np.arange(nn)
    full = nn * nn
    Mm = np.zeros((full, full))
    K = np.zeros((full, full))
    C = np.zeros((full, full))
    area = h * h / 2.0
    Me = area / 12.0 * np.array([[2, 1, 1], [1, 2, 1], [1, 1, 2]])

    def add(nodes):
        P = np.array([[xs[i], xs[j]] for (i, j) in nodes])
        Bm = np.array([P[1] - P[0], P[2] - P[0]]).T          # columns: edges
        Binv = np.linalg.inv(Bm)
        # gradients of the barycentric functions
        g = np.array([-Binv[0] - Binv[1], Binv[0], Binv[1]])
        Ke = area * (g @ g.T)
        idx = [j * nn + i for (i, j) in nodes]
        Mm[np.ix_(idx, idx)] += Me
        K[np.ix_(idx, idx)] += Ke
        if velocity:
            mids = [(P[0] + P[1]) / 2, (P[1] + P[2]) / 2, (P[2] + P[0]) / 2]
            lam = [np.array([0.5, 0.5, 0.0]), np.array([0.0, 0.5, 0.5]), np.array([0.5, 0.0, 0.5])]
            Ce = np.zeros((3, 3))
            for q in range(3):
                ux, uy = -mids[q][1], mids[q][0]
                adv = g @ np.array([ux, uy])                 # u . grad phi_j
                Ce += (area / 3.0) * np.outer(lam[q], adv)
            C[np.ix_(idx, idx)] += Ce

    for j in range(nn - 1):
        for i in range(nn - 1):
            add([(i, j), (i + 1, j), (i + 1, j + 1)])
            add([(i, j), (i + 1, j + 1), (i, j + 1)])
    inner = np.array([j * nn + i for j in range(1, nn - 1) for i in range(1, nn - 1)])
    sel = np.ix_(inner, inner)
    return Mm[sel], K[sel], C[sel]


def paper_pde(pde: str = "diffusion", n: int = 49, N: int = 4, T: float = 6.4,
              dt: float = 1e-3, center: Tuple[float, float] = (0.2, 0.0),
              width: float = 0.1, batch: int = 1, tol: float = 1e-10,
              precision: str = "fp64", discretization: str = "fd") -> Workload:
    """A Sec. 4 test problem as a dense-operator workload.

    Unit square centred at the origin, n x n interior points of a grid with
    h = 1/(n+1) (n = 49: the paper's h = 2e-2), Dirichlet 0.  Finite
    differences stand in for the paper's finite elements: the 5-point
    Laplacian times mu, central differences for u . grad y, and -r y, as a
    dense M x M matrix A (M = n^2, row-major states).  Fine propagator:
    backward Euler with the paper's dt = 1e-3 (round(T / (N dt)) steps per
    slice); coarse: one backward-Euler step per slice.  y0: a Gaussian of
    standard deviation `width` at `center` (off the centre, so that the
    rotation moves it).  discretization = "fem": P1 finite elements (the
    paper's discretisation, `fem_p1_matrices`), the semi-discrete system
    Mm y' = -(mu K + C + r Mm) y written as y' = A y with
    A = -Mm^{-1}(mu K + C) - r I, so that backward Euler on it is the
    mass-matrix step (Mm + dt (mu K + C + r Mm)) y+ = Mm y.
    """
    mu, r, adv = PAPER_PDES[pde]
    h = 1.0 / (n + 1)
    xs = -0.5 + h * np.arange(1, n + 1)
    M = n * n
    if discretization == "fem":
        Mm, K, C = fem_p1_matrices(n, adv)
        A = -np.linalg.solve(Mm, mu * K + C) - r * np.eye(M)
        X, Y = np.meshgrid(xs, xs, indexing="xy")
        g = np.exp(-((X - center[0]) ** 2 + (Y - center[1]) ** 2) / (2.0 * width ** 2)).ravel()
        m = max(1, int(round(T / (N * dt))))
        return Workload(f"paper_{pde}_fem_n{n}_N{N}", "dense", M, 1, 0.0, T, N, ("ie", m),
                        ("ie", 1), np.tile(g, (batch, 1)), A=A, tol=tol, precision=precision)
    if discretization != "fd":
        raise ValueError(discretization)
    A = np.zeros((M, M))
    idx = np.arange(M).reshape(n, n)          # idx[j, i]: point (x_i, y_j)
    diag = -4.0 * mu / h ** 2 - r
    A[idx.ravel(), idx.ravel()] = diag
    for dj, di in ((0, 1), (0, -1), (1, 0), (-1, 0)):
        j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        jj, ii = j + dj, i + di
        ok = (jj >= 0) & (jj < n) & (ii >= 0) & (ii < n)
        rows = idx[j[ok], i[ok]]
        cols = idx[jj[ok], ii[ok]]
        val = np.full(rows.shape, mu / h ** 2)
        if adv:
            # -(u_x dy/dx + u_y dy/dy), u = (-y, x), central differences
            ux = -xs[j[ok]]
            uy = xs[i[ok]]
            if di != 0:
                val = val - ux * di / (2.0 * h)
            else:
                val = val - uy * dj / (2.0 * h)
        A[rows, cols] += val
    X, Y = np.meshgrid(xs, xs, indexing="xy")
    g = np.exp(-((X - center[0]) ** 2 + (Y - center[1]) ** 2) / (2.0 * width ** 2)).ravel()
    y0 = np.tile(g, (batch, 1))
    m = max(1, int(round(T / (N * dt))))
    return Workload(f"paper_{pde}_n{n}_N{N}", "dense", M, 1, 0.0, T, N, ("ie", m), ("ie", 1),
                    y0, A=A, tol=tol, precision=precision)


def serving_request(j: int, rate: float = 200.0, seed: int = SEED_SERVING,
                    m1d: Tuple[int, int] = (63, 4095), n2d: Tuple[int, int] = (32, 256),
                    nslices: Tuple[int, int] = (16, 1024),
                    nu_range: Tuple[float, float] = (1e-3, 1e-1)) -> Tuple[float, Workload]:
    """Request ``j`` of the serving stream: (inter-arrival gap in s, workload).

    Half the requests are 1D heat (IE fine, 100 steps per slice), half 2D heat
    (RK4 fine, m = max(50, ceil(dT nu / (0.2 h^2)))); T = 1; coarse = IE 1 step.
    """
    s = SeededStream(seed + j)
    gap = -math.log(1.0 - float(s.uniform(1)[0])) / rate
    is2d = bool(s.uniform(1)[0] >= 0.5)
    N = int(s.integers(nslices[0], nslices[1], 1)[0])
    nu = float(math.exp(s.uniform(1, math.log(nu_range[0]), math.log(nu_range[1]))[0]))
    if not is2d:
        M = int(s.integers(m1d[0], m1d[1], 1)[0])
        x = np.arange(1, M + 1) / (M + 1.0)
        kk = s.integers(1, 8, 4)
        a = s.normal(4)
        u = sum(a[i] / kk[i] * np.sin(kk[i] * np.pi * x) for i in range(4))
        w = Workload(f"req{j}_heat1d_M{M}_N{N}", "heat1d", M, 1, nu, 1.0, N, ("ie", 100),
                     ("ie", 1), u[None, :].copy(), tol=1e-6, precision="mixed")
    else:
        n = int(s.integers(n2d[0], n2d[1], 1)[0])
        h = 1.0 / (n + 1)
        m = max(50, int(math.ceil((1.0 / N) * nu / (0.2 * h * h))))
        u = gaussian_bumps(s, n, 4)
        w = Workload(f"req{j}_heat2d_{n}x{n}_N{N}", "heat2d", n, n, nu, 1.0, N, ("rk4", m),
                     ("ie", 1), u[None, :].copy(), tol=1e-6, precision="mixed")
    return gap, w


def serving_stream(count: int = 4096, rate: float = 200.0, seed: int = SEED_SERVING,
                   **kw) -> List[Workload]:
    """Poisson request stream; each workload's ``arrival`` is its arrival time (s)."""
    t = 0.0
    out = []
    for j in range(count):
        gap, w = serving_request(j, rate, seed, **kw)
        t += gap
        w.arrival = t
        out.append(w)
    return out
