"""GPU parity of the periodic advection-diffusion path (cluster/DSMEM fine
kernel, band-parallel coarse sweep) against the FP64 oracle.

The coarse propagator on the GPU is a fixed linear approximation of the
implicit-Euler step (K Chebyshev steps on the Jacobi-scaled system from
x = b, interval [1 - rho, 1 + rho] with rho = max (D - 1)/D); it is restated
here in numpy on the oracle's assembled operator to check the sweep element
by element.  The solution of eq. (4) does not depend on G, so converged
solves are compared with the oracle's serial fine trajectory.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import OracleProblem, spatial_operator
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

K_CHEB = 8


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _rand(w, seed):
    return inputs.SeededStream(seed).normal(w.batch * (w.N + 1) * w.M).reshape(w.batch, w.N + 1, w.M)


def _jacobi_sweep(w, Q, K=K_CHEB):
    """z_0 = q_0, z_n = q_n + Gt z_{n-1}; Gt b = K Chebyshev steps for
    (I - dT L) x = b with diagonal scaling, from x = b (Saad, Iterative
    Methods for Sparse Linear Systems, Alg. 12.1)."""
    L = spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy)
    A = (sp.identity(w.M) - (w.T / w.N) * L).tocsr()
    D = A.diagonal()
    rho = np.max((D - 1) / D)
    theta, delta = 1.0, rho
    sigma = theta / delta
    Z = np.empty_like(Q)
    Z[0] = Q[0]
    for n in range(1, w.N + 1):
        b = Z[n - 1]
        x = b.copy()
        r = b - A @ x
        d = r / D / theta
        rk = 1.0 / sigma
        for k in range(K):
            x = x + d
            if k == K - 1:
                break
            r = r - A @ d
            rn = 1.0 / (2 * sigma - rk)
            d = rn * rk * d + (2 * rn / delta) * (r / D)
            rk = rn
        Z[n] = Q[n] + x
    return Z


CASES = [dict(n=32, N=3), dict(n=64, N=4, batch=2), dict(n=128, N=2)]


@pytest.mark.parametrize("case", CASES)
def test_advdiff_fine_operator_fp64_and_fp32(case):
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(T=0.5 * case["N"] / 256, **case)
    X = _rand(w, 1)
    ref = np.stack([OracleProblem.from_workload(w, member=b).apply_F(X[b]) for b in range(w.batch)])
    with pit.Problem(w, "mixed") as p:
        got64 = p.apply("F", X, precision="fp64")
        got32 = p.apply("F", X, precision="mixed")
        gotff = p.apply("F", X, precision="ff")
    assert _rel(got64, ref) < 1e-12
    assert _rel(got32, ref) < 2e-5
    # float-float: about 48 significant bits per operation
    assert _rel(gotff, ref) < 1e-11


@pytest.mark.parametrize("case", CASES)
def test_advdiff_sweep_matches_jacobi_restatement(case):
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(T=0.5 * case["N"] / 256, **case)
    X = _rand(w, 2)
    ref = np.stack([_jacobi_sweep(w.member(b) if w.batch > 1 else w, X[b]) for b in range(w.batch)])
    with pit.Problem(w, "mixed") as p:
        got64 = p.apply("Ginv", X, precision="fp64")
        got32 = p.apply("Ginv", X, precision="mixed")
    assert _rel(got64, ref) < 1e-12
    assert _rel(got32, ref) < 1e-5


def test_advdiff_solves_reach_serial_trajectory():
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(n=64, N=16, T=0.5 * 16 / 256)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "fp64") as p:
        X64, i64 = p.bicgstab_solve(tol=1e-11)
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-8, tol_mode="rhs", inner_tol=1e-5, residual_precision="fp64")
        lam_gpu = p.serial_fine("fp64")
        Xf, infof = p.bicgstab_solve(tol=1e-8, tol_mode="rhs", inner_tol=1e-5, residual_precision="ff")
        lam_ff = p.serial_fine("ff")
    assert i64[0]["status"] == 0 and info[0]["status"] == 0 and infof[0]["status"] == 0
    assert np.linalg.norm(X64[0] - lam) / np.linalg.norm(lam) < 1e-9
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6
    assert np.linalg.norm(Xf[0] - lam) / np.linalg.norm(lam) < 1e-6
    assert _rel(lam_gpu[0], lam) < 1e-12
    assert _rel(lam_ff[0], lam) < 1e-10


def test_advdiff_full_size_sampled():
    """512 x 512 periodic, N = 256, 13 RK4 steps: the 16-CTA-cluster FP32 and
    FP64 fine batches on sampled slices against the oracle."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d()
    o = OracleProblem.from_workload(w)
    X = _rand(w, 3)
    Xd = torch.from_numpy(X).cuda()
    with pit.Problem(w, "mixed") as p:
        Y32 = p.apply("F", Xd, precision="mixed").cpu().numpy()[0]
        Y64 = p.apply("F", Xd, precision="fp64").cpu().numpy()[0]
        Yff = p.apply("F", Xd, precision="ff").cpu().numpy()[0]
    rows = [1, 2, 128, 255, 256]
    ref = X[0][rows] - o.F(X[0][[r - 1 for r in rows]])
    assert _rel(Y64[rows], ref) < 1e-12
    assert _rel(Yff[rows], ref) < 1e-11
    assert _rel(Y32[rows], ref) < 1e-4


@pytest.mark.parametrize("case", [dict(n=64, N=3, batch=2), dict(n=128, N=2)])
def test_advdiff_float_float_fp32_coefficients(case, monkeypatch):
    """The workload's velocities are FP32 values, so every coefficient v / h
    is exact in FP32 and the float-float kernel reads them as such (their low
    parts are zero): the same results bit for bit as the general (hi, lo)
    kernel, and the oracle's within 1e-11."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(**case, T=0.5 * case["N"] / 256)
    assert np.array_equal(w.vx.astype(np.float32).astype(np.float64), w.vx)
    X = _rand(w, 91)
    monkeypatch.setenv("PIT_ADV_COEF32", "1")
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="ff")
    monkeypatch.setenv("PIT_ADV_COEF32", "0")
    with pit.Problem(w, "mixed") as p:
        gen = p.apply("F", X, precision="ff")
    assert np.array_equal(got, gen)
    ref = np.stack([OracleProblem.from_workload(w, member=b).apply_F(X[b]) for b in range(w.batch)])
    assert _rel(got, ref) < 1e-11
