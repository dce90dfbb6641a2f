"""GPU parity of the periodic advection-diffusion path (cluster/DSMEM fine
kernel, band-parallel coarse sweep) against the FP64 oracle.

The coarse propagator is implicit Euler with its linear solve replaced by K
Chebyshev steps (the workload's ``coarse_inner``); the oracle states that
operator in ``oracle.chebyshev_ie_propagator`` (pinned against the closed
Chebyshev form and the exact implicit-Euler step in the oracle pins), so the
sweep, the operators and fixed-k iterates of Algorithm 1 are compared with
the oracle element by element.  The solution of eq. (4) does not depend on G,
so converged solves are also compared with the serial fine trajectory.
"""
import numpy as np
import pytest

from oracle import OracleProblem, pitsbicg
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


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


def _oracle_sweep(w, X):
    return np.stack([OracleProblem.from_workload(w, member=b).sweep_Ginv(X[b])
                     for b in range(w.batch)])


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
def test_advdiff_sweep_matches_oracle(case):
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(T=0.5 * case["N"] / 256, **case)
    X = _rand(w, 2)
    ref = _oracle_sweep(w, X)
    with pit.Problem(w, "mixed") as p:
        got64 = p.apply("Ginv", X, precision="fp64")
        got32 = p.apply("Ginv", X, precision="mixed")
    assert _rel(got64, ref) < 1e-12
    assert _rel(got32, ref) < 1e-5


@pytest.mark.parametrize("K", [1, 2, 3, 24, 64])
def test_advdiff_sweep_chebyshev_count(K):
    """The coarse step's Chebyshev count is part of the problem: every count
    from 1 to the maximum gives the oracle's operator."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(n=64, N=3, T=0.5 * 3 / 256, coarse_inner=K)
    X = _rand(w, 12)
    ref = _oracle_sweep(w, X)
    with pit.Problem(w, "fp64") as p:
        got = p.apply("Ginv", X, precision="fp64")
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("case", [dict(n=64, N=6), dict(n=128, N=4, coarse_inner=24)])
def test_advdiff_bicgstab_fixed_iterations_match_oracle(case):
    """k iterations of Algorithm 1 in FP64 (k = 1, 2, 3): the iterates agree
    with the oracle's to 1e-12 and the matvec counts are identical."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(T=0.5 * case["N"] / 256, precision="fp64", **case)
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "fp64") as p:
        for k in (1, 2, 3):
            X, info = p.bicgstab_solve(tol=0.0, max_iter=k)
            Xo, oi = pitsbicg(o, tol=0.0, max_iter=k)
            assert info[0]["iterations"] == k and oi.iterations == k
            assert info[0]["matvecs"] == oi.matvecs
            assert _rel(X[0], Xo) < 1e-12


def test_advdiff_bicgstab_converged_matches_oracle_iterations():
    """Converged FP64 solve: the same iteration count as the oracle's
    Algorithm 1 and the serial fine trajectory within the tolerance."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(n=64, N=8, T=0.5 * 8 / 256, precision="fp64")
    o = OracleProblem.from_workload(w)
    lam = o.serial_fine()
    Xo, oi = pitsbicg(o, tol=1e-10)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-10)
    assert info[0]["status"] == 0 and oi.status == "ok"
    assert info[0]["iterations"] == oi.iterations
    assert _rel(X[0], Xo) < 1e-10
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-8


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


@pytest.mark.parametrize("n,N,batch", [(256, 3, 2), (512, 2, 1)])
def test_advdiff_sweep_large_grids(n, N, batch):
    """Bands of 2 (n = 256) and 4 rows (n = 512, the workload's grid): the
    FP64 and FP32 sweeps against the oracle's operator."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(n=n, N=N, T=0.5 * N / 256, batch=batch)
    X = _rand(w, 31)
    ref = _oracle_sweep(w, X)
    with pit.Problem(w, "mixed") as p:
        got64 = p.apply("Ginv", X, precision="fp64")
        got32 = p.apply("Ginv", X, precision="mixed")
    assert _rel(got64, ref) < 1e-12
    assert _rel(got32, ref) < 1e-5


@pytest.mark.parametrize("n,N,batch", [(256, 2, 2), (512, 2, 1)])
def test_advdiff_fine_wide_tiles_match(n, N, batch, monkeypatch):
    """8 x 8 thread tiles (PIT_ADV_RX=8: n/2 threads per CTA, for n >= 256)
    against the default 8 x 4 tiles: every point takes the same operations
    on the same operands (rows r and r + 4 share a packed pair in both), so
    the FP32, float-float and FP64 fine operators agree bit for bit, and
    with the oracle."""
    from paper_2203_10148_gb300 import pit
    w = inputs.advdiff2d(n=n, N=N, T=0.5 * N / 256, batch=batch)
    X = _rand(w, 17)
    out = {}
    for rx in ("4", "8"):
        monkeypatch.setenv("PIT_ADV_RX", rx)
        with pit.Problem(w, "mixed") as p:
            out[rx] = [p.apply("F", X, precision=pr) for pr in ("mixed", "ff", "fp64")]
    for a, b in zip(out["4"], out["8"]):
        np.testing.assert_array_equal(a, b)
    ref = np.stack([OracleProblem.from_workload(w, member=b).apply_F(X[b]) for b in range(w.batch)])
    assert _rel(out["8"][2], ref) < 1e-12
    assert _rel(out["8"][1], ref) < 1e-11
