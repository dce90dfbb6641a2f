"""GPU parity of the heat-equation paths against the FP64 oracle.

Every test calls the CUDA path through the C-ABI (the ctypes binding) and
compares element by element with the oracle on the same seeded inputs.
Tolerances: FP64 path 1e-12 relative (operators to 1e-13); FP32 fine stepping
from FP64 inputs: m steps x 4 stages of FP32 rounding on O(1) data,
bounded here by 2e-5 relative; mixed-precision solves: 1e-6 against the
serial FP64 fine trajectory.
"""
import numpy as np
import pytest

from oracle import OracleProblem, parareal, pitsbicg
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _pit():
    from paper_2203_10148_gb300 import pit
    return pit


def _rand_block(w, seed, scale=1.0):
    s = inputs.SeededStream(seed)
    return (scale * s.normal(w.batch * (w.N + 1) * w.M)).reshape(w.batch, w.N + 1, w.M)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _oracle_apply(w, which, X):
    out = []
    for b in range(w.batch):
        o = OracleProblem.from_workload(w, member=b)
        x = X[b]
        if which == "F":
            out.append(o.apply_F(x))
        elif which == "Ginv":
            out.append(o.sweep_Ginv(x))
        elif which == "GinvF":
            out.append(o.apply_GinvF(x))
        else:
            out.append(o.residual(x))
    return np.stack(out)


# ------------------------------------------------------------------- 1D heat

HEAT1D_CASES = [dict(), dict(M=31, N=5, fine_steps=7), dict(M=100, N=3, fine_steps=20),
                dict(M=1, N=2, fine_steps=3), dict(M=257, N=9, fine_steps=11, batch=2),
                dict(M=2000, N=4, fine_steps=5), dict(M=4095, N=2, fine_steps=3)]


@pytest.mark.parametrize("case", HEAT1D_CASES)
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF", "residual"])
def test_heat1d_operators_fp64(case, which):
    pit = _pit()
    w = inputs.heat1d(**case)
    X = _rand_block(w, 1)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
        dev = p.apply(which, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = _oracle_apply(w, which, X)
    assert _rel(got, ref) < 1e-13
    np.testing.assert_array_equal(got, dev)


SMALL_CASES = [dict(M=1, N=3, fine_steps=4), dict(M=31, N=5, fine_steps=7),
               dict(M=63, N=16, fine_steps=100, batch=3), dict(M=63, N=400, fine_steps=5),
               dict(M=128, N=7, fine_steps=9, batch=2), dict(M=200, N=300, fine_steps=3),
               dict(M=256, N=4, fine_steps=6)]


PHI_CASES = [dict(M=63, N=16, fine_steps=100, batch=3), dict(M=31, N=5, fine_steps=7),
             dict(M=1, N=3, fine_steps=4), dict(M=250, N=5, fine_steps=400, batch=2)]


@pytest.mark.parametrize("case", PHI_CASES)
def test_heat1d_fine_propagator_matrix(case, monkeypatch):
    """Small grids with many fine steps: the FP64 fine batch as one product
    with Phi = A^{-m} (formed on the host by m Thomas solves of each unit
    vector) instead of m steps per slice; within 1e-13 of the oracle and of
    the stepping kernel (PIT_HEAT1D_PHI=0), for F, the residual and a solve."""
    pit = _pit()
    w = inputs.heat1d(**case)
    X = _rand_block(w, 73)
    out = {}
    for phi in ("1", "0"):
        monkeypatch.setenv("PIT_HEAT1D_PHI", phi)
        with pit.Problem(w, "fp64") as p:
            out[phi] = [p.apply(which, X) for which in ("F", "residual")]
    for which, g, t in zip(("F", "residual"), out["1"], out["0"]):
        ref = _oracle_apply(w, which, X)
        assert _rel(g, ref) < 1e-13, which
        assert _rel(g, t) < 1e-13, which


POW_CASES = [dict(), dict(M=31, N=5, fine_steps=7), dict(M=100, N=3, fine_steps=20, batch=2),
             dict(M=1, N=2, fine_steps=3), dict(M=63, N=40, fine_steps=10, batch=2)]


@pytest.mark.parametrize("case", POW_CASES)
def test_heat1d_sweep_through_powers(case, monkeypatch):
    """Small grids: the FP64 sweep as the independent products G^(n-k) q_k
    (G^j formed on the host by j coarse solves per column) summed over k in
    order, instead of N dependent solves; within 1e-13 of the oracle and of
    the sequential sweep (PIT_HEAT1D_POW=0), also in place (the solver's use)
    and through a converged solve."""
    pit = _pit()
    w = inputs.heat1d(**case)
    X = _rand_block(w, 79)
    out = {}
    for pw in ("1", "0"):
        monkeypatch.setenv("PIT_HEAT1D_POW", pw)
        with pit.Problem(w, "fp64") as p:
            out[pw] = [p.apply(which, X) for which in ("Ginv", "GinvF", "residual")]
            Xs, info = p.bicgstab_solve(tol=1e-10)
            out[pw].append(np.array(Xs))
    for which, g, t in zip(("Ginv", "GinvF", "residual"), out["1"], out["0"]):
        assert _rel(g, _oracle_apply(w, which, X)) < 1e-13, which
        assert _rel(g, t) < 1e-13, which
    assert _rel(out["1"][3], out["0"][3]) < 1e-11


@pytest.mark.parametrize("variant", ["warp", "cta"])
@pytest.mark.parametrize("case", SMALL_CASES)
def test_heat1d_small_grid_kernels(variant, case, monkeypatch):
    """Grids of M <= 256 points: the one-warp kernels (scan multipliers formed
    once per launch; E = 2, 4, 8 points per lane) and the CTA-wide scans,
    each in FP64, float-float and FP32, against the oracle."""
    monkeypatch.setenv("PIT_HEAT1D_SMALL", variant)
    monkeypatch.setenv("PIT_HEAT1D_PHI", "0")   # the steps, not the propagator matrix
    monkeypatch.setenv("PIT_HEAT1D_POW", "0")   # the sequential sweep, not the powers of G
    pit = _pit()
    w = inputs.heat1d(**case)
    X = _rand_block(w, 71)
    with pit.Problem(w, "mixed") as p:
        got = {which: p.apply(which, X, precision="fp64") for which in ("F", "Ginv", "residual")}
        ff = p.apply("F", X, precision="ff")
        f32 = p.apply("F", X, precision="mixed")
    for which, g in got.items():
        assert _rel(g, _oracle_apply(w, which, X)) < 1e-13, which
    refF = _oracle_apply(w, "F", X)
    assert _rel(ff, refF) < 1e-11
    assert _rel(f32, refF) < 2e-5


@pytest.mark.parametrize("which", ["F", "GinvF"])
def test_heat1d_operators_fp32_fine(which):
    pit = _pit()
    w = inputs.heat1d(M=63, N=8, fine_steps=100)
    X = _rand_block(w, 2)
    with pit.Problem(w, "mixed") as p:
        got = p.apply(which, X, precision="mixed")
    ref = _oracle_apply(w, which, X)
    assert _rel(got, ref) < 2e-5


@pytest.mark.parametrize("case", HEAT1D_CASES)
def test_heat1d_float_float_fine_matches_oracle(case):
    """The float-float Thomas recurrences (true residuals of the mixed path):
    within 1e-11 of the FP64 oracle for every thread layout (M = 1 .. 4095),
    the serial trajectory too."""
    pit = _pit()
    w = inputs.heat1d(**case)
    X = _rand_block(w, 61)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="ff")
        res = p.apply("residual", X, precision="ff")
        lam = p.serial_fine("ff")
    assert _rel(got, _oracle_apply(w, "F", X)) < 1e-11
    # the mixed residual's sweep is FP32-class (it only preconditions)
    assert _rel(res, _oracle_apply(w, "residual", X)) < max(2e-5, 3e-8 * w.M)
    for b in range(w.batch):
        assert _rel(lam[b], OracleProblem.from_workload(w, member=b).serial_fine()) < 1e-11


@pytest.mark.parametrize("resid", ["split", "fp64"])
def test_heat1d_mixed_solve_float_float_residual(resid):
    """Mixed 1D solves with float-float true residuals (split means
    float-float for this operator) reach the serial FP64 trajectory within
    1e-6 in the same refinement rounds as with FP64 residuals."""
    pit = _pit()
    w = inputs.heat1d(M=1000, N=64)
    lam = OracleProblem.from_workload(w).serial_fine()
    opts = dict(tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(residual_precision=resid, **opts)
        X64, info64 = p.bicgstab_solve(residual_precision="fp64", **opts)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6
    assert info[0]["refinements"] == info64[0]["refinements"]


def test_heat1d_bicgstab_fixed_iterations_match_oracle():
    """Same k iterations of Algorithm 1: iterates agree to 1e-12."""
    pit = _pit()
    w = inputs.heat1d()
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "fp64") as p:
        for k in (1, 2, 3, 5):
            X, info = p.bicgstab_solve(tol=0.0, max_iter=k)
            Xo, oi = pitsbicg(o, tol=0.0, max_iter=k)
            assert info[0]["iterations"] == k and oi.iterations == k
            assert info[0]["matvecs"] == oi.matvecs
            assert _rel(X[0], Xo) < 1e-12


def test_heat1d_bicgstab_converged_matches_serial_and_oracle():
    pit = _pit()
    w = inputs.heat1d()
    o = OracleProblem.from_workload(w)
    lam = o.serial_fine()
    Xo, oi = pitsbicg(o, tol=1e-10)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-10, history_len=64)
        lam_gpu = p.serial_fine()
    assert info[0]["status"] == 0
    assert info[0]["iterations"] == oi.iterations
    assert _rel(X[0], Xo) < 1e-12
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-9
    assert _rel(lam_gpu[0], lam) < 1e-13
    h = info[0]["history"]
    assert len(h) == oi.iterations + 1
    np.testing.assert_allclose(h, oi.history, rtol=1e-9)


def test_heat1d_restart_paths_match_oracle():
    """eps0 = 1 forces the restart branch every iteration."""
    pit = _pit()
    w = inputs.heat1d(M=15, N=6, fine_steps=10)
    o = OracleProblem.from_workload(w)
    Xo, oi = pitsbicg(o, tol=1e-12, eps0=1.0, max_iter=200)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-12, eps0=1.0, max_iter=200)
    assert info[0]["restarts"] == oi.restarts and info[0]["iterations"] == oi.iterations
    assert _rel(X[0], Xo) < 1e-12


def test_heat1d_maxiter_and_x0_modes():
    pit = _pit()
    w = inputs.heat1d(M=31, N=8, fine_steps=10)
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-30, max_iter=2)
        assert info[0]["status"] == pit.PIT_E_MAXITER and info[0]["iterations"] == 2
        Xz, iz = p.bicgstab_solve(tol=0.0, max_iter=3, x0="zero")
        X0 = _rand_block(w, 5, 0.1)
        Xg, ig = p.bicgstab_solve(X=X0.copy(), tol=0.0, max_iter=3, x0="given")
    assert _rel(Xz[0], pitsbicg(o, tol=0.0, max_iter=3, x0="zero")[0]) < 1e-12
    assert _rel(Xg[0], pitsbicg(o, tol=0.0, max_iter=3, x0=X0[0])[0]) < 1e-12


def test_heat1d_parareal_matches_oracle_and_is_exact_at_N():
    pit = _pit()
    w = inputs.heat1d()
    o = OracleProblem.from_workload(w)
    lam = o.serial_fine()
    with pit.Problem(w, "fp64") as p:
        for k in (1, 4):
            X, info = p.parareal_solve(kmax=k)
            Xo, _ = parareal(o, kmax=k)
            assert _rel(X[0], Xo) < 1e-12
            assert _rel(X[0][:k + 1], lam[:k + 1]) < 1e-12
        X, info = p.parareal_solve(kmax=w.N)
    assert _rel(X[0], lam) < 1e-12
    assert info[0]["matvecs"] == w.N + 1


def test_heat1d_batch_members_are_independent():
    pit = _pit()
    w = inputs.heat1d(M=63, N=8, fine_steps=20, batch=3)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-11)
    for b in range(3):
        with pit.Problem(w.member(b), "fp64") as p1:
            Xb, ib = p1.bicgstab_solve(tol=1e-11)
        np.testing.assert_array_equal(X[b], Xb[0])
        assert info[b]["iterations"] == ib[0]["iterations"]


# ------------------------------------------------------------------- 2D heat

HEAT2D_CASES = [dict(n=16, N=4, fine_steps=5), dict(n=20, N=3, fine_steps=7),
                dict(n=5, N=2, fine_steps=3), dict(n=37, N=3, fine_steps=4, batch=2),
                dict(n=128, N=2, fine_steps=3), dict(n=100, N=2, fine_steps=2)]


@pytest.mark.parametrize("case", HEAT2D_CASES)
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF", "residual"])
def test_heat2d_operators_fp64(case, which):
    pit = _pit()
    w = inputs.heat2d(**case, precision="fp64")
    X = _rand_block(w, 3)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, torch.from_numpy(X).cuda()).cpu().numpy()
    ref = _oracle_apply(w, which, X)
    assert _rel(got, ref) < 1e-12


@pytest.mark.parametrize("case", HEAT2D_CASES[:4])
@pytest.mark.parametrize("which", ["F", "Ginv"])
def test_heat2d_operators_mixed(case, which):
    pit = _pit()
    w = inputs.heat2d(**case)
    X = _rand_block(w, 4)
    with pit.Problem(w, "mixed") as p:
        got = p.apply(which, X, precision="mixed")
    ref = _oracle_apply(w, which, X)
    assert _rel(got, ref) < 2e-5


def test_heat2d_fp64_bicgstab_fixed_iterations():
    pit = _pit()
    w = inputs.heat2d(n=24, N=8, fine_steps=10, precision="fp64")
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "fp64") as p:
        for k in (1, 3):
            X, info = p.bicgstab_solve(tol=0.0, max_iter=k)
            Xo, _ = pitsbicg(o, tol=0.0, max_iter=k)
            assert _rel(X[0], Xo) < 1e-11


def test_heat2d_mixed_solve_reaches_serial_fp64():
    pit = _pit()
    w = inputs.heat2d(n=32, N=16)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, history_len=16)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6
    assert info[0]["refinements"] >= 1


def test_block_reduce_matches_numpy():
    pit = _pit()
    s = inputs.SeededStream(12)
    for nb, M in ((1, 1), (5, 63), (17, 2049), (513, 300)):
        U = s.normal(nb * M).reshape(nb, M)
        V = s.normal(nb * M).reshape(nb, M)
        dot, norms, ninf = pit.block_reduce(torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda(), nb, M)
        assert dot == pytest.approx(float(np.sum(U * V)), rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(norms, np.linalg.norm(U, axis=1), rtol=1e-13)
        assert ninf == pytest.approx(np.linalg.norm(U, axis=1).max(), rel=1e-13)


@pytest.mark.parametrize("case", [dict(n=16, N=4, fine_steps=5), dict(n=37, N=3, fine_steps=40, batch=2),
                                  dict(n=128, N=3, fine_steps=400)])
def test_heat2d_float_float_fine_matches_oracle(case):
    """Float-float stepping (about 48 bits) agrees with the FP64 oracle to 1e-12
    (RK4-stable cases: dt nu 8/h^2 below 2.78, so rounding is not amplified)."""
    pit = _pit()
    w = inputs.heat2d(**case)
    X = _rand_block(w, 6)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="ff")
        lam = p.serial_fine("ff")
    assert _rel(got, _oracle_apply(w, "F", X)) < 1e-12
    assert _rel(lam[0], OracleProblem.from_workload(w).serial_fine()) < 1e-11


@pytest.mark.parametrize("resid", ["ff", "fp64"])
@pytest.mark.parametrize("tol_mode", ["r0", "rhs"])
def test_heat2d_mixed_residual_precisions_and_tol_modes(resid, tol_mode):
    pit = _pit()
    w = inputs.heat2d(n=32, N=16)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-8 if tol_mode == "rhs" else 1e-7, residual_precision=resid,
                                   tol_mode=tol_mode, inner_tol=1e-5)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6


def test_tol_mode_rhs_fp64_threshold():
    """PIT_TOL_RHS stops on ||R|| <= tol ||G^-1 B||; the oracle with the same
    absolute threshold takes the same iterations."""
    pit = _pit()
    w = inputs.heat1d()
    o = OracleProblem.from_workload(w)
    rhs = np.max(np.linalg.norm(o.coarse_prediction(), axis=1))
    Xo, oi = pitsbicg(o, tol=0.0, abs_tol=1e-9 * rhs)
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-9, tol_mode="rhs")
    assert info[0]["iterations"] == oi.iterations
    assert _rel(X[0], Xo) < 1e-12
