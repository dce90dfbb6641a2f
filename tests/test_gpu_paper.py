"""The Sec. 4 test problems (eq. (9) on P1 finite elements as in the paper,
and on finite differences; backward-Euler fine propagator, which on the
finite-element system is the mass-matrix step; dense-operator mode) on the
GPU against the FP64 oracle:
the operators element by element, PiTSBiCG's and parareal's residual
histories iteration by iteration, and the Fig. 1 re-run driver."""
import numpy as np
import pytest

from oracle import OracleProblem, parareal, pitsbicg
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

PDES = list(inputs.PAPER_PDES)
DISC = ["fem", "fd"]


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


@pytest.mark.parametrize("disc", DISC)
@pytest.mark.parametrize("pde", PDES)
@pytest.mark.parametrize("which", ["F", "Ginv", "residual"])
def test_paper_operators_fp64(pde, which, disc):
    from paper_2203_10148_gb300 import pit
    w = inputs.paper_pde(pde, n=9, N=4, discretization=disc)
    X = inputs.SeededStream(41).normal((w.N + 1) * w.M).reshape(1, w.N + 1, w.M)
    o = OracleProblem.from_workload(w)
    ref = {"F": o.apply_F, "Ginv": o.sweep_Ginv, "residual": o.residual}[which](X[0])
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
    assert _rel(got[0], ref) < 1e-11


@pytest.mark.parametrize("disc", DISC)
@pytest.mark.parametrize("pde", PDES)
@pytest.mark.parametrize("N", [4, 8])
def test_paper_residual_histories_match_oracle(pde, N, disc):
    """Residual ||G^{-1}(B - F X^k)||_{N,inf} of PiTSBiCG (recursive, per
    iteration) and of parareal (per correction) against the oracle's runs of
    Algorithm 1 and eq. (6), while above 1e-9 of the first residual."""
    from paper_2203_10148_gb300 import pit
    w = inputs.paper_pde(pde, n=9, N=N, discretization=disc)
    o = OracleProblem.from_workload(w)
    _, oi = pitsbicg(o, tol=1e-12, max_iter=N + 2)
    with pit.Problem(w, "fp64") as p:
        _, gi = p.bicgstab_solve(tol=1e-12, max_iter=N + 2, history_len=N + 4)
        ph = []
        for k in range(0, 4):
            _, pinfo = p.parareal_solve(kmax=k, tol=0.0)
            ph.append(pinfo[0]["precond_resid"])
    hist = gi[0]["history"]
    ref = oi.history
    r0 = ref[0]
    for k in range(min(len(hist), len(ref))):
        if ref[k] < 1e-9 * r0:
            break
        assert abs(hist[k] - ref[k]) <= 1e-9 * r0 + 1e-9 * ref[k], (k, hist[k], ref[k])
    _, opi = parareal(o, kmax=3)
    for k in range(4):
        assert abs(ph[k] - opi.history[k]) <= 1e-10 * r0 + 1e-9 * opi.history[k], (k, ph[k], opi.history[k])


def test_paper_fig1_driver_small():
    """The re-run driver at h = 0.1 (n = 9): both methods' residuals fall, and
    the histories it reports have the matvec counts of Sec. 4."""
    from paper_2203_10148_gb300 import paper_fig1
    for pde, disc in zip(PDES, ["fem", "fd", "fem"]):
        r = paper_fig1.run(pde, N=8, n=9, discretization=disc)
        b, q = r["pitsbicg"], r["parareal"]
        assert b["residual"][-1] < 1e-8 * b["residual"][0]
        assert q["residual"][-1] < q["residual"][0]
        assert b["matvecs"][:3] == [1, 3, 5] and q["matvecs"][:3] == [1, 2, 3]
        assert len(b["residual"]) == len(b["matvecs"])


@pytest.mark.parametrize("disc", DISC)
def test_paper_mixed_solve_reaches_serial(disc):
    """The mixed path on a paper problem (FP32 products, float-float or FP64
    residual) within 1e-6 of the FP64 serial trajectory."""
    from paper_2203_10148_gb300 import pit
    w = inputs.paper_pde("advection_diffusion_reaction", n=15, N=8, precision="mixed",
                         discretization=disc)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-9, tol_mode="rhs", inner_tol=1e-5)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6


def test_paper_fem_full_size_operator_sampled():
    """The paper's size (h = 2e-2: n = 49, M = 2401, dt = 1e-3, T = 6.4) at
    N = 16: one application of F on the GPU against the oracle's mass-matrix
    backward Euler, on three sampled slices."""
    from paper_2203_10148_gb300 import pit
    w = inputs.paper_pde("advection_diffusion_reaction", n=49, N=16, discretization="fem")
    assert w.M == 2401 and w.fine == ("ie", 400)
    X = inputs.SeededStream(43).normal((w.N + 1) * w.M).reshape(1, w.N + 1, w.M)
    with pit.Problem(w, "fp64") as p:
        got = p.apply("F", X)[0]
    o = OracleProblem.from_workload(w)
    for i in (1, 7, 16):
        ref = X[0, i] - o.F(X[0, i - 1:i])[0]
        assert _rel(got[i], ref) < 1e-10, i
