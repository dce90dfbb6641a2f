"""Problems with a time-independent source, y' = L y + f (eq. (1) with
f != 0): B = (y0, c, ..., c) with c = F_f(0), the offset of the affine fine
propagator.  The GPU's residuals, serial trajectories and solves against the
oracle, which steps the affine propagators directly."""
import numpy as np
import pytest

from oracle import OracleProblem, parareal
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


def _cases():
    return [
        inputs.with_source(inputs.heat1d(M=31, N=6, fine_steps=20)),
        inputs.with_source(inputs.heat1d(M=40, N=5, fine_steps=12, batch=2)),
        inputs.with_source(inputs.heat2d(n=16, N=4, fine_steps=20, precision="fp64")),
        inputs.with_source(inputs.heat2d(n=20, N=3, fine_steps=30, batch=2, precision="fp64")),
        inputs.with_source(inputs.dense(M=24, N=5, T=1.0, fine_steps=37)),
        inputs.with_source(inputs.paper_pde("advection_diffusion_reaction", n=7, N=4)),
    ]


@pytest.mark.parametrize("idx", range(6))
def test_source_residual_and_serial_match_oracle(idx):
    from paper_2203_10148_gb300 import pit
    w = _cases()[idx]
    X = inputs.SeededStream(51).normal(w.batch * (w.N + 1) * w.M).reshape(w.batch, w.N + 1, w.M)
    with pit.Problem(w, "fp64") as p:
        res = p.apply("residual", X, precision="fp64")
        app = p.apply("F", X, precision="fp64")
        lam = p.serial_fine("fp64")
    for b in range(w.batch):
        o = OracleProblem.from_workload(w, member=b)
        assert _rel(res[b], o.residual(X[b])) < 1e-11
        assert _rel(app[b], o.apply_F(X[b])) < 1e-12        # the Krylov operator stays linear
        assert _rel(lam[b], o.serial_fine()) < 1e-11


@pytest.mark.parametrize("idx", range(6))
def test_source_solves_reach_forced_trajectory(idx):
    from paper_2203_10148_gb300 import pit
    w = _cases()[idx]
    o = OracleProblem.from_workload(w)
    lam = o.serial_fine()
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-12)
        Xp, _ = p.parareal_solve(kmax=w.N, tol=0.0)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-9
    assert _rel(Xp[0], lam) < 1e-11
    _, oinfo = parareal(o, kmax=w.N)
    if w.kind != "heat2d":
        w2 = inputs.dataclasses.replace(w, precision="mixed")
        with pit.Problem(w2, "mixed") as p:
            Xm, im = p.bicgstab_solve(tol=1e-9, tol_mode="rhs", inner_tol=1e-5)
        assert im[0]["status"] == 0
        assert np.linalg.norm(Xm[0] - lam) / np.linalg.norm(lam) < 1e-6


def test_source_mixed_heat2d_and_removal():
    from paper_2203_10148_gb300 import pit
    w = inputs.with_source(inputs.heat2d(n=32, N=16))
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
        assert info[0]["status"] == 0
        assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6
        p.set_source(None)                      # back to y' = L y
        lam0 = p.serial_fine("fp64")
    w0 = inputs.dataclasses.replace(w, f=None)
    assert _rel(lam0[0], OracleProblem.from_workload(w0).serial_fine()) < 1e-12


def test_source_errors():
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(n=16, N=4, fine_steps=20)
    with pit.Problem(w) as p:
        f = np.zeros((1, w.M))
        f[0, 3] = np.nan
        with pytest.raises(pit.PitError) as e:
            p.set_source(f)
        assert e.value.status == pit.PIT_E_NONFINITE
    adv = inputs.advdiff2d(n=32, N=2)
    with pit.Problem(adv) as p:
        with pytest.raises(pit.PitError) as e:
            p.set_source(np.ones((1, adv.M)))
        assert e.value.status == pit.PIT_E_UNSUPPORTED
    with pit.Server(max_slots=1) as srv:
        with pytest.raises(ValueError):
            srv.submit(inputs.with_source(w))
