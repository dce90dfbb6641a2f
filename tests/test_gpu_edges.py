"""Degenerate and extreme sizes on the GPU against the FP64 oracle.

* one time slice (N = 1: two blocks, one fine propagation) for every
  operator kind, operators and a converged solve;
* the smallest 2D grids (n = 1, 2, 3: tiles mostly outside the grid);
* the largest 1D grid one CTA holds (M = 8192) and the sizes just past each
  kind's limit, which must be refused with PIT_E_UNSUPPORTED;
* a given initial guess that already solves eq. (4) (no iteration needed).
Tolerances as everywhere: FP64 1e-12, FP32 fine 2e-5.
"""
import numpy as np
import pytest

from oracle import OracleProblem
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


def _rand_block(w, seed):
    s = inputs.SeededStream(seed)
    return s.normal(w.batch * (w.N + 1) * w.M).reshape(w.batch, w.N + 1, w.M)


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _oracle_apply(w, which, X):
    out = []
    for b in range(w.batch):
        o = OracleProblem.from_workload(w, member=b)
        fn = {"F": o.apply_F, "Ginv": o.sweep_Ginv, "GinvF": o.apply_GinvF,
              "residual": o.residual}[which]
        out.append(fn(X[b]))
    return np.stack(out)


ONE_SLICE = {
    "heat1d": lambda prec: inputs.heat1d(M=40, N=1, fine_steps=20),
    "heat2d": lambda prec: inputs.heat2d(n=24, N=1, fine_steps=30, precision=prec),
    "dense": lambda prec: inputs.dense(M=64, N=1, T=10.0 / 4096, fine_steps=200, precision=prec),
    "advdiff": lambda prec: inputs.advdiff2d(n=32, N=1, T=0.5 / 256, fine_steps=4, precision=prec),
}


@pytest.mark.parametrize("kind", list(ONE_SLICE))
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF", "residual"])
def test_one_slice_operators_fp64(kind, which):
    pit = _pit()
    w = ONE_SLICE[kind]("fp64")
    assert w.N == 1
    X = _rand_block(w, 61)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
    assert _rel(got, _oracle_apply(w, which, X)) < 1e-12


@pytest.mark.parametrize("kind", list(ONE_SLICE))
def test_one_slice_solves(kind):
    """With N = 1 the exact solution is (y0, F y0): FP64 within 1e-12, the
    mixed path (where the kind has one) within 1e-6."""
    pit = _pit()
    w = ONE_SLICE[kind]("fp64")
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "fp64") as p:
        X, info = p.bicgstab_solve(tol=1e-13)
    assert info[0]["status"] == 0
    assert _rel(X[0], lam) < 1e-12
    if kind != "heat1d":
        wm = ONE_SLICE[kind]("mixed")
        with pit.Problem(wm, "mixed") as p:
            Xm, im = p.bicgstab_solve(tol=1e-9, inner_tol=1e-5, tol_mode="rhs")
        assert im[0]["status"] == 0
        assert _rel(Xm[0], lam) < 1e-6


@pytest.mark.parametrize("n", [1, 2, 3])
@pytest.mark.parametrize("which", ["F", "Ginv", "residual"])
def test_smallest_2d_grids(n, which):
    pit = _pit()
    w = inputs.heat2d(n=n, N=3, fine_steps=4, precision="fp64")
    X = _rand_block(w, 62)
    ref = _oracle_apply(w, which, X)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
    assert _rel(got, ref) < 1e-12
    wm = inputs.heat2d(n=n, N=3, fine_steps=4)
    with pit.Problem(wm, "mixed") as p:
        g32 = p.apply(which, X, precision="mixed")
    assert _rel(g32, ref) < 2e-5


@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF"])
def test_largest_1d_grid(which):
    """M = 8192, the largest grid one CTA of the 1D kernels holds."""
    pit = _pit()
    w = inputs.heat1d(M=8192, N=3, fine_steps=5)
    X = _rand_block(w, 63)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
    assert _rel(got, _oracle_apply(w, which, X)) < 1e-12


@pytest.mark.parametrize("make", [lambda: inputs.heat1d(M=8193, N=2, fine_steps=2),
                                  lambda: inputs.heat2d(n=257, N=2, fine_steps=2),
                                  lambda: inputs.advdiff2d(n=48, N=2, T=0.01)])
def test_sizes_past_the_limits_are_refused(make):
    pit = _pit()
    w = make()
    with pytest.raises(pit.PitError) as e:
        pit.Problem(w, "mixed" if w.kind != "heat1d" else "fp64")
    assert e.value.status == pit.PIT_E_UNSUPPORTED


@pytest.mark.parametrize("kind", ["heat1d", "heat2d", "dense"])
def test_given_exact_solution_needs_no_iteration(kind):
    """X0 = the serial fine trajectory solves eq. (4): the initial residual is
    at rounding level and the solve returns it unchanged after 0 iterations."""
    pit = _pit()
    w = {"heat1d": lambda: inputs.heat1d(M=31, N=6, fine_steps=10),
         "heat2d": lambda: inputs.heat2d(n=16, N=6, fine_steps=10, precision="fp64"),
         "dense": lambda: inputs.dense(M=32, N=6, T=1.0, fine_steps=20, precision="fp64")}[kind]()
    with pit.Problem(w, "fp64") as p:
        lam = p.serial_fine("fp64")
        X, info = p.bicgstab_solve(X=lam.copy(), x0="given", tol=1e-8, tol_mode="rhs")
    assert info[0]["iterations"] == 0 and info[0]["status"] == 0
    assert np.array_equal(X, lam)
