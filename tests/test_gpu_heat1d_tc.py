"""1D heat coarse sweep in the sine basis on the tensor cores (mixed path):
G^{-1} of eq. (7) with the implicit-Euler step (I - dT nu D2)^{-1}, diagonal
in the discrete sine basis, as two split-TF32 transforms of all slices
around a per-mode recurrence over the slices.

Tolerance: each transform sums M products in FP32 on the tensor core, and
that accumulation error grows linearly with M (measured about 1.7e-8 M
relative, against 2.6e-5 at most for the sequential FP32 Thomas sweep at the
same sizes), so the bound is max(2e-5, 3e-8 M) against the FP64 oracle (the
sequential Thomas sweep) and that plus 4e-5 against the FP32 Thomas sweep it
replaces (PIT_HEAT1D_TC=0).  The sweep only preconditions: the mixed solves
below reach the FP64 serial trajectory within 1e-6 as with the Thomas sweep.
Grids from M = 16 to the largest one serving admits (4095: 32 x 9 output
tiles, more than one per SM), ragged M (not a multiple of the 32-wide
padding), batches, and mixed solves that mask converged members.
"""
import numpy as np
import pytest

from oracle import OracleProblem
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [dict(M=16, N=5, fine_steps=10), dict(M=63, N=16, fine_steps=100),
         dict(M=100, N=7, fine_steps=20, batch=2), dict(M=257, N=40, fine_steps=30),
         dict(M=1023, N=12, fine_steps=10), dict(M=4095, N=1024, fine_steps=2)]


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


def _apply(w, which, X, tc, monkeypatch):
    monkeypatch.setenv("PIT_HEAT1D_TC", "1" if tc else "0")
    pit = _pit()
    with pit.Problem(w, "mixed") as p:
        return p.apply(which, X, precision="mixed")


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("which", ["Ginv", "GinvF"])
def test_tc_sweep_matches_oracle_and_thomas(case, which, monkeypatch):
    w = inputs.heat1d(**case)
    X = _rand_block(w, 71)
    got = _apply(w, which, X, True, monkeypatch)
    ref = []
    for b in range(w.batch):
        o = OracleProblem.from_workload(w, member=b)
        ref.append({"Ginv": o.sweep_Ginv, "GinvF": o.apply_GinvF}[which](X[b]))
    tol = max(2e-5, 3e-8 * w.M)
    assert _rel(got, np.stack(ref)) < tol
    alt = _apply(w, which, X, False, monkeypatch)
    assert _rel(got, alt) < tol + 4e-5
    assert np.array_equal(got, _apply(w, which, X, True, monkeypatch))


@pytest.mark.parametrize("case", [dict(M=511, N=64, fine_steps=100, batch=2),
                                  dict(M=2047, N=256, fine_steps=100),
                                  dict(M=4095, N=128, fine_steps=100)])
def test_tc_mixed_solve_reaches_serial(case, monkeypatch):
    monkeypatch.setenv("PIT_HEAT1D_TC", "1")
    pit = _pit()
    w = inputs.heat1d(**case)
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")
    for b in range(w.batch):
        assert info[b]["status"] == 0
        lam = OracleProblem.from_workload(w, member=b).serial_fine()
        assert _rel(X[b], lam) < 1e-6
