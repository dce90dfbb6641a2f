"""Tensor-core sine transforms of the 2D heat coarse sweep (G^{-1} of
eq. (7) in the sine basis, split-TF32 tcgen05 products) against the FP64
oracle and against the FP32-pipe transforms they replace.

Grids 96 <= n <= 256 (n % 4 == 0) use them in the mixed path (one 128^2
output tile per block with S resident up to n = 128, 2 x 2 tiles with S
streamed beyond); both kinds of input are covered (FP64 blocks, converted first, and the FP32 rows of the
fine kernel), single and several tiles per CTA (N + 1 above the SM count:
both accumulators and every stage parity reused), batches, and solves that
mask converged members.  Tolerances: 2e-5 against the oracle, as for every
FP32 sweep; 1e-5 between the two FP32-class transforms.

The per-mode recurrence between the transforms runs in one pass per mode
when members x modes reach 2^16 (n = 256 here, n = 192 with two members,
the 128^2 bench batch) and as the chunked scan below that (the other
cases); both against the oracle.
"""
import numpy as np
import pytest

from oracle import OracleProblem
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [dict(n=128, N=3, fine_steps=3), dict(n=100, N=2, fine_steps=2, batch=2),
         dict(n=96, N=4, fine_steps=2), dict(n=124, N=2, fine_steps=3),
         # 2 x 2 output tiles per block, S streamed with A
         dict(n=256, N=3, fine_steps=3), dict(n=160, N=2, fine_steps=2, batch=2),
         dict(n=132, N=2, fine_steps=2), dict(n=200, N=3, fine_steps=2)]


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
        fn = {"Ginv": o.sweep_Ginv, "GinvF": o.apply_GinvF}[which]
        out.append(fn(X[b]))
    return np.stack(out)


def _apply(w, which, X, tc, monkeypatch):
    monkeypatch.setenv("PIT_HEAT2D_TC", "1" if tc else "0")
    pit = _pit()
    with pit.Problem(w, "mixed") as p:
        return p.apply(which, X, precision="mixed")


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("which", ["Ginv", "GinvF"])
def test_tc_sweep_matches_oracle_and_fp32_pipe(case, which, monkeypatch):
    w = inputs.heat2d(**case)
    X = _rand_block(w, 51)
    got = _apply(w, which, X, True, monkeypatch)
    ref = _oracle_apply(w, which, X)
    assert _rel(got, ref) < 2e-5
    alt = _apply(w, which, X, False, monkeypatch)
    assert _rel(got, alt) < 1e-5
    again = _apply(w, which, X, True, monkeypatch)
    assert np.array_equal(got, again)


@pytest.mark.parametrize("n,N", [(128, 300), (256, 80)])
def test_tc_sweep_many_tiles_per_cta(n, N, monkeypatch):
    """More output tiles than SMs (301 blocks of 128^2; 81 blocks of 256^2 =
    324 tiles) on one launch of at most one CTA per SM: every CTA walks
    several tiles, both accumulators and every stage parity are reused."""
    w = inputs.heat2d(n=n, N=N, fine_steps=2)
    X = _rand_block(w, 52)
    got = _apply(w, "Ginv", X, True, monkeypatch)
    alt = _apply(w, "Ginv", X, False, monkeypatch)
    assert _rel(got, alt) < 1e-5
    o = OracleProblem.from_workload(w)
    # the first 41 slices of the recurrence z_n = q_n + G(z_{n-1}) of eq. (7)
    ref = [X[0][0]]
    for k in range(1, 41):
        ref.append(X[0][k] + o.G(ref[-1][None, :])[0])
    assert _rel(got[0][:41], np.stack(ref)) < 2e-5


@pytest.mark.parametrize("case", [dict(n=128, N=24, fine_steps=50, batch=2),
                                  dict(n=112, N=16, fine_steps=40),
                                  dict(n=192, N=16, fine_steps=80, batch=2)])
def test_tc_mixed_solve_reaches_serial(case, monkeypatch):
    """Mixed solves whose sweeps run on the tensor cores: every member within
    1e-6 of the FP64 serial fine trajectory (converged members are masked)."""
    monkeypatch.setenv("PIT_HEAT2D_TC", "1")
    pit = _pit()
    w = inputs.heat2d(**case)
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")
    for b in range(w.batch):
        assert info[b]["status"] == 0
        lam = OracleProblem.from_workload(w, member=b).serial_fine()
        assert _rel(X[b], lam) < 1e-6
