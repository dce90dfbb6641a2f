"""Operator timing (pit_set_timing): with enable = 1 every operator class is
bracketed by events (the iterations replay one graph per iteration); with
enable = 2 only the launches outside the BiCGStab iterations are timed by
class and each launch of the iterations as a whole ("inner"), which then run
as the untimed loop graph.  Timing never changes a result."""
import numpy as np
import pytest

from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _solve(p, w, mode):
    X = torch.zeros((w.batch, w.N + 1, w.M), dtype=torch.float64, device="cuda")
    p.set_timing(mode)
    for _ in range(2):            # the second solve replays the captured graphs
        p.bicgstab_solve(X, tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    torch.cuda.synchronize()
    t = p.timing()
    p.set_timing(False)
    return X.cpu().numpy(), t


@pytest.mark.parametrize("kind", ["heat2d", "dense"])
def test_timing_modes_do_not_change_results(kind):
    from paper_2203_10148_gb300 import pit
    w = (inputs.heat2d(n=32, N=16, batch=2) if kind == "heat2d"
         else inputs.dense(M=128, N=16, T=10.0 * 16 / 4096))
    with pit.Problem(w, "mixed") as p:
        ref, t0 = _solve(p, w, 0)
        full, t1 = _solve(p, w, 1)
        top, t2 = _solve(p, w, 2)
    np.testing.assert_array_equal(full, ref)
    np.testing.assert_array_equal(top, ref)
    assert all(c == 0 for c, _ in t0.values())
    # every class inside the iterations is timed, nothing as a whole
    assert t1["fine_fp32"][0] > 0 and t1["krylov"][0] > 0 and t1["inner"][0] == 0
    # only the residuals, the sweeps outside the iterations and the
    # iterations as a whole
    assert t2["inner"][0] > 0 and t2["fine_fp32"][0] == 0
    assert t2["fine_split"][0] + t2["fine_ff"][0] > 0
    assert t2["inner"][1] > 0.0
