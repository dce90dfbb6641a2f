"""Mixed solves into host buffers: the solution's copy to host memory starts
while its own true residual is checked, and a refinement round that goes on
waits for that copy before it changes the solution.  Whatever the number of
rounds, and for pinned as for pageable host memory, the caller's buffer must
hold exactly what a solve into device memory returns."""
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


def _solve(w, out, **kw):
    from paper_2203_10148_gb300 import pit
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(out, **kw)
    return (X.cpu().numpy() if torch.is_tensor(X) else np.array(X)), info


@pytest.mark.parametrize("tol,refine_max", [(1e-7, 8), (1e-13, 3)])
@pytest.mark.parametrize("make", ["device", "pinned", "pageable"])
def test_host_buffers_match_device_solve(tol, refine_max, make):
    """tol = 1e-13 is below what the mixed path reaches: every allowed round
    runs (each after an early copy that the next round supersedes) and the
    solve ends at refine_max; the returned X is the last round's."""
    w = inputs.heat2d(n=32, N=16, batch=2)
    shape = (w.batch, w.N + 1, w.M)
    kw = dict(tol=tol, tol_mode="rhs", refine_max=refine_max, inner_tol=1e-5)
    ref, rinfo = _solve(w, torch.zeros(shape, dtype=torch.float64, device="cuda"), **kw)
    if make == "device":
        out = torch.zeros(shape, dtype=torch.float64, device="cuda")
    elif make == "pinned":
        out = torch.zeros(shape, dtype=torch.float64).pin_memory().numpy()
    else:
        out = np.zeros(shape, dtype=np.float64)
    got, info = _solve(w, out, **kw)
    np.testing.assert_array_equal(got, ref)
    assert [i["refinements"] for i in info] == [i["refinements"] for i in rinfo]
    if tol < 1e-12:
        assert all(i["refinements"] == refine_max for i in info), info
    else:
        assert all(i["status_name"] == "ok" for i in info), info
