"""Full-size parity on the benchmark workload (2D heat 128 x 128, N = 512,
50 RK4 fine steps per slice): the GPU against the oracle's own Algorithm 1
run stored in tests/golden/oracle_solve_heat2d_128_N512.json (written by
tests/golden/make_oracle_solve_heat2d.py, which calls only oracle/).
Compared: iteration and matvec counts, the residual history, and sampled
solution values (every 64th slice at 16 points), on the launch
configuration bench.py times."""
import json
import os

import numpy as np
import pytest

from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
GOLD = os.path.join(os.path.dirname(__file__), "golden", "oracle_solve_heat2d_128_N512.json")


@pytest.fixture(scope="module")
def gold():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return json.load(open(GOLD))


def _samples(X, g):
    return np.array([[X[n, i] for i in g["sample_points"]] for n in g["sample_slices"]])


def test_fp64_path_matches_oracle_at_full_size(gold):
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d()
    with pit.Problem(w, "fp64") as p:
        X = torch.zeros((1, w.N + 1, w.M), dtype=torch.float64, device="cuda")
        X, info = p.bicgstab_solve(X, tol=1e-6, history_len=64)
        lam = p.serial_fine("fp64")
    Xh = X.cpu().numpy()[0]
    assert info[0]["iterations"] == gold["iterations"]
    assert info[0]["matvecs"] == gold["matvecs"]
    np.testing.assert_allclose(info[0]["history"], gold["history"], rtol=1e-9)
    ref = np.array(gold["X_samples"])
    assert np.abs(_samples(Xh, gold) - ref).max() <= 1e-12 * np.abs(ref).max()
    sref = np.array(gold["serial_samples"])
    assert np.abs(_samples(lam[0], gold) - sref).max() <= 1e-12 * np.abs(sref).max()


def test_mixed_path_full_size_within_1e6(gold):
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d()
    with pit.Problem(w, "mixed") as p:
        X = torch.zeros((1, w.N + 1, w.M), dtype=torch.float64, device="cuda")
        X, info = p.bicgstab_solve(X, tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    Xh = X.cpu().numpy()[0]
    sref = np.array(gold["serial_samples"])
    assert info[0]["status"] == 0
    assert np.abs(_samples(Xh, gold) - sref).max() <= 1e-6 * np.abs(sref).max()
