"""The split RK4 arithmetic (PIT_SPLIT) of the 2D heat fine propagator: each
RK4 step's first-order term Z u (Z = dt L) in float-float, the higher-order
terms Z^2 u/2 + Z^3 u/6 + Z^4 u/24 in FP32, the state in float-float.

Error bound written into the tests: with z = 8 nu dt / h^2 >= ||Z||, the
FP32 terms have size at most q(z) = z^2/2 + z^3/6 + z^4/24 times |u|, and
their rounding (a few FP32 units, 2^-24 each) costs at most about
4 * 2^-24 * q(z) |u| per step, so m steps stay within m times that plus the
float-float part (2^-44 per operation).  On smooth data the higher-order
terms are much smaller than this worst case (they scale with the square of
the mode's own |Z|): on the workload's Gaussian bumps the split serial
trajectory stays within 1e-9 of the oracle's (measured 2.5e-11 at 64^2,
N = 8; 2.3e-10 at 128^2, N = 16; 7.3e-11 in the 2-norm at 128^2, N = 512)
after hundreds of steps, where the white-noise bound is about 3e-10 per
step at the workload's z = 0.052.  Steps with z > 1/8 run
the float-float kernel (bit for bit).
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


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300)


def _rand_block(w, seed):
    s = inputs.SeededStream(seed)
    return s.normal(w.batch * (w.N + 1) * w.M).reshape(w.batch, w.N + 1, w.M)


def _z(w):
    h = 1.0 / (w.nx + 1)
    return 8.0 * w.nu * (w.T / w.N / w.fine[1]) / h ** 2


def _bound(w):
    z = _z(w)
    q = z * z / 2 + z ** 3 / 6 + z ** 4 / 24
    return w.fine[1] * 4 * 2.0 ** -24 * q + 1e-12


def _oracle_F(w, X):
    return np.stack([OracleProblem.from_workload(w, member=b).apply_F(X[b]) for b in range(w.batch)])


# z = 0.048, 0.028, 0.114 (near the 1/8 limit), 0.052 (the workload's), 0.101, 0.104
CASES = [dict(n=16, N=4, fine_steps=120), dict(n=37, N=3, T=3 / 512, fine_steps=8, batch=2),
         dict(n=100, N=2, T=2 / 512, fine_steps=14), dict(n=128, N=3, T=3 / 512),
         dict(n=160, N=3, T=3 / 512, fine_steps=40, batch=2), dict(n=256, N=2, T=2 / 512, fine_steps=100)]


@pytest.mark.parametrize("case", CASES)
def test_split_fine_on_white_noise_within_the_bound(case):
    """One-CTA (n <= 128) and cluster (n > 128) kernels, ragged tiles, batch
    2: white-noise input, the worst case for the FP32 terms."""
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(**case)
    assert _z(w) <= 0.125
    X = _rand_block(w, 71)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="split")
        gff = p.apply("F", X, precision="ff")
    ref = _oracle_F(w, X)
    assert _rel(got, ref) < _bound(w)
    assert _rel(gff, ref) < 1e-12
    assert not np.array_equal(got, gff)          # the split kernel ran


@pytest.mark.parametrize("case", [dict(n=64, N=8, T=8 / 512), dict(n=128, N=16, T=16 / 512),
                                  dict(n=192, N=4, T=4 / 512)])
def test_split_serial_trajectory_on_smooth_data(case):
    """The serial fine trajectory from the workload's smooth initial value
    (Gaussian bumps) over 400 to 800 steps: the split arithmetic agrees with
    the oracle to 1e-9, far inside the white-noise bound."""
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(**case)
    assert _z(w) <= 0.125
    ref = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        lam = p.serial_fine("split")[0]
    assert _rel(lam, ref) < 1e-9


def test_split_large_steps_run_float_float():
    """z > 1/8: the float-float kernel, bit for bit."""
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(n=48, N=4, fine_steps=20)
    assert 0.125 < _z(w) < 2.78                  # RK4-stable
    X = _rand_block(w, 72)
    with pit.Problem(w, "mixed") as p:
        np.testing.assert_array_equal(p.apply("F", X, precision="split"),
                                      p.apply("F", X, precision="ff"))


@pytest.mark.parametrize("n,N", [(32, 16), (128, 64), (192, 8)])
def test_split_true_residual_solves_within_1e6(n, N):
    """Mixed solves with split true residuals reach the serial FP64
    trajectory within 1e-6, in as many refinement rounds as float-float, and
    the two solutions agree to the solve tolerance (1e-7)."""
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(n=n, N=N, T=N / 512)
    lam = OracleProblem.from_workload(w).serial_fine()
    opts = dict(tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(residual_precision="split", **opts)
        Xf, infof = p.bicgstab_solve(residual_precision="ff", **opts)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6
    assert info[0]["refinements"] == infof[0]["refinements"]
    assert _rel(X[0], Xf[0]) < 1e-7
