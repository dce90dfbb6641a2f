"""2D heat on grids of 129..256 points per side: the thread-block-cluster
fine kernel (row bands per CTA, halo rows over distributed shared memory)
and the tiled sine transforms of the coarse sweep, against the FP64 oracle.

Cluster shapes covered: FP32 bands of 64 rows (3 or 4 CTAs per slice),
FP64 / float-float bands of 32 rows (5 to 8 CTAs), ragged n (not a multiple
of the band or of the 8-column thread tile), batches of two members.
Tolerances as for the one-CTA kernels: FP64 1e-12, FP32 2e-5, float-float
1e-12 on RK4-stable cases, mixed solves 1e-6 against the serial fine
trajectory.
"""
import numpy as np
import pytest

from oracle import OracleProblem
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CASES = [dict(n=160, N=3, fine_steps=4), dict(n=256, N=2, fine_steps=3),
         dict(n=201, N=2, fine_steps=3, batch=2), dict(n=129, N=3, fine_steps=2)]


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


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF", "residual"])
def test_cluster_operators_fp64(case, which):
    pit = _pit()
    w = inputs.heat2d(**case, precision="fp64")
    X = _rand_block(w, 31)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, torch.from_numpy(X).cuda()).cpu().numpy()
    assert _rel(got, _oracle_apply(w, which, X)) < 1e-12


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF"])
def test_cluster_operators_mixed(case, which):
    pit = _pit()
    w = inputs.heat2d(**case)
    X = _rand_block(w, 32)
    with pit.Problem(w, "mixed") as p:
        got = p.apply(which, X, precision="mixed")
    assert _rel(got, _oracle_apply(w, which, X)) < 2e-5


@pytest.mark.parametrize("case", [dict(n=256, N=2, fine_steps=8, nu=5e-5),
                                  dict(n=160, N=3, fine_steps=6, nu=1e-4, batch=2)])
def test_cluster_float_float_fine(case):
    """RK4-stable cases (dt nu 8/h^2 below 2.78)."""
    pit = _pit()
    w = inputs.heat2d(**case)
    h = 1.0 / (w.nx + 1)
    assert w.nu * (w.T / w.N / w.fine[1]) * 8 / h ** 2 < 2.78
    X = _rand_block(w, 33)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="ff")
        lam = p.serial_fine("ff")
    assert _rel(got, _oracle_apply(w, "F", X)) < 1e-12
    assert _rel(lam[0], OracleProblem.from_workload(w).serial_fine()) < 1e-11


def test_cluster_serial_fine_fp64():
    pit = _pit()
    w = inputs.heat2d(n=192, N=4, fine_steps=5, nu=1e-4, precision="fp64")
    with pit.Problem(w, "fp64") as p:
        lam = p.serial_fine()
    assert _rel(lam[0], OracleProblem.from_workload(w).serial_fine()) < 1e-12


def test_cluster_mixed_solve_reaches_serial_fp64():
    pit = _pit()
    w = inputs.heat2d(n=192, N=16, fine_steps=120)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")
    assert info[0]["status"] == 0
    assert _rel(X[0], lam) < 1e-6


def test_cluster_served_equals_solo():
    """Large-grid requests through the server, overlapped with small ones."""
    pit = _pit()
    ws = [inputs.serving_request(j, n2d=(129, 256), nslices=(16, 48), m1d=(63, 300))[1]
          for j in range(4)]
    ws += [inputs.serving_request(50 + j, n2d=(32, 64), nslices=(16, 48))[1] for j in range(4)]
    opts = dict(tol=1e-7, inner_tol=1e-5, tol_mode="rhs", residual_precision="ff")
    with pit.Server(max_slots=4) as srv:
        tickets = [srv.submit(w, **opts) for w in ws]
        res = [srv.wait(t, timeout=600.0) for t in tickets]
    for w, (st, X, _) in zip(ws, res):
        assert st == pit.PIT_OK, w.name
        with pit.Problem(w) as p:
            Xs, _ = p.bicgstab_solve(**opts)
        assert np.array_equal(X, Xs), w.name


@pytest.mark.parametrize("variants", ["0,0", "1,0", "2,2", "3,0"])
@pytest.mark.parametrize("case", [dict(n=128, N=3, fine_steps=3), dict(n=100, N=2, fine_steps=4, batch=2),
                                  dict(n=37, N=3, fine_steps=4)])
def test_fine_variants_small_grids(variants, case, monkeypatch):
    """Every fine-kernel variant for n <= 128 (one CTA of 4- or 8-column tiles
    of 8 rows, one CTA of 4 x 4 tiles, a cluster of 8 x 4 tiles) matches the
    oracle and the others bit for bit."""
    pit = _pit()
    monkeypatch.setenv("PIT_HEAT2D_VARIANTS", variants)
    w = inputs.heat2d(**case)
    X = _rand_block(w, 34)
    with pit.Problem(w, "mixed") as p:
        g32 = p.apply("F", X, precision="mixed")
        gff = p.apply("F", X, precision="ff")
    ref = _oracle_apply(w, "F", X)
    assert _rel(g32, ref) < 2e-5
    assert _rel(gff, ref) < 1e-11 or w.nu * (w.T / w.N / w.fine[1]) * 8 * (w.nx + 1) ** 2 >= 2.78
    monkeypatch.setenv("PIT_HEAT2D_VARIANTS", "0,0")
    with pit.Problem(w, "mixed") as p:
        b32 = p.apply("F", X, precision="mixed")
        bff = p.apply("F", X, precision="ff")
    assert np.array_equal(g32, b32)
    assert np.array_equal(gff, bff)


@pytest.mark.parametrize("case", [dict(n=256, N=2, fine_steps=3), dict(n=160, N=3, fine_steps=2, batch=2),
                                  dict(n=201, N=2, fine_steps=3), dict(n=129, N=2, fine_steps=2)])
def test_wide_clusters_equal_narrow_ones(case, monkeypatch):
    """For n > 128 the clusters of 4-column tiles (512 threads, thread rows of
    two warps whose boundary columns go through shared memory) give the
    8-column clusters' results bit for bit, FP32 and float-float, and match
    the oracle."""
    pit = _pit()
    w = inputs.heat2d(**case)
    X = _rand_block(w, 35)
    out = {}
    for big in ("0,0", "1,1"):
        monkeypatch.setenv("PIT_HEAT2D_VARIANTS", "0,0," + big)
        with pit.Problem(w, "mixed") as p:
            out[big] = (p.apply("F", X, precision="mixed"), p.apply("F", X, precision="ff"))
    assert np.array_equal(out["0,0"][0], out["1,1"][0])
    assert np.array_equal(out["0,0"][1], out["1,1"][1])
    ref = _oracle_apply(w, "F", X)
    assert _rel(out["1,1"][0], ref) < 2e-5
