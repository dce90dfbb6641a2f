"""The Krylov kernels' cluster reductions: a block of 2 to 8 chunks of 2048
values is one thread-block cluster whose CTAs add their partial sums in
distributed shared memory, in chunk order, so that one partial per block
reaches global memory (PIT_KRYLOV_CLUSTERS=1).  The order of additions is
that of the per-chunk partials (the default), so the solves agree bit for
bit."""
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


@pytest.mark.parametrize("n,N,batch,prec", [(64, 16, 2, "mixed"), (128, 8, 3, "mixed"),
                                            (100, 6, 1, "fp64"), (45, 9, 2, "fp64")])
def test_cluster_reductions_equal_chunk_partials(n, N, batch, prec, monkeypatch):
    """M = 4096 (2 chunks), 16384 (8), 10000 (5) and 2025 (1: no cluster)."""
    from paper_2203_10148_gb300 import pit
    w = inputs.heat2d(n=n, N=N, T=N / 512, batch=batch, precision=prec)
    out = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("PIT_KRYLOV_CLUSTERS", flag)
        with pit.Problem(w, prec) as p:
            X, info = p.bicgstab_solve(tol=1e-9 if prec == "fp64" else 1e-7, tol_mode="rhs",
                                       inner_tol=1e-5)
        out[flag] = (X, [(i["iterations"], i["matvecs"], i["precond_resid"]) for i in info])
    np.testing.assert_array_equal(out["1"][0], out["0"][0])
    assert out["1"][1] == out["0"][1]
