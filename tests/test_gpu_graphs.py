"""Each BiCGStab iteration replayed as a captured CUDA graph: results, solver
statistics, per-class timing counts and the kernel-launch count equal those
of eager launches (PIT_GRAPHS=0), bit for bit."""
import os

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


def _pit():
    from paper_2203_10148_gb300 import pit
    return pit


def _solve(w, precision, graphs, timing=False, device=False, **kw):
    pit = _pit()
    old = os.environ.get("PIT_GRAPHS")
    os.environ["PIT_GRAPHS"] = "1" if graphs else "0"
    try:
        p = pit.Problem(w, precision)
    finally:
        if old is None:
            del os.environ["PIT_GRAPHS"]
        else:
            os.environ["PIT_GRAPHS"] = old
    with p:
        if timing:
            p.set_timing(True)
        k0 = pit.kernel_launches()
        if device:
            X = torch.zeros((w.batch, w.N + 1, w.M), dtype=torch.float64, device="cuda")
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                X, info = p.bicgstab_solve(X, stream=s.cuda_stream, **kw)
            torch.cuda.synchronize()
            X = X.cpu().numpy()
        else:
            X, info = p.bicgstab_solve(**kw)
        launches = pit.kernel_launches() - k0
        tm = p.timing() if timing else None
    return X, info, launches, tm


CASES = [
    ("heat2d", dict(n=32, N=16), "mixed", dict(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")),
    ("heat2d", dict(n=24, N=8, fine_steps=10, batch=3), "fp64", dict(tol=1e-10)),
    ("heat1d", dict(), "fp64", dict(tol=1e-10)),
    ("heat1d", dict(N=40), "mixed", dict(tol=1e-8, inner_tol=1e-5)),
    ("heat2d", dict(n=200, N=64, fine_steps=50), "mixed", dict(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")),
]


@pytest.mark.parametrize("kind,kw,prec,opts", CASES)
def test_graph_replay_matches_eager(kind, kw, prec, opts):
    w = getattr(inputs, kind)(**kw)
    Xe, ie, le, _ = _solve(w, prec, graphs=False, **opts)
    Xg, ig, lg, _ = _solve(w, prec, graphs=True, **opts)
    assert ie[0]["status"] == 0
    assert np.array_equal(Xe, Xg)
    for a, b in zip(ie, ig):
        for k in ("iterations", "matvecs", "restarts", "refinements", "status"):
            assert a[k] == b[k], k
    assert ie[0]["graph_iterations"] == 0
    assert ig[0]["graph_iterations"] > 0
    assert le == lg


def test_graph_replay_timing_classes_and_device_stream():
    w = inputs.heat2d(n=48, N=32)
    opts = dict(tol=1e-7, inner_tol=1e-5, tol_mode="rhs")
    Xe, ie, _, te = _solve(w, "mixed", graphs=False, timing=True, device=True, **opts)
    Xg, ig, _, tg = _solve(w, "mixed", graphs=True, timing=True, device=True, **opts)
    assert np.array_equal(Xe, Xg)
    assert ig[0]["graph_iterations"] > 0
    for cls in te:
        assert te[cls][0] == tg[cls][0], cls
        if tg[cls][0]:
            assert tg[cls][1] > 0.0, cls
