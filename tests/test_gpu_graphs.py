"""The BiCGStab iterations replayed from captured CUDA graphs: results,
solver statistics, per-class timing counts and the kernel-launch count equal
those of eager launches (PIT_GRAPHS=0), bit for bit.

Two graph forms: the loop graph (a conditional while node around the
captured iteration and a one-warp condition kernel; PIT_GRAPH_LOOP = k
iterations per launch, the default 16) and, where it does not apply (event
timing, a per-iteration residual history) or PIT_GRAPH_LOOP=0, one graph
launch per iteration.  The loop graph adds exactly one kernel (the condition)
per replayed iteration."""
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


def _solve(w, precision, graphs, timing=False, device=False, loop=None, **kw):
    pit = _pit()
    env = {"PIT_GRAPHS": "1" if graphs else "0"}
    if loop is not None:
        env["PIT_GRAPH_LOOP"] = str(loop)
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        p = pit.Problem(w, precision)
    finally:
        for k, v in old.items():
            if v is None:
                del os.environ[k]
            else:
                os.environ[k] = v
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


@pytest.mark.parametrize("loop", [0, 1, 3, None])
@pytest.mark.parametrize("kind,kw,prec,opts", CASES)
def test_graph_replay_matches_eager(kind, kw, prec, opts, loop):
    w = getattr(inputs, kind)(**kw)
    Xe, ie, le, _ = _solve(w, prec, graphs=False, **opts)
    Xg, ig, lg, _ = _solve(w, prec, graphs=True, loop=loop, **opts)
    assert ie[0]["status"] == 0
    assert np.array_equal(Xe, Xg)
    for a, b in zip(ie, ig):
        for k in ("iterations", "matvecs", "restarts", "refinements", "status"):
            assert a[k] == b[k], k
    assert ie[0]["graph_iterations"] == 0
    assert ig[0]["graph_iterations"] > 0
    # the loop graph's condition kernel runs once per replayed iteration
    assert lg == le + (0 if loop == 0 else ig[0]["graph_iterations"])


def test_loop_graph_many_iterations_and_members():
    """A batch whose members converge at different iterations, with more
    iterations than one loop-graph launch runs (the host relaunches): the
    same iterates and statistics as eager launches."""
    w = inputs.heat1d(M=63, N=48, batch=5)
    opts = dict(tol=1e-12)
    Xe, ie, le, _ = _solve(w, "fp64", graphs=False, **opts)
    Xg, ig, lg, _ = _solve(w, "fp64", graphs=True, loop=2, **opts)
    assert np.array_equal(Xe, Xg)
    assert [a["iterations"] for a in ie] == [b["iterations"] for b in ig]
    assert max(a["iterations"] for a in ie) > 4
    assert lg == le + ig[0]["graph_iterations"]


def test_history_keeps_per_iteration_graphs():
    """With a residual history (recorded by the host after every iteration)
    the solve replays one graph per iteration: no condition kernels."""
    pit = _pit()
    w = inputs.heat1d(N=24)
    with pit.Problem(w, "fp64") as p:
        k0 = pit.kernel_launches()
        X1, i1 = p.bicgstab_solve(tol=1e-10)
        l1 = pit.kernel_launches() - k0
        k0 = pit.kernel_launches()
        X2, i2 = p.bicgstab_solve(tol=1e-10, history_len=64)
        l2 = pit.kernel_launches() - k0
    assert np.array_equal(X1, X2)
    assert i1[0]["iterations"] == i2[0]["iterations"]
    hist = i2[0]["history"]
    assert 2 <= len(hist) <= i2[0]["iterations"] + 1 and hist[-1] < hist[0]
    assert i2[0]["graph_iterations"] == i1[0]["graph_iterations"] > 0
    assert l1 == l2 + i1[0]["graph_iterations"]


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
