"""Serving runtime (pit_server_* / pit_serve_*) on the GPU.

A served result must be the same alone and in the mix: each request of a
mixed stream (1D and 2D heat of different N and grid size, submitted at once
so that their solves overlap on the device) is compared with the same
problem solved alone through pit_bicgstab_solve, and with the serial FP64
fine trajectory of the oracle, which is the exact solution of the
all-at-once system (Section 2, Eq. 4): mixed-precision solves match it
within 1e-6 relative.
"""
import numpy as np
import pytest

from oracle import OracleProblem
from paper_2203_10148_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# solve options of every served request (tolerance relative to ||G^-1 B||)
OPTS = dict(tol=1e-7, inner_tol=1e-5, tol_mode="rhs", residual_precision="ff")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _pit():
    from paper_2203_10148_gb300 import pit
    return pit


def _small_stream(count, first=0):
    """Requests of the serving stream at sizes the oracle finishes in seconds."""
    return [inputs.serving_request(first + j, m1d=(63, 400), n2d=(32, 96),
                                   nslices=(16, 96))[1] for j in range(count)]


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_served_equals_solo_and_oracle():
    pit = _pit()
    ws = _small_stream(12)
    kinds = {w.kind for w in ws}
    assert kinds == {"heat1d", "heat2d"}
    with pit.Server(max_slots=4) as srv:
        tickets = [srv.submit(w, **OPTS) for w in ws]
        results = [srv.wait(t, timeout=300.0) for t in tickets]
        stats = srv.stats()
    bad = [(w.name, r[0] if r else None, r[2][0].get("error") if r else None) for w, r in zip(ws, results)
           if r is None or r[0] != pit.PIT_OK]
    assert not bad, bad   # (request, status, the library's error message)
    assert stats["completed"] == len(ws) and stats["failed"] == 0
    assert stats["max_running"] >= 2, "requests submitted together must overlap"
    for w, res in zip(ws, results):
        st, X, info = res
        assert info[0]["latency_seconds"] >= info[0]["queue_seconds"] >= 0.0
        assert 0 < info[0]["device_bytes"] <= pit.serve_footprint(w), w.name
        with pit.Problem(w) as p:
            Xs, _ = p.bicgstab_solve(**OPTS)
        assert _rel(X, Xs) <= 1e-6, w.name
        lam = OracleProblem.from_workload(w).serial_fine()
        assert _rel(X[0], lam) <= 1e-6, (w.name, _rel(X[0], lam))


def test_served_grid_sizes_alternate_concurrently():
    """2D heat requests of two grid sizes, solved eight at a time: the same
    kernels launch at once with different shared-memory sizes from different
    worker threads.  The kernels' shared-memory limit belongs to the process,
    so a worker that lowered it under another's launch would fail that
    launch; every request must succeed and equal its solo solve."""
    pit = _pit()
    sizes = (40, 96)
    ws = [inputs.heat2d(n=sizes[j % 2], N=16, fine_steps=20) for j in range(32)]
    with pit.Server(max_slots=8) as srv:
        tickets = [srv.submit(w, **OPTS) for w in ws]
        results = [srv.wait(t, timeout=300.0) for t in tickets]
        stats = srv.stats()
    bad = [(w.name, r[0] if r else None, r[2][0].get("error") if r else None) for w, r in zip(ws, results)
           if r is None or r[0] != pit.PIT_OK]
    assert not bad, bad
    assert stats["max_running"] >= 2, "requests submitted together must overlap"
    for n in sizes:
        w = next(w for w in ws if w.nx == n)
        with pit.Problem(w) as p:
            Xs, _ = p.bicgstab_solve(**OPTS)
        for wj, (st, X, info) in zip(ws, results):
            if wj.nx == n:
                assert _rel(X, Xs) <= 1e-6, wj.name


@pytest.mark.parametrize("resid", ["ff", "split"])
def test_served_bitwise_equals_solo(resid):
    """Kernels, launch shapes and reduction orders depend on the request
    alone, so the served iterate is bit for bit the solo one, with
    float-float and with split RK4 true residuals (the library default)."""
    pit = _pit()
    ws = _small_stream(6, first=100)
    opts = dict(OPTS, residual_precision=resid)
    with pit.Server(max_slots=3) as srv:
        tickets = [srv.submit(w, **opts) for w in ws]
        results = [srv.wait(t, timeout=300.0) for t in tickets]
    for w, (st, X, _) in zip(ws, results):
        assert st == pit.PIT_OK, w.name
        with pit.Problem(w) as p:
            Xs, _ = p.bicgstab_solve(**opts)
        assert np.array_equal(X, Xs), w.name
        if resid == "split":
            lam = OracleProblem.from_workload(w).serial_fine()
            assert _rel(X[0], lam) <= 1e-6, (w.name, _rel(X[0], lam))


def test_budget_admission_and_queueing():
    """With room for about one large request at a time, admission keeps the
    reserved footprints within the budget and requests wait in the queue."""
    pit = _pit()
    ws = _small_stream(8, first=200)
    fp = [pit.serve_footprint(w) for w in ws]
    budget = int(1.2 * max(fp))
    with pit.Server(hbm_budget_bytes=budget, max_slots=4) as srv:
        tickets = [srv.submit(w, **OPTS) for w in ws]
        results = [srv.wait(t, timeout=300.0) for t in tickets]
        stats = srv.stats()
    bad = [(w.name, r[0], r[2][0]) for w, r in zip(ws, results) if r is None or r[0] != pit.PIT_OK]
    assert not bad, bad
    assert stats["hbm_reserved_peak"] <= budget
    assert stats["hbm_reserved"] == 0 and stats["running"] == 0
    assert stats["completed"] == len(ws)
    assert stats["queue_p99"] > 0.0
    assert stats["latency_p50"] <= stats["latency_p99"]


def test_over_budget_and_unsupported_rejected_at_submit():
    pit = _pit()
    w = _small_stream(1)[0]
    with pit.Server(hbm_budget_bytes=pit.serve_footprint(w) - 1, max_slots=1) as srv:
        with pytest.raises(pit.PitError) as e:
            srv.submit(w, **OPTS)
        assert e.value.status == pit.PIT_E_NOMEM
        adv = inputs.advdiff2d(n=32, N=4)
        with pytest.raises(pit.PitError) as e:
            srv.submit(adv, **OPTS)
        assert e.value.status == pit.PIT_E_UNSUPPORTED


def test_nonfinite_request_fails_alone():
    """A request with a NaN in y0 reports PIT_E_NONFINITE; the others finish."""
    pit = _pit()
    ws = _small_stream(3, first=300)
    bad = ws[1]
    bad.y0 = bad.y0.copy()
    bad.y0[0, 3] = np.nan
    with pit.Server(max_slots=2) as srv:
        tickets = [srv.submit(w, **OPTS) for w in ws]
        res = [srv.wait(t, timeout=300.0) for t in tickets]
    assert res[0][0] == pit.PIT_OK and res[2][0] == pit.PIT_OK
    assert res[1][0] == pit.PIT_E_NONFINITE


def test_cancel_queued_and_running():
    pit = _pit()
    big = inputs.serving_request(7, m1d=(63, 400), n2d=(96, 128), nslices=(600, 1000))[1]
    small = _small_stream(2, first=400)
    with pit.Server(max_slots=1) as srv:
        t_big = srv.submit(big, **OPTS)
        t_q = srv.submit(small[0], **OPTS)     # waits behind the big one (one slot)
        srv.cancel(t_q)
        st_q = srv.wait(t_q, timeout=60.0)
        assert st_q[0] == pit.PIT_E_CANCELLED
        srv.cancel(t_big)                      # queued or running: either way it stops
        st_b = srv.wait(t_big, timeout=300.0)
        assert st_b[0] in (pit.PIT_E_CANCELLED, pit.PIT_OK)
        t_ok = srv.submit(small[1], **OPTS)    # the server keeps serving
        st_ok = srv.wait(t_ok, timeout=300.0)
        assert st_ok[0] == pit.PIT_OK
        with pytest.raises(pit.PitError):
            srv.poll(t_ok)                     # the result was released
        s = srv.stats()
    assert s["cancelled"] >= 1


def test_poll_pending_then_done():
    pit = _pit()
    w = inputs.serving_request(11, n2d=(96, 128), nslices=(300, 400))[1]
    with pit.Server(max_slots=1) as srv:
        t = srv.submit(w, **OPTS)
        first = srv.poll(t)
        out = srv.wait(t, timeout=300.0)
    assert out is not None and out[0] == pit.PIT_OK
    assert first is None or first[0] == pit.PIT_OK


def test_open_loop_poisson_stream():
    """Requests submitted at Poisson arrival times (one client thread) while
    earlier ones run; statistics count every request once."""
    import time
    pit = _pit()
    ws = _small_stream(24, first=500)
    for j, w in enumerate(ws):
        w.arrival = 0.002 * j
    with pit.Server(max_slots=4) as srv:
        t0 = time.perf_counter()
        tickets = []
        for w in ws:
            while time.perf_counter() - t0 < w.arrival:
                time.sleep(0.0005)
            tickets.append(srv.submit(w, **OPTS))
        res = [srv.wait(t, timeout=300.0) for t in tickets]
        s = srv.stats(reset=True)
        s2 = srv.stats()
    bad = [(w.name, r[0], r[2][0]) for w, r in zip(ws, res) if r[0] != pit.PIT_OK]
    assert not bad, bad
    assert s["completed"] == len(ws) and s["submitted"] == len(ws)
    assert s["solves_per_s"] > 0 and s["slice_steps_per_s"] > 0
    assert s["latency_p99"] >= s["latency_p50"] > 0
    assert s2["completed"] == 0 and s2["submitted"] == 0
