"""The C-ABI library loads and exports every symbol include/pit.h declares,
and its host-side argument validation rejects bad descriptors (no GPU needed:
validation runs before any CUDA call)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            text = open(os.path.join(ROOT, "include", h)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"\b(pit_[a-z0-9_]+)\s*\(", text)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2203_10148_gb300 import build, pit
    build.build()
    return pit.load()


def test_library_exports_every_declared_symbol(lib):
    from paper_2203_10148_gb300 import pit
    declared = _declared_functions()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(pit.EXPORTS) <= set(declared)


def test_every_environment_switch_is_documented():
    """Each environment variable the library reads is listed in the public
    header with its meaning."""
    csrc = os.path.join(ROOT, "paper_2203_10148_gb300", "csrc")
    names = set()
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h")):
            names |= set(re.findall(r'getenv\("([A-Z0-9_]+)"\)', open(os.path.join(csrc, f)).read()))
    assert names, "no getenv found"
    header = "".join(open(os.path.join(ROOT, "include", h)).read()
                     for h in os.listdir(os.path.join(ROOT, "include")) if h.endswith(".h"))
    assert sorted(n for n in names if n not in header) == []


def test_version_and_defaults(lib):
    from paper_2203_10148_gb300 import pit
    assert b"sm_103a" in lib.pit_version()
    o = pit.SolveOpts()
    lib.pit_default_opts(C.byref(o))
    assert o.tol == 1e-10 and o.restart_eps0 == 1e-8 and o.x0_mode == 0 and o.refine_max >= 1
    assert o.residual_precision == pit.PIT_SPLIT


def _desc(pit, y0, **kw):
    op = pit.OperatorDesc(kw.get("kind", 1), kw.get("nx", y0.size), kw.get("ny", 1),
                          kw.get("nu", 0.1), None, None, None)
    return pit.ProblemDesc(op, y0.ctypes.data_as(C.POINTER(C.c_double)), kw.get("batch", 1),
                           kw.get("T", 1.0), kw.get("N", 4),
                           pit.StepperDesc(1, kw.get("fine_steps", 10)), pit.StepperDesc(1, 1),
                           kw.get("precision", 0))


@pytest.mark.parametrize("bad", [dict(N=0), dict(T=0.0), dict(T=-1.0), dict(fine_steps=0),
                                 dict(kind=9), dict(batch=0), dict(precision=7), dict(ny=3),
                                 dict(nu=-1.0), dict(N=65535), dict(batch=65536)])
def test_create_rejects_invalid_descriptors(lib, bad):
    from paper_2203_10148_gb300 import pit
    y0 = np.ones(8)
    h = C.c_void_p()
    st = lib.pit_problem_create(C.byref(_desc(pit, y0, **bad)), C.byref(h))
    assert st == pit.PIT_E_INVALID
    assert "pit_problem_create" in pit.last_error()


def test_create_rejects_nonfinite_initial_value(lib):
    from paper_2203_10148_gb300 import pit
    y0 = np.ones(8)
    y0[3] = np.nan
    h = C.c_void_p()
    assert lib.pit_problem_create(C.byref(_desc(pit, y0)), C.byref(h)) == pit.PIT_E_NONFINITE


def test_null_arguments(lib):
    from paper_2203_10148_gb300 import pit
    assert lib.pit_problem_create(None, None) == pit.PIT_E_INVALID
    assert lib.pit_problem_destroy(None) == pit.PIT_OK
    assert lib.pit_apply_operator(None, 1, 0, None, None, 0, None) == pit.PIT_E_INVALID
    assert lib.pit_bicgstab_solve(None, None, None, 0, None) == pit.PIT_E_INVALID
    assert lib.pit_parareal_solve(None, 3, 0.0, None, 0, None) == pit.PIT_E_INVALID


def test_serve_footprint_is_host_only_and_monotone(lib):
    from paper_2203_10148_gb300 import inputs, pit
    small = inputs.serving_request(0, m1d=(100, 101), nslices=(16, 17))[1]
    f = pit.serve_footprint
    base = inputs.heat1d()
    b1 = f(base)
    base.N *= 2
    assert f(base) > b1
    w2 = inputs.heat2d(n=32, N=16)
    w1 = inputs.heat1d(M=1024, N=16)
    # the 2D sweep's sine-mode work makes a 2D request larger than a 1D one of equal size
    assert f(w2) > f(w1)
    # eight Krylov block vectors at least
    vlen = (w2.N + 1) * w2.M * w2.batch
    assert f(w2) >= 64 * vlen
    assert f(small) > 0
    bad = pit.ProblemDesc()
    out = C.c_size_t()
    assert lib.pit_serve_footprint(C.byref(bad), C.byref(out)) == pit.PIT_E_INVALID


@pytest.mark.parametrize("M,N,batch", [(63, 16, 2), (8, 128, 64)])
def test_serve_footprint_counts_the_fp64_heat1d_tables(lib, M, N, batch):
    """An FP64 1D heat request on a small grid stores the fine propagator
    matrix (M^2 doubles), the N powers of G (M^2 rounded up to even doubles
    each) and the sweep's (N+1)(N+2)/2 products of M doubles per member; the
    footprint the server reserves holds them on top of eight Krylov block
    vectors (at N = 128 the products are eight times those vectors)."""
    from paper_2203_10148_gb300 import inputs, pit
    w = inputs.heat1d(M=M, N=N, batch=batch)
    assert w.precision == "fp64" and w.fine[1] == 100 and w.coarse[1] == 1
    vlen = (N + 1) * M * batch
    tables = 8 * (M * M + N * ((M * M + 1) // 2 * 2) + batch * (N + 1) * (N + 2) // 2 * M)
    assert pit.serve_footprint(w) >= 64 * vlen + tables


@pytest.mark.parametrize("M,m", [(17, 100), (63, 100), (63, 3), (100, 7), (128, 50), (200, 40), (200, 400),
                                 (250, 2000), (256, 100), (257, 1000)])
def test_bench_matrix_label_agrees_with_the_library(lib, M, m):
    """bench.py names the 1D heat FP64 roofline kernel after the library's
    choice of fine batch (the stored propagator matrix, or the steps).  The
    library's choice is read from the serving footprint, which counts the
    matrix's M^2 doubles only where set-up stores it: at N = 200 no powers of
    G are stored, and one fine step stores no matrix on these grids."""
    import bench
    from paper_2203_10148_gb300 import inputs, pit
    w = inputs.heat1d(M=M, N=200, fine_steps=m)
    one = inputs.heat1d(M=M, N=200, fine_steps=1)
    stored = pit.serve_footprint(w) - pit.serve_footprint(one)
    assert stored in (0, 8 * M * M)
    assert bench.heat1d_uses_matrix(w) == (stored == 8 * M * M)


def test_binding_rejects_arrays_of_the_wrong_size():
    """The library reads or writes a fixed number of values through each
    array pointer; the binding refuses arrays of another size before any call
    (a short array would be accessed out of bounds)."""
    from paper_2203_10148_gb300 import inputs, pit
    assert pit._array_arg(np.zeros(6), 6)[1] == 0
    with pytest.raises(ValueError):
        pit._array_arg(np.zeros(5), 6)
    with pytest.raises(ValueError):
        pit._array_arg(np.zeros(6, dtype=np.float32), 6)
    with pytest.raises(ValueError):
        pit._array_arg(np.zeros((3, 4)).T, 12)          # not C-contiguous
    w = inputs.heat1d(M=10, N=3, batch=2)
    pit.problem_desc(w, pit.PIT_FP64)
    w.y0 = w.y0[:, :9]                                  # rows of 9 values, M = 10
    with pytest.raises(ValueError):
        pit.problem_desc(w, pit.PIT_FP64)
    d = inputs.dense(M=12, N=2, T=0.1)
    d.A = d.A[:, :11]
    with pytest.raises(ValueError):
        pit.problem_desc(d, pit.PIT_FP64)
    a = inputs.advdiff2d(n=8, N=2)
    a.vx = a.vx.reshape(-1)[:-1]
    with pytest.raises(ValueError):
        pit.problem_desc(a, pit.PIT_FP64)


def test_server_calls_reject_null_handles(lib):
    from paper_2203_10148_gb300 import pit
    info = pit.SolveInfo()
    st = pit.ServerStats()
    assert lib.pit_serve_poll(None, 1, None, C.byref(info)) == pit.PIT_E_INVALID
    assert lib.pit_serve_wait(None, 1, C.c_double(0.0), None, C.byref(info)) == pit.PIT_E_INVALID
    assert lib.pit_serve_cancel(None, 1) == pit.PIT_E_INVALID
    assert lib.pit_server_stats(None, 0, C.byref(st)) == pit.PIT_E_INVALID
    t = C.c_uint64()
    assert lib.pit_serve_submit(None, None, None, C.byref(t)) == pit.PIT_E_INVALID
    assert lib.pit_server_destroy(None) == pit.PIT_OK
    assert lib.pit_server_create(0, 0, None) == pit.PIT_E_INVALID


@pytest.mark.parametrize("name", ["pit_block_reduce", "pit_block_reduce_noalloc"])
def test_reductions_reject_more_blocks_than_grid_rows(lib, name):
    """One grid row per block: nblocks > 65535 is refused before any device
    call (the pointers are never dereferenced), also where the allocation-free
    variant's scratch would hold the partial sums (M = 1)."""
    from paper_2203_10148_gb300 import pit
    fake = C.c_void_p(256)
    st = getattr(lib, name)(fake, fake, 65536, 1, fake, None, fake)
    assert st == pit.PIT_E_INVALID
    assert "65535" in pit.last_error()
