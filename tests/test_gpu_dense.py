"""GPU parity of the dense-propagator mode (y' = A y, Phi = R(dt A)^m applied
to all slices as one product, G = (I - dT A)^{-1}) against the FP64 oracle.
Tolerances: FP64 path 1e-12 relative; FP32 product 2e-5; mixed solves 1e-6
against the serial FP64 trajectory."""
import numpy as np
import pytest

from oracle import OracleProblem, pitsbicg
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


def _rand(w, seed):
    return inputs.SeededStream(seed).normal(w.batch * (w.N + 1) * w.M).reshape(w.batch, w.N + 1, w.M)


def _oracle(w, which, X):
    out = []
    for b in range(w.batch):
        o = OracleProblem.from_workload(w, member=b)
        out.append({"F": o.apply_F, "Ginv": o.sweep_Ginv, "GinvF": o.apply_GinvF,
                    "residual": o.residual}[which](X[b]))
    return np.stack(out)


CASES = [dict(M=24, N=8, T=1.0, fine_steps=37), dict(M=100, N=5, T=2.0, fine_steps=20, batch=2),
         dict(M=1, N=3, T=1.0, fine_steps=4), dict(M=257, N=6, T=10.0 * 6 / 4096, fine_steps=200)]


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("which", ["F", "Ginv", "GinvF", "residual"])
def test_dense_operators_fp64(case, which):
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(**case, precision="fp64")
    X = _rand(w, 1)
    with pit.Problem(w, "fp64") as p:
        got = p.apply(which, X)
    assert _rel(got, _oracle(w, which, X)) < 1e-12


@pytest.mark.parametrize("case", CASES[:2])
def test_dense_fine_product_fp32(case):
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(**case)
    X = _rand(w, 2)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="mixed")
    assert _rel(got, _oracle(w, "F", X)) < 2e-5


@pytest.mark.parametrize("case", [dict(M=64, N=8, T=1.0, fine_steps=37),
                                  dict(M=128, N=5, T=2.0, fine_steps=20, batch=2),
                                  dict(M=256, N=70, T=10.0 * 70 / 4096, fine_steps=200),
                                  dict(M=1, N=3, T=1.0, fine_steps=4),
                                  dict(M=100, N=5, T=2.0, fine_steps=20, batch=2),
                                  dict(M=257, N=6, T=10.0 * 6 / 4096, fine_steps=200)])
def test_dense_float_float_product(case):
    """The compensated float-float product (Dot2 form on (hi, lo) pairs) used
    by the mixed path's true residual: within 1e-11 of the FP64 oracle, on
    row counts that are not multiples of the 64-row tile and any M (operand
    rows padded to 64)."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(**case)
    X = _rand(w, 5)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="ff")
        res = p.apply("residual", X, precision="ff")
    assert _rel(got, _oracle(w, "F", X)) < 1e-11
    assert _rel(res, _oracle(w, "residual", X)) < 1e-10


SPLIT_CASES = [dict(M=64, N=8, T=1.0, fine_steps=37),
               dict(M=128, N=5, T=2.0, fine_steps=20, batch=2),
               dict(M=256, N=70, T=10.0 * 70 / 4096, fine_steps=200),
               dict(M=1, N=3, T=1.0, fine_steps=4),
               dict(M=100, N=5, T=2.0, fine_steps=20, batch=2),
               dict(M=257, N=6, T=10.0 * 6 / 4096, fine_steps=200),
               dict(M=1000, N=130, T=10.0 * 130 / 4096, fine_steps=200, batch=2)]


@pytest.mark.parametrize("case", SPLIT_CASES)
def test_dense_split_product(case):
    """The product by error-free splitting on the tensor cores (PIT_SPLIT,
    the mixed path's default true residual: 7 slices of 6-bit digits per
    operand, every anti-diagonal of slice products accumulated exactly in
    FP32): within 1e-11 of the FP64 oracle like the float-float product, on
    row counts that are not multiples of the 128-row tile, several members
    and any M up to 1024 (operands padded to 128)."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(**case)
    X = _rand(w, 5)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="split")
        res = p.apply("residual", X, precision="split")
    assert _rel(got, _oracle(w, "F", X)) < 1e-11
    assert _rel(res, _oracle(w, "residual", X)) < 1e-10


def test_dense_split_product_rows_of_any_scale():
    """Each row is split relative to its own largest magnitude: zero rows,
    rows scaled by 1e-200 and 1e200, rows whose entries span 12 decades and
    rows of one sign.  Every element of the row x_n - Phi x_(n-1) is within
    2^-36 sum_k |Phi_ck| |x_(n-1),k| (the splitting's bound, 2^-42 per operand
    row maximum, with margin) plus the rounding of the final FP64
    subtraction, 2^-53 |x_n|."""
    from oracle.operators import dense_rk4_propagator_matrix, spatial_operator
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=128, N=9, T=1.0, fine_steps=37)
    X = _rand(w, 9)
    X[0, 1] = 0.0
    X[0, 2] *= 1e-200
    X[0, 3] *= 1e200
    X[0, 4, ::2] *= 1e-12
    X[0, 5] = np.abs(X[0, 5])
    X[0, 6] = -np.abs(X[0, 6]) * 1e-30
    Phi = dense_rk4_propagator_matrix(spatial_operator(w.kind, w.nx, w.ny, w.nu, w.vx, w.vy, w.A),
                                      w.T / w.N, w.fine[1])
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="split")[0]
    for n in range(1, w.N + 1):
        prod = Phi @ X[0, n - 1]
        bound = np.abs(Phi) @ np.abs(X[0, n - 1])
        err = np.abs(got[n] - (X[0, n] - prod))
        assert np.all(err <= 2.0 ** -36 * bound + 2.0 ** -53 * np.abs(X[0, n]) + 1e-300), \
            (n, err.max(), bound.max())
    np.testing.assert_array_equal(got[0], X[0, 0])


def test_dense_split_falls_back_beyond_its_exact_width():
    """Beyond K = 1024 the diagonal sums are no longer exact in FP32: PIT_SPLIT
    then runs the float-float product, bit for bit."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=1100, N=3, T=10.0 * 3 / 4096, fine_steps=200)
    X = _rand(w, 4)
    with pit.Problem(w, "mixed") as p:
        a = p.apply("F", X, precision="split")
        b = p.apply("F", X, precision="ff")
    np.testing.assert_array_equal(a, b)


def test_dense_fp64_bicgstab_matches_oracle():
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=64, N=32, T=1.0, fine_steps=50, precision="fp64")
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "fp64") as p:
        for k in (1, 2):
            X, info = p.bicgstab_solve(tol=0.0, max_iter=k)
            assert _rel(X[0], pitsbicg(o, tol=0.0, max_iter=k)[0]) < 1e-11
        X, info = p.bicgstab_solve(tol=1e-10)
        lam = p.serial_fine()
    ref = o.serial_fine()
    assert info[0]["status"] == 0
    assert _rel(lam[0], ref) < 1e-12
    assert np.linalg.norm(X[0] - ref) / np.linalg.norm(ref) < 1e-8


def test_dense_mixed_solve_within_1e6():
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=128, N=64, T=64 * 10.0 / 4096, fine_steps=200)
    ref = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-8, tol_mode="rhs", inner_tol=1e-5)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - ref) / np.linalg.norm(ref) < 1e-6


def test_dense_full_size_sampled():
    """M = 1024, N = 4096 (the dense-propagator workload): the FP64 operator on
    sampled slices against the oracle's propagator and coarse solve."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense()
    o = OracleProblem.from_workload(w)
    X = _rand(w, 3)
    Xd = torch.from_numpy(X).cuda()
    with pit.Problem(w, "mixed") as p:
        Y = p.apply("F", Xd, precision="fp64").cpu().numpy()[0]
        Y32 = p.apply("F", Xd, precision="mixed").cpu().numpy()[0]
        Yff = p.apply("F", Xd, precision="ff").cpu().numpy()[0]
        Ysp = p.apply("F", Xd, precision="split").cpu().numpy()[0]
    rows = [1, 2, 777, 2048, 4095, 4096]
    ref = X[0][rows] - o.F(X[0][[r - 1 for r in rows]])
    assert _rel(Y[rows], ref) < 1e-12
    assert _rel(Yff[rows], ref) < 1e-11
    assert _rel(Ysp[rows], ref) < 1e-11
    assert _rel(Y32[rows], ref) < 1e-4
    np.testing.assert_array_equal(Y[0], X[0][0])


@pytest.mark.parametrize("N", [1, 2, 8, 10, 63, 200])
def test_dense_mixed_sweep_chunked_scan(N):
    """The FP32 chunked scan of the coarse sweep (L = ceil(sqrt(N+1)) blocks per
    chunk, partial last chunk) against the oracle's sequential forward
    substitution of eq. (7): FP32 accuracy."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=96, N=N, T=N * 10.0 / 4096, fine_steps=10, batch=2)
    X = _rand(w, 7)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("Ginv", X, precision="mixed")
        got64 = p.apply("Ginv", X, precision="fp64")
    ref = _oracle(w, "Ginv", X)
    assert _rel(got, ref) < 2e-5
    assert _rel(got64, ref) < 1e-12


def test_dense_mixed_sweep_full_size():
    from paper_2203_10148_gb300 import pit
    w = inputs.dense()
    X = _rand(w, 8)
    o = OracleProblem.from_workload(w)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("Ginv", torch.from_numpy(X).cuda(), precision="mixed").cpu().numpy()[0]
    ref = o.sweep_Ginv(X[0])
    assert _rel(got, ref) < 1e-4


@pytest.mark.parametrize("M,N,batch", [(128, 16, 1), (128, 16, 2), (256, 300, 1), (384, 5, 3),
                                       (1, 4, 1), (24, 9, 2), (100, 33, 1), (257, 7, 2)])
def test_dense_tensor_core_product(M, N, batch):
    """The tcgen05 3xTF32 product for any M (rows padded to 128 columns, the
    padding never written): block-operator rows against the oracle to FP32
    accuracy, including partial row tiles."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=M, N=N, T=N * 10.0 / 4096, fine_steps=200, batch=batch)
    X = _rand(w, 9)
    with pit.Problem(w, "mixed") as p:
        got = p.apply("F", X, precision="mixed")
        res = p.apply("residual", X, precision="mixed")
    ref = _oracle(w, "F", X)
    assert _rel(got, ref) < 2e-5
    ref_res = _oracle(w, "residual", X)
    assert _rel(res, ref_res) < 2e-5


def test_dense_large_grid_sweep_and_serial_trajectory_fp64():
    """M = 1100 is beyond the persistent sweep's shared memory in FP64: the
    sweep runs one matrix-vector kernel per slice, like the serial fine
    trajectory; both against the oracle."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=1100, N=3, T=3 * 10.0 / 4096, fine_steps=20, precision="fp64", batch=2)
    X = _rand(w, 13)
    with pit.Problem(w, "fp64") as p:
        got = p.apply("Ginv", X)
        lam = p.serial_fine("fp64")
    assert _rel(got, _oracle(w, "Ginv", X)) < 1e-12
    for b in range(w.batch):
        ref = OracleProblem.from_workload(w, member=b).serial_fine()
        assert _rel(lam[b], ref) < 1e-12


@pytest.mark.parametrize("M", [100, 200])
def test_dense_mixed_solve_any_M_within_1e6(M):
    """Mixed solves with M not a multiple of the tensor-core tile (tcgen05
    inner products, float-float true residuals): within 1e-6 of the serial
    FP64 trajectory."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=M, N=32, T=32 * 10.0 / 4096, fine_steps=200)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed") as p:
        X, info = p.bicgstab_solve(tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6


@pytest.mark.parametrize("M,N,batch", [(128, 16, 1), (100, 33, 2), (257, 7, 1)])
def test_dense_bf16x3_product(M, N, batch):
    """PIT_MIXED_BF16: the product split in BF16 on tcgen05 kind::f16 (both
    operands BF16, FP32 accumulation).  Each operand keeps about 17 bits
    (x - xh - xl <= 2^-18 |x|, the dropped xl pl term about 2^-18), so the
    rows agree with the oracle to 1e-4 of their maximum, and less closely
    than the split-TF32 product of the same problem."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=M, N=N, T=N * 10.0 / 4096, fine_steps=200, batch=batch)
    X = _rand(w, 19)
    ref = _oracle(w, "F", X)
    with pit.Problem(w, "mixed_bf16") as p:
        gbf = p.apply("F", X, precision="mixed")
    with pit.Problem(w, "mixed") as p:
        gtf = p.apply("F", X, precision="mixed")
    ebf, etf = _rel(gbf, ref), _rel(gtf, ref)
    assert ebf < 1e-4
    assert etf < ebf


def test_dense_bf16x3_mixed_solve_within_1e6():
    """Refinement with float-float true residuals carries the BF16-split
    inner solves to the same 1e-6 bar."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=128, N=64, T=64 * 10.0 / 4096, fine_steps=200)
    lam = OracleProblem.from_workload(w).serial_fine()
    with pit.Problem(w, "mixed_bf16") as p:
        X, info = p.bicgstab_solve(tol=1e-7, tol_mode="rhs", inner_tol=1e-5)
    assert info[0]["status"] == 0
    assert np.linalg.norm(X[0] - lam) / np.linalg.norm(lam) < 1e-6


@pytest.mark.parametrize("M,N", [(64, 7), (200, 127), (256, 128), (500, 300), (1000, 1), (1024, 700)])
def test_dense_tensor_core_sweep(M, N, monkeypatch):
    """The mixed coarse sweep of one member on the tensor cores (chunked scan
    of at most 128 chunks, doubling scan of the carries, 3xTF32 products
    summed over an 8-CTA cluster) against the oracle's sequential forward
    substitution of eq. (7) and against the CUDA-core chunked scan
    (PIT_DENSE_SWEEP_TC=0): FP32 accuracy on both, by different arithmetic."""
    from paper_2203_10148_gb300 import pit
    w = inputs.dense(M=M, N=N, T=N * 10.0 / 4096, fine_steps=10)
    X = _rand(w, 17)
    with pit.Problem(w, "mixed") as p:
        tc = p.apply("Ginv", X, precision="mixed")
        tcF = p.apply("GinvF", X, precision="mixed")
    monkeypatch.setenv("PIT_DENSE_SWEEP_TC", "0")
    with pit.Problem(w, "mixed") as p:
        cc = p.apply("Ginv", X, precision="mixed")
        ccF = p.apply("GinvF", X, precision="mixed")
    ref = _oracle(w, "Ginv", X)
    assert _rel(tc, ref) < 2e-5
    assert _rel(cc, ref) < 2e-5
    # G^{-1} F also carries the FP32-class fine product, common to both paths:
    # the tensor-core sweep adds no more than the CUDA-core one
    refF = _oracle(w, "GinvF", X)
    assert _rel(tcF, refF) < max(1e-4, 2 * _rel(ccF, refF))
    if N > 1:
        assert not np.array_equal(tc, cc)
