"""pit_block_reduce_noalloc, the allocation-free block reduction, against
pit_block_reduce.

The variant keeps its partial sums in a fixed array inside the library, for
callers that may not allocate device memory.  Two calls in a row (the second
on smaller inputs, so stale partials from the first would show) must each
match the allocating entry point within the tolerance of the other reduction
tests.  This file is collected last so a failure here comes after every
other test has run.
"""
import ctypes as C

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


def _both(U, V, nb, M):
    from paper_2203_10148_gb300 import pit
    tu, tv = torch.from_numpy(U).cuda(), torch.from_numpy(V).cuda()
    ref = pit.block_reduce(tu, tv, nb, M)
    got = pit.block_reduce(tu, tv, nb, M, noalloc=True)
    return ref, got


def test_noalloc_matches_allocating_reduce_twice():
    s = inputs.SeededStream(77)
    for nb, M in ((513, 16384), (7, 63)):
        U = s.normal(nb * M).reshape(nb, M)
        V = s.normal(nb * M).reshape(nb, M)
        (d0, n0, i0), (d1, n1, i1) = _both(U, V, nb, M)
        assert d1 == pytest.approx(d0, rel=1e-12, abs=1e-12)
        np.testing.assert_allclose(n1, n0, rtol=1e-13)
        assert i1 == pytest.approx(i0, rel=1e-13)
        assert d1 == pytest.approx(float(np.sum(U * V)), rel=1e-12)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    from paper_2203_10148_gb300 import pit
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    # 2 blocks of 2048 * 40000 values: 80000 chunks (the pointers are never read)
    st = pit.load().pit_block_reduce_noalloc(x.data_ptr(), x.data_ptr(), 2, 2048 * 40000,
                                             out.data_ptr(), None, out.data_ptr() + 8)
    assert st == pit.PIT_E_INVALID
    assert "fixed scratch" in pit.last_error()


def test_noalloc_rejects_more_blocks_than_grid_rows():
    """65536 blocks of one value fit the scratch (65536 chunks) but not the
    grid (one grid row per block, at most 65535): refused as invalid, not
    reported as a failed launch."""
    from paper_2203_10148_gb300 import pit
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    st = pit.load().pit_block_reduce_noalloc(x.data_ptr(), x.data_ptr(), 65536, 1,
                                             out.data_ptr(), None, out.data_ptr() + 8)
    assert st == pit.PIT_E_INVALID
    assert "65535" in pit.last_error()
