"""The integer-pipe FP64 <-> FP32 conversions used by the FP32 kernels agree
bit for bit with CUDA's hardware conversions (round to nearest even)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_conversions_match_hardware_bitwise():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2203_10148_gb300 import inputs, pit
    s = inputs.SeededStream(31)
    vals = [s.normal(100000), s.uniform(50000, -1e-30, 1e-30), s.normal(20000) * 1e37,
            np.array([0.0, -0.0, 1e-40, -1e-45, 1e-46, 3.4028234663852886e38, 3.5e38, 1e39,
                      -1e300, np.inf, -np.inf, np.nan, 1.17549435e-38, 1.1754942e-38, 1.0, -2.5])]
    # exact halfway points between neighbouring floats (ties to even), both parities
    f = np.float32(1.0) + np.arange(64, dtype=np.float32) * np.float32(2.0 ** -23)
    mids = (f[:-1].astype(np.float64) + f[1:].astype(np.float64)) / 2.0
    vals += [mids, -mids, mids * 2.0 ** 100, np.nextafter(mids, np.inf), np.nextafter(mids, -np.inf)]
    x = np.concatenate(vals).astype(np.float64)
    d = torch.from_numpy(x).cuda()
    f32 = torch.empty(x.size, dtype=torch.float32, device="cuda")
    back = torch.empty(x.size, dtype=torch.float64, device="cuda")
    pit.check(pit.load().pit_selftest_convert(d.data_ptr(), x.size, f32.data_ptr(), back.data_ptr()))
    ref = d.float()
    got = f32.view(torch.int32).cpu().numpy()
    exp = ref.view(torch.int32).cpu().numpy()
    nan = np.isnan(x)
    np.testing.assert_array_equal(got[~nan], exp[~nan])
    assert np.isnan(f32.cpu().numpy()[nan]).all()
    rb = ref.double().view(torch.int64).cpu().numpy()
    gb = back.view(torch.int64).cpu().numpy()
    np.testing.assert_array_equal(gb[~nan], rb[~nan])
