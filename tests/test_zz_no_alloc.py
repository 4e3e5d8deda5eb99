"""The allocation-free conserved sums (tvlbm_conserved_sums_static): for callers that cannot
allocate device memory on this path.  Checked through the C ABI against the regular
tvlbm_conserved_sums on the same state, on two calls in a row (the second reuses the fixed
device scratch the first one left behind)."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("velset,storage", [("D2Q16", "fp32_dev"), ("D2Q36", "fp16_dev"), ("D2Q16", "fp64")])
def test_static_sums_match_regular_sums(velset, storage):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv

    fn = tv.lib.tvlbm_conserved_sums_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p]
    nx, ny = 77, 53
    sim = tv.Simulation(nx, ny, velset, tau=0.8, storage=storage)
    sim.init_moments(*workloads.random_smooth(nx, ny, seed=21, amp_u=0.08, amp_T=0.08))
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(7)
        want = sim.conserved_sums()
        raw = sim.raw_populations()
        dev = torch.from_numpy(raw.view(np.uint8).reshape(-1)).to("cuda")
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        rc = fn(dev.data_ptr(), tv.VELSETS[velset], tv.STORAGES[storage], nx, ny, 1.0, out.data_ptr(),
                stream.cuda_stream)
        assert rc == tv.TVLBM_OK, (call, rc)
        stream.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:4], want[:4], rtol=0, atol=1e-12 * abs(want[0]))
        assert got[4] == want[4] == 0


def test_static_sums_reject_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv

    fn = tv.lib.tvlbm_conserved_sums_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p]
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert fn(buf.data_ptr(), 16, 1, 1, 1, 1.0, None, None) == tv.TVLBM_EINVAL
    assert fn(buf.data_ptr(), 17, 1, 1, 1, 1.0, out.data_ptr(), None) == tv.TVLBM_EINVAL
    assert fn(buf.data_ptr(), 36, 1, 1 << 16, 1 << 16, 1.0, out.data_ptr(), None) == tv.TVLBM_EINVAL
