"""The allocation-free conserved sums (tvlbm_conserved_sums_static): for callers that cannot
allocate device memory on this path.  Checked through the C ABI against the regular
tvlbm_conserved_sums on the same state, on two calls in a row (the second reuses the fixed
device scratch the first one left behind), for every velocity set, full and deviation storages
and a reference density other than 1; and for the property itself: repeated calls leave the
device's free memory unchanged, and a call captured in a CUDA graph (where any allocation
fails the capture) replays to the same sums."""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


def _static_fn(tv):
    fn = tv.lib.tvlbm_conserved_sums_static
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p]
    return fn


def _setup(velset, storage, rho0, nx=77, ny=53):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv
    sim = tv.Simulation(nx, ny, velset, tau=0.8, storage=storage, rho0=rho0)
    sim.init_moments(*workloads.random_smooth(nx, ny, seed=21, amp_u=0.08, amp_T=0.08))
    return torch, tv, sim


@pytest.mark.parametrize("velset,storage,rho0", [("D2Q16", "fp32_dev", 1.0), ("D2Q36", "fp16_dev", 1.0),
                                                 ("D2Q16", "fp64", 1.0), ("D2Q9", "fp32", 1.0),
                                                 ("D2Q16", "bf16_dev", 1.0), ("D2Q16", "fp32_dev", 1.3),
                                                 ("D2Q36", "fp16_dev", 0.85)])
def test_static_sums_match_regular_sums(velset, storage, rho0):
    nx, ny = 77, 53
    torch, tv, sim = _setup(velset, storage, rho0, nx, ny)
    fn = _static_fn(tv)
    stream = torch.cuda.current_stream()
    for call in range(2):
        sim.step(7)
        want = sim.conserved_sums()
        raw = sim.raw_populations()
        dev = torch.from_numpy(raw.view(np.uint8).reshape(-1)).to("cuda")
        out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
        rc = fn(dev.data_ptr(), tv.VELSETS[velset], tv.STORAGES[storage], nx, ny, rho0, out.data_ptr(),
                stream.cuda_stream)
        assert rc == tv.TVLBM_OK, (call, rc)
        stream.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got[:4], want[:4], rtol=0, atol=1e-12 * abs(want[0]))
        assert got[4] == want[4] == 0
    # a wrong reference density shifts the mass by (rho0' - rho0) sum w = the cell count times it
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    if storage.endswith("_dev"):
        assert fn(dev.data_ptr(), tv.VELSETS[velset], tv.STORAGES[storage], nx, ny, rho0 + 0.25, out.data_ptr(),
                  stream.cuda_stream) == tv.TVLBM_OK
        stream.synchronize()
        assert abs(out[0].item() - want[0] - 0.25 * nx * ny) <= 1e-9 * nx * ny


def test_static_sums_allocate_nothing():
    """Free device memory is unchanged over repeated calls, and a call captured in a CUDA graph
    (global capture mode: an allocation on any thread invalidates the capture) replays to the
    sums of an uncaptured call."""
    nx, ny, velset, storage = 96, 64, "D2Q16", "fp32_dev"
    torch, tv, sim = _setup(velset, storage, 1.0, nx, ny)
    fn = _static_fn(tv)
    sim.step(5)
    raw = sim.raw_populations()
    dev = torch.from_numpy(raw.view(np.uint8).reshape(-1)).to("cuda")
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    args = (dev.data_ptr(), tv.VELSETS[velset], tv.STORAGES[storage], nx, ny, 1.0, out.data_ptr(), side.cuda_stream)
    assert fn(*args) == tv.TVLBM_OK  # loads the kernels and records the scratch address
    side.synchronize()
    want = out.cpu().numpy().copy()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        assert fn(*args) == tv.TVLBM_OK
    side.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    np.testing.assert_array_equal(out.cpu().numpy(), want)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = fn(*args)
    assert rc == tv.TVLBM_OK
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), want)


def test_static_sums_reject_bad_arguments():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1004_5059_gb300 as tv

    fn = _static_fn(tv)
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    assert fn(buf.data_ptr(), 16, 1, 1, 1, 1.0, None, None) == tv.TVLBM_EINVAL
    assert fn(buf.data_ptr(), 17, 1, 1, 1, 1.0, out.data_ptr(), None) == tv.TVLBM_EINVAL
    assert fn(buf.data_ptr(), 36, 1, 1 << 16, 1 << 16, 1.0, out.data_ptr(), None) == tv.TVLBM_EINVAL
    assert fn(buf.data_ptr(), 16, 1, 1, 1, 0.0, out.data_ptr(), None) == tv.TVLBM_EINVAL
