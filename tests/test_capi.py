"""C ABI checks that need no GPU: the library loads, exports every symbol include/*.h
declares, validates arguments, and its host-side velocity sets and streaming tables agree with
the oracle's independently built ones."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tv():
    import paper_1004_5059_gb300 as tv  # built by conftest at session start
    return tv


@pytest.mark.parametrize("header,least", [("tvlbm.h", 20), ("tvlbm_closure.h", 12)])
def test_exports_every_declared_symbol(tv, header, least):
    text = open(os.path.join(ROOT, "include", header)).read()
    names = set(re.findall(r"\b(tvlbm_[a-z0-9_]+)\s*\(", text))
    assert len(names) >= least
    for n in sorted(names):
        assert hasattr(tv.lib, n), n


@pytest.mark.parametrize("name", ["D2Q9", "D2Q16", "D2Q36"])
def test_velocity_set_matches_oracle(tv, name):
    import oracle
    cx, cy, w, N = tv.tvlbm_velocity_set(tv.VELSETS[name])
    vs = oracle.velocity_set(name)
    np.testing.assert_allclose(cx, vs["cx"], rtol=0, atol=2e-15)
    np.testing.assert_allclose(cy, vs["cy"], rtol=0, atol=2e-15)
    np.testing.assert_allclose(w, vs["w"], rtol=0, atol=2e-16)
    assert N == vs["N"]


@pytest.mark.parametrize("name,dt", [("D2Q16", 1.0), ("D2Q36", 1.0), ("D2Q16", 0.3), ("D2Q9", 1 / math.sqrt(3))])
def test_stream_table_matches_oracle(tv, name, dt):
    import oracle
    sx, sy, ax, ay = tv.tvlbm_stream_table(tv.VELSETS[name], dt)
    vs = oracle.velocity_set(name)
    osx, oax = oracle.stream_table(vs["cx"], dt)
    osy, oay = oracle.stream_table(vs["cy"], dt)
    assert np.array_equal(sx, osx) and np.array_equal(sy, osy)
    np.testing.assert_allclose(ax, oax, rtol=0, atol=1e-15)
    np.testing.assert_allclose(ay, oay, rtol=0, atol=1e-15)


def test_memory_bytes_and_validation(tv):
    b = tv.tvlbm_memory_bytes(1024, 1024, tv.TVLBM_D2Q16, None, tv.TVLBM_FP32)
    assert b > 2 * 16 * 1024 * 1024 * 4
    walls = (0.0, 1.0, 0.1, 1.1)
    assert tv.tvlbm_memory_bytes(64, 64, tv.TVLBM_D2Q36, walls, tv.TVLBM_BF16_DEV) > 0
    bad = [
        (0, 8, tv.TVLBM_D2Q16, None, tv.TVLBM_FP32),
        (8, 8, 17, None, tv.TVLBM_FP32),
        (8, 8, tv.TVLBM_D2Q16, None, 9),
        (8, 4, tv.TVLBM_D2Q16, walls, tv.TVLBM_FP32),  # walls need ny >= 9
        (8, 16, tv.TVLBM_D2Q16, (0.0, -1.0, 0.0, 1.0), tv.TVLBM_FP32),  # T_lo <= 0
    ]
    for args in bad:
        with pytest.raises(tv.TvlbmError) as e:
            tv.tvlbm_memory_bytes(*args)
        assert e.value.code == tv.TVLBM_EINVAL


def test_create_rejects_bad_parameters_without_touching_cuda(tv):
    for tau, dt in [(0.4, 1.0), (0.8, 0.0), (0.8, 2.0)]:  # tau <= dt/2; dt <= 0; shift >= 4 cells
        with pytest.raises(tv.TvlbmError) as e:
            tv.tvlbm_create(16, 16, tv.TVLBM_D2Q36, tau, dt, None, tv.TVLBM_FP32, 1.0)
        assert e.value.code == tv.TVLBM_EINVAL


def test_create_without_gpu_reports_cuda_error(tv):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(tv.TvlbmError) as e:
        tv.tvlbm_create(16, 16, tv.TVLBM_D2Q16, 0.8, 1.0, None, tv.TVLBM_FP32, 1.0)
    assert e.value.code == tv.TVLBM_ECUDA


def test_strerror(tv):
    assert tv.lib.tvlbm_strerror(0) == b"ok"
    assert tv.lib.tvlbm_strerror(-3) == b"CUDA error"
    assert tv.lib.tvlbm_last_error(None) == b""
