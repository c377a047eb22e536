"""The C ABI library on a machine without a GPU: it builds for sm_103a, loads,
exports every entry point declared in include/shf.h, and its host-only logic
(strain bookkeeping, quench noise, argument validation) is right."""
import ctypes
import os
import re

import numpy as np
import pytest

import oracle
import paper_0710_5912_gb300 as shf
from paper_0710_5912_gb300 import _native, inputs

HEADER = os.path.join(_native.INCLUDE, "shf.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(shf_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    return shf.lib()


def test_library_exports_every_declared_symbol(lib):
    names = declared_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # and the binding declares the same set (argument marshalling only)
    assert sorted(_native.SIGNATURES) == names


def test_library_is_built_for_sm_103a_only():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_native.ARCH_FLAGS)
    data = open(_native.LIB_PATH, "rb").read()
    assert b"sm_103a" in data


def test_version_and_strerror(lib):
    assert shf.shf_version() >= 10000
    assert lib.shf_strerror(shf.SHF_EINVAL) == b"invalid argument"
    assert lib.shf_strerror(12345) == b"unknown error"


@pytest.mark.parametrize("gdot,dt,nx,ny", [(0.01, 0.005, 64, 64), (1.0, 2.0 ** -6, 64, 64),
                                            (0.003, 0.005, 1024, 1024), (0.051, 0.004, 1024, 512),
                                            (-0.013, 0.7, 64, 64)])
def test_host_strain_matches_oracle_bit_for_bit(gdot, dt, nx, ny):
    for n in list(range(0, 300, 7)) + [10000, 33333, 10 ** 6, 2 * 10 ** 5]:
        assert shf.shf_strain(n, gdot, dt, nx, ny) == oracle.strain(n, gdot, dt, nx, ny)


def test_host_noise_matches_input_generator():
    for seed in (0, 1, 95):
        got = shf.shf_noise_fill(64 * 32, seed, 0.01)
        want = inputs.quench_noise(64, 32, seed, 0.01).ravel()
        assert np.array_equal(got, want)


def test_invalid_sizes_are_rejected_before_any_device_work(lib):
    h = ctypes.c_void_p()
    for nx, ny, dx in [(63, 64, 1.0), (64, 128, 1.0), (8192, 64, 1.0), (64, 64, 0.0), (8, 8, 1.0),
                       (64, 64, float("nan"))]:
        rc = lib.shf_create_grid(ctypes.byref(h), nx, ny, dx, 32, 0, None)
        assert rc == shf.SHF_EINVAL
    assert lib.shf_create_grid(ctypes.byref(h), 64, 64, 1.0, 16, 0, None) == shf.SHF_EINVAL
    assert lib.shf_create_grid(ctypes.byref(h), 64, 64, 1.0, 32, 7, None) == shf.SHF_EINVAL
    assert lib.shf_strain(0, 1.0, 1.0, 64, 48, ctypes.byref(ctypes.c_double()),
                          ctypes.byref(ctypes.c_int64())) == shf.SHF_EINVAL


def test_no_device_gives_cuda_error_not_a_fallback(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.shf_create_grid(ctypes.byref(h), 64, 64, 1.0, 32, 0, None) == shf.SHF_ECUDA
    with pytest.raises(shf.ShfError):
        shf.Grid(64, 64)
