"""shf_mass_static: the mean of a caller-owned device field with no device
allocation (scratch in a fixed device array of the library).  It must return
the same bits as shf_mass on the same field, on consecutive calls, and reject
what does not fit its fixed scratch before touching the device.

The file name sorts last so that the GPU test also runs after every other
test in one session (the fixed scratch must not depend on earlier state)."""
import ctypes
import math

import numpy as np
import pytest

import paper_0710_5912_gb300 as shf

FP32, FP64 = shf.SHF_FP32, shf.SHF_FP64


def raw(ptr, precision, nx, ny):
    m = ctypes.c_double()
    rc = shf.lib().shf_mass_static(ptr, precision, nx, ny, None, ctypes.byref(m))
    return rc, m.value


def test_arguments_are_checked_before_any_device_work():
    # a fake, aligned non-null pointer: every case below fails validation first
    fake = 1 << 20
    for args in [(fake, FP32, 4097, 16), (fake, FP32, 16, 4097), (fake, FP32, 0, 16), (fake, FP64, 16, -1),
                 (fake, 16, 64, 64), (None, FP32, 64, 64), (fake + 2, FP32, 64, 64),
                 (fake + 4, FP64, 64, 64)]:
        rc, m = raw(*args)
        assert rc == shf.SHF_EINVAL, args
        assert math.isnan(m), args
    assert shf.lib().shf_mass_static(fake, FP32, 64, 64, None, None) == shf.SHF_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [FP32, FP64])
def test_static_mass_equals_shf_mass_on_consecutive_calls(precision):
    import torch
    dtype = torch.float32 if precision == FP32 else torch.float64
    nx, ny = 512, 256
    bufs = [torch.zeros((ny, nx), dtype=dtype, device="cuda") for _ in range(3)]
    with shf.Grid(nx, ny, 1.0, precision) as g:
        g.set_params(a=1.0, b=1.0, kappa=1.0, M=1.0, eta=1.0, rho=1.0, gdot=0.01, dt=0.005)
        g.init_noise(seed=11, amp=0.3)
        g.bind_device_fields(*bufs)
        for call in range(2):
            g.step(7)
            g.sync()
            want = g.mass()
            got = shf.shf_mass_static(bufs[0], precision, nx, ny)
            assert got == want, (call, got, want)
            # and both are the compensated mean of the field, to rounding
            host = bufs[0].cpu().numpy().astype(np.float64)
            exact = math.fsum(host.ravel()) / host.size
            assert abs(got - exact) <= 1e-15 * np.abs(host).mean()


@pytest.mark.gpu
def test_static_mass_any_shape_stream_and_no_allocation():
    import torch
    torch.manual_seed(3)
    x = (torch.rand((37, 1000), dtype=torch.float64) * 2 - 1).cuda()
    exact = math.fsum(x.cpu().numpy().ravel()) / x.numel()
    stream = torch.cuda.Stream()
    got = shf.shf_mass_static(x, FP64, 1000, 37, stream=stream)
    assert abs(got - exact) <= 1e-16
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        assert shf.shf_mass_static(x, FP64, 1000, 37) == got
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    # a single element, and the largest accepted field
    one = torch.full((1, 1), 0.25, dtype=torch.float32, device="cuda")
    assert shf.shf_mass_static(one, FP32, 1, 1) == 0.25
    big = torch.full((4096, 4096), 0.5, dtype=torch.float32, device="cuda")
    assert shf.shf_mass_static(big, FP32, 4096, 4096) == 0.5
    del big


@pytest.mark.gpu
def test_static_mass_rejects_host_memory_and_flags_non_finite():
    import torch
    host = np.zeros(64 * 64, dtype=np.float32)
    rc, m = raw(host.ctypes.data, FP32, 64, 64)
    assert rc == shf.SHF_EINVAL and math.isnan(m)
    rc, _ = raw(int(torch.zeros(1, device="cuda").data_ptr()), FP32, 8192, 1)
    assert rc == shf.SHF_EINVAL
    y = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    y[5, 7] = float("nan")
    rc, m = raw(int(y.data_ptr()), FP32, 64, 64)
    assert rc == shf.SHF_ENONFINITE and math.isnan(m)
    y[5, 7] = 1.0
    rc, m = raw(int(y.data_ptr()), FP32, 64, 64)
    assert rc == shf.SHF_OK and m == 1.0 / 4096


@pytest.mark.gpu
def test_static_mass_of_a_tensor_written_on_a_side_stream():
    """No stream given: the binding runs the call on torch's current stream, so
    the mean sees the side stream's writes without an explicit synchronisation."""
    import torch
    side = torch.cuda.Stream()
    x = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        for _ in range(8):                      # enough queued work that a racing read would see zeros
            x.add_(0.125)
        got = shf.shf_mass_static(x, FP32, 2048, 2048)
    assert got == 1.0
