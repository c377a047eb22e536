"""GB300-native stepper for 2D binary-fluid phase separation under steady shear.

A thin Python binding over the C ABI of ``include/shf.h`` (libshf.so, built
in-tree for sm_103a).  Every function named ``shf_*`` here mirrors the C entry
point of the same name; the binding only marshals arguments (numpy arrays,
torch streams and device pointers) and turns error codes into ``ShfError``.
All arithmetic of the time step runs in the library's CUDA kernels: there is no
CPU fallback, and calling any ``shf_*`` function without the compiled library
raises.

``Grid`` and ``Ensemble`` wrap the handles for convenience.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native

SHF_OK, SHF_EINVAL, SHF_ENOMEM, SHF_ECUDA, SHF_ENONFINITE, SHF_ETIMEOUT, SHF_EIO, SHF_ESTATE = \
    0, -1, -2, -3, -4, -5, -6, -7
SHF_FP32, SHF_FP64 = 32, 64
SHF_REMAP_SHIFT, SHF_REMAP_NONE = 0, 1


class ShfError(RuntimeError):
    def __init__(self, code, message):
        super().__init__(f"{message} (code {code})")
        self.code = code


def lib():
    """The loaded libshf (built on first use if missing or stale)."""
    return _native.load()


def _check(code, handle=None, what=""):
    if code != SHF_OK:
        L = lib()
        msg = L.shf_last_error(handle).decode() if handle else ""
        if not msg:
            msg = L.shf_strerror(code).decode()
        raise ShfError(code, f"{what}: {msg}" if what else msg)


def _dptr(a):
    return a.ctypes.data_as(_native.P_double) if a is not None else None


def _as_field(a, nx, ny):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (ny, nx):
        raise ValueError(f"field shape {a.shape} != ({ny}, {nx})")
    return a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream", stream))


# --------------------------------------------------------------- raw binding

def shf_version() -> int:
    return lib().shf_version()


def shf_strain(n, gdot, dt, nx, ny):
    s, K = ctypes.c_double(), ctypes.c_int64()
    _check(lib().shf_strain(int(n), float(gdot), float(dt), int(nx), int(ny), ctypes.byref(s),
                            ctypes.byref(K)), what="shf_strain")
    return s.value, K.value


def shf_noise_fill(count, seed, amp):
    out = np.empty(int(count), dtype=np.float64)
    _check(lib().shf_noise_fill(_dptr(out), int(count), int(seed) & (2 ** 64 - 1), float(amp)),
           what="shf_noise_fill")
    return out


def shf_mass_static(d_field, precision, nx, ny, stream=None):
    """Mean of a device field (pointer or tensor) without device allocation.

    With a torch tensor and no stream, the call runs on torch's current stream
    of the tensor's device, so it is ordered after the work that wrote the
    tensor there; with a raw pointer and no stream it runs on the legacy
    default stream."""
    ptr = int(d_field.data_ptr()) if hasattr(d_field, "data_ptr") else d_field
    if stream is None and hasattr(d_field, "device") and getattr(d_field.device, "type", "") == "cuda":
        import torch
        stream = torch.cuda.current_stream(d_field.device)
    m = ctypes.c_double()
    _check(lib().shf_mass_static(ptr, int(precision), int(nx), int(ny), _stream_handle(stream),
                                 ctypes.byref(m)), what="shf_mass_static")
    return m.value


def shf_fma_peak(precision=SHF_FP32, device=0):
    """Measured FMA rate of a GPU in FLOP/s (2 per fused multiply-add)."""
    r = ctypes.c_double()
    _check(lib().shf_fma_peak(int(precision), int(device), ctypes.byref(r)), what="shf_fma_peak")
    return r.value


def shf_create_grid(nx, ny, dx=1.0, precision=SHF_FP32, remap_mode=SHF_REMAP_SHIFT, stream=None):
    h = ctypes.c_void_p()
    _check(lib().shf_create_grid(ctypes.byref(h), int(nx), int(ny), float(dx), int(precision),
                                 int(remap_mode), _stream_handle(stream)), what="shf_create_grid")
    return h.value


def shf_destroy_grid(h):
    _check(lib().shf_destroy_grid(h), h, "shf_destroy_grid")


def shf_set_params(h, a, b, kappa, M, eta, rho, gdot, dt):
    _check(lib().shf_set_params(h, *(float(v) for v in (a, b, kappa, M, eta, rho, gdot, dt))), h,
           "shf_set_params")


def shf_set_fields(h, nx, ny, phi, psi=None, omega=None):
    phi, psi, omega = (_as_field(a, nx, ny) for a in (phi, psi, omega))
    _check(lib().shf_set_fields(h, _dptr(phi), _dptr(psi), _dptr(omega)), h, "shf_set_fields")


def shf_init_noise(h, seed, amp=0.01):
    _check(lib().shf_init_noise(h, int(seed) & (2 ** 64 - 1), float(amp)), h, "shf_init_noise")


def shf_bind_device_fields(h, d_phi, d_psi, d_omega=None):
    _check(lib().shf_bind_device_fields(h, d_phi, d_psi, d_omega), h, "shf_bind_device_fields")


def shf_set_step(h, n):
    _check(lib().shf_set_step(h, int(n)), h, "shf_set_step")


def shf_step(h, nsteps=1):
    _check(lib().shf_step(h, int(nsteps)), h, "shf_step")


KERNEL_KINDS = ("stage1", "colpass_phi", "rowinv_phi", "stage2", "lowmode", "colpass_flow", "rowinv_flow")


def shf_profile_step(h, nsteps):
    """Mean device ms per step of each launch kind of a step ("lowmode" runs for
    FP32 grids only; 0 for FP64)."""
    out = np.zeros(len(KERNEL_KINDS))
    _check(lib().shf_profile_step(h, int(nsteps), _dptr(out), len(KERNEL_KINDS)), h, "shf_profile_step")
    return dict(zip(KERNEL_KINDS, out.tolist()))


def shf_sync(h):
    _check(lib().shf_sync(h), h, "shf_sync")


def shf_get_fields(h, nx, ny):
    phi, psi, omega = (np.empty((ny, nx)) for _ in range(3))
    _check(lib().shf_get_fields(h, _dptr(phi), _dptr(psi), _dptr(omega)), h, "shf_get_fields")
    return phi, psi, omega


def shf_get_time(h):
    n, t, s, K = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    _check(lib().shf_get_time(h, ctypes.byref(n), ctypes.byref(t), ctypes.byref(s), ctypes.byref(K)), h,
           "shf_get_time")
    return n.value, t.value, s.value, K.value


def shf_mass(h):
    m = ctypes.c_double()
    _check(lib().shf_mass(h, ctypes.byref(m)), h, "shf_mass")
    return m.value


def shf_gradient_tensor(h):
    """((G_xx, G_xy, G_yy), (L_par, L_perp)) of the current state."""
    G = np.zeros(3)
    L = np.zeros(2)
    _check(lib().shf_gradient_tensor(h, _dptr(G), _dptr(L)), h, "shf_gradient_tensor")
    return tuple(G), tuple(L)


def _fptr(a):
    return a.ctypes.data_as(_native.P_float) if a is not None else None


def shf_set_fields_f32(h, nx, ny, phi, psi=None, omega=None):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (phi, psi, omega)]
    for a in arrs:
        if a is not None and a.shape != (ny, nx):
            raise ValueError(f"field shape {a.shape} != ({ny}, {nx})")
    _check(lib().shf_set_fields_f32(h, *[_fptr(a) for a in arrs]), h, "shf_set_fields_f32")


def shf_get_fields_f32(h, nx, ny):
    out = [np.empty((ny, nx), dtype=np.float32) for _ in range(3)]
    _check(lib().shf_get_fields_f32(h, *[_fptr(a) for a in out]), h, "shf_get_fields_f32")
    return tuple(out)


def shf_step_host_f32(h, nx, ny, nsteps, phi=None, psi=None, omega=None, out=None):
    """Upload (phi, psi, omega) if phi is given, advance nsteps, download into
    `out` (three float32 (ny, nx) arrays, allocated when None); returns `out`."""
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.float32) for a in (phi, psi, omega)]
    for a in arrs:
        if a is not None and a.shape != (ny, nx):
            raise ValueError(f"field shape {a.shape} != ({ny}, {nx})")
    if out is None:
        out = tuple(np.empty((ny, nx), dtype=np.float32) for _ in range(3))
    for a in out:
        if a is not None and (a.shape != (ny, nx) or a.dtype != np.float32 or not a.flags.c_contiguous):
            raise ValueError("outputs must be C-contiguous float32 arrays of shape (ny, nx)")
    _check(lib().shf_step_host_f32(h, int(nsteps), *[_fptr(a) for a in arrs], *[_fptr(a) for a in out]), h,
           "shf_step_host_f32")
    return out


def shf_autotune(h, cache_path=None, nclasses=8):
    """Tune the launch variants per size class; returns
    [(stage1_points, stage2_points), ...]."""
    out = (ctypes.c_int * (2 * nclasses))()
    path = None if cache_path is None else str(cache_path).encode()
    _check(lib().shf_autotune(h, path, out, 2 * nclasses), h, "shf_autotune")
    pairs = [(out[2 * c], out[2 * c + 1]) for c in range(nclasses)]
    return [t for t in pairs if t[0] > 0]


def shf_structure_factor(h, nbins=0):
    moments = np.zeros(5)
    bins = np.zeros(max(int(nbins), 1))
    _check(lib().shf_structure_factor(h, _dptr(bins) if nbins > 0 else None, int(nbins), _dptr(moments)), h,
           "shf_structure_factor")
    return moments, (bins[:nbins] if nbins > 0 else None)


def shf_save(h, path):
    _check(lib().shf_save(h, str(path).encode()), h, "shf_save")


def shf_load(h, path):
    _check(lib().shf_load(h, str(path).encode()), h, "shf_load")


def shf_create_ensemble(nx, ny, params, dx=None, seeds=None, amp=0.01, precision=SHF_FP32, stream=None):
    nr = len(nx)
    nxa = (ctypes.c_int * nr)(*[int(v) for v in nx])
    nya = (ctypes.c_int * nr)(*[int(v) for v in ny])
    P = np.ascontiguousarray(np.asarray(params, dtype=np.float64).reshape(nr, 8))
    dxa = np.ascontiguousarray(np.asarray(dx, dtype=np.float64)) if dx is not None else None
    sa = (ctypes.c_uint64 * nr)(*[int(v) & (2 ** 64 - 1) for v in seeds]) if seeds is not None else None
    h = ctypes.c_void_p()
    _check(lib().shf_create_ensemble(ctypes.byref(h), nr, nxa, nya, _dptr(dxa), _dptr(P), sa, float(amp),
                                     int(precision), _stream_handle(stream)), what="shf_create_ensemble")
    return h.value


def shf_ensemble_member(h, r):
    v = ctypes.c_void_p()
    _check(lib().shf_ensemble_member(h, int(r), ctypes.byref(v)), h, "shf_ensemble_member")
    return v.value


# --------------------------------------------------------------- convenience

class Grid:
    """Owns one shf_grid handle (a single run)."""

    def __init__(self, nx, ny, dx=1.0, precision=SHF_FP32, remap_mode=SHF_REMAP_SHIFT, stream=None):
        self.nx, self.ny, self.dx, self.precision = int(nx), int(ny), float(dx), int(precision)
        self.handle = shf_create_grid(nx, ny, dx, precision, remap_mode, stream)

    def close(self):
        if self.handle:
            shf_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_params(self, a=1.0, b=1.0, kappa=1.0, M=1.0, eta=1.0, rho=1.0, gdot=0.0, dt=0.005):
        shf_set_params(self.handle, a, b, kappa, M, eta, rho, gdot, dt)

    def set_fields(self, phi, psi=None, omega=None):
        shf_set_fields(self.handle, self.nx, self.ny, phi, psi, omega)

    def init_noise(self, seed, amp=0.01):
        shf_init_noise(self.handle, seed, amp)

    def set_step(self, n):
        shf_set_step(self.handle, n)

    def step(self, nsteps=1):
        shf_step(self.handle, nsteps)

    def sync(self):
        shf_sync(self.handle)

    def profile_step(self, nsteps):
        return shf_profile_step(self.handle, nsteps)

    def get_fields(self):
        return shf_get_fields(self.handle, self.nx, self.ny)

    def set_fields_f32(self, phi, psi=None, omega=None):
        shf_set_fields_f32(self.handle, self.nx, self.ny, phi, psi, omega)

    def get_fields_f32(self):
        return shf_get_fields_f32(self.handle, self.nx, self.ny)

    def step_host_f32(self, nsteps, phi=None, psi=None, omega=None, out=None):
        return shf_step_host_f32(self.handle, self.nx, self.ny, nsteps, phi, psi, omega, out)

    def get_time(self):
        return shf_get_time(self.handle)

    def mass(self):
        return shf_mass(self.handle)

    def structure_factor(self, nbins=0):
        return shf_structure_factor(self.handle, nbins)

    def gradient_tensor(self):
        return shf_gradient_tensor(self.handle)

    def autotune(self, cache_path=None):
        return shf_autotune(self.handle, cache_path)

    def save(self, path):
        shf_save(self.handle, path)

    def load(self, path):
        shf_load(self.handle, path)

    def bind_device_fields(self, phi, psi, omega=None):
        """Adopt torch (or any) device tensors as the state; caller keeps them alive."""
        ptr = lambda t: None if t is None else int(t.data_ptr())
        shf_bind_device_fields(self.handle, ptr(phi), ptr(psi), ptr(omega))


class Member:
    """Non-owning view of one ensemble run."""

    def __init__(self, ens, r):
        self.ens, self.r = ens, r
        self.nx, self.ny = ens.nx[r], ens.ny[r]
        self.handle = shf_ensemble_member(ens.handle, r)

    def set_fields(self, phi, psi=None, omega=None):
        shf_set_fields(self.handle, self.nx, self.ny, phi, psi, omega)

    def get_fields(self):
        return shf_get_fields(self.handle, self.nx, self.ny)

    def mass(self):
        return shf_mass(self.handle)

    def structure_factor(self, nbins=0):
        return shf_structure_factor(self.handle, nbins)

    def gradient_tensor(self):
        return shf_gradient_tensor(self.handle)

    def get_time(self):
        return shf_get_time(self.handle)


class Ensemble:
    """Independent runs of uneven sizes and parameters advanced together."""

    def __init__(self, nx, ny, params, dx=None, seeds=None, amp=0.01, precision=SHF_FP32, stream=None):
        self.nx, self.ny = [int(v) for v in nx], [int(v) for v in ny]
        self.handle = shf_create_ensemble(nx, ny, params, dx, seeds, amp, precision, stream)
        self.members = [Member(self, r) for r in range(len(nx))]

    def close(self):
        if self.handle:
            shf_destroy_grid(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps=1):
        shf_step(self.handle, nsteps)

    def autotune(self, cache_path=None):
        return shf_autotune(self.handle, cache_path)

    def sync(self):
        shf_sync(self.handle)

    def set_step(self, n):
        shf_set_step(self.handle, n)
