"""Pins of the FP32 psi error model (fp32_model.psi32_model_ratio) on the CPU.

The model must accept psi computed from the oracle's own state with FP32
arithmetic in the flow solve (single-precision products, transforms and
division), at a ratio of order one, and must reject plausible mistakes: a
wrong sheared wavenumber, a dropped term of the chemical potential, a sign
error in the body-force curl, and a 1e-4 relative perturbation of psi (the
model admits uniform relative errors of about 2e-5, the FP32 tolerance)."""
import numpy as np
import pytest
import scipy.fft as sfft

import oracle
from fp32_model import PSI32_MODEL_MAX, psi32_model_ratio
from paper_0710_5912_gb300 import inputs

f32 = np.float32


def fp32_flow_solve(phi, omega_star, s, p, flip_sign=False, drop_cubic=False, s_k2=None):
    """psi^{n+1} of Appendix B items 2-3 (or the Stokes solve) with every
    operation after phi^{n+1} in binary32: stencils, transforms, multipliers."""
    ny, nx = phi.shape
    ph = phi.astype(f32)
    h = f32(p.dx)

    def sh(a, di, dj):
        return np.roll(a, (-dj, -di), axis=(0, 1))

    def dx(a):
        return (sh(a, 1, 0) - sh(a, -1, 0)) / (f32(2) * h)

    def dy(a):
        w1 = f32(abs(s) / 2)
        w0 = f32(1) - w1
        d = -2 if s >= 0 else 2
        return (w0 * (sh(a, 0, 1) - sh(a, 0, -1)) + w1 * (sh(a, d, 1) - sh(a, -d, -1))) / (f32(2) * h)

    ss = f32(s)
    dxx = (sh(ph, 1, 0) - f32(2) * ph + sh(ph, -1, 0)) / (h * h)
    dyy = (sh(ph, 0, 1) - f32(2) * ph + sh(ph, 0, -1)) / (h * h)
    dxy = (sh(ph, 1, 1) - sh(ph, 1, -1) - sh(ph, -1, 1) + sh(ph, -1, -1)) / (f32(4) * h * h)
    lap = (f32(1) + ss * ss) * dxx - f32(2) * ss * dxy + dyy
    cubic = f32(0) if drop_cubic else f32(p.b) * ((ph * ph) * ph)
    mu = -f32(p.a) * ph + cubic - f32(p.kappa) * lap
    F = dx(ph) * dy(mu) + (1 if flip_sign else -1) * dy(ph) * dx(mu)
    QX, QY, nyq = oracle.wavenumbers(nx, ny, p.dx)
    k2 = oracle.sheared_k2(QX, QY, s if s_k2 is None else s_k2).astype(f32)
    k0 = k2 == 0
    safe = np.where(k0, f32(1), k2)
    if p.rho == 0:
        Psi = sfft.fft2(-F / f32(p.eta)) / (safe * safe)
    else:
        W = sfft.fft2(omega_star.astype(f32))
        G = sfft.fft2(-F / f32(p.rho))
        cn = f32(0.5 * p.dt * p.eta / p.rho) * k2
        W = ((f32(1) - cn) * W + f32(p.dt) * G) / (f32(1) + cn)
        W[k0] = 0
        Psi = W / safe
    Psi[k0] = 0
    Psi[nyq] = 0
    assert Psi.dtype == np.complex64
    return np.real(sfft.ifft2(Psi)).astype(np.float64)


def reference(phi, omega_star, s, p):
    """The oracle's psi^{n+1} from the same phi^{n+1} and omega* (FP64)."""
    QX, QY, nyq = oracle.wavenumbers(*phi.shape[::-1], p.dx)
    psi, _ = oracle.flow_substep(phi, omega_star, s, p, QX, QY, nyq)
    return psi


CASES = [
    ("quench 256^2 Stokes", 256, 256, 0.0, 0.01, 0.003),
    ("quench 256^2 inertial", 256, 256, 1.0, 0.01, 0.003),
    ("rough 128x32 Stokes", 128, 32, 0.0, 0.5, 0.3),
    ("rough 64^2 inertial", 64, 64, 0.7, 0.5, -0.3),
]


@pytest.mark.parametrize("name,nx,ny,rho,amp,s", CASES)
def test_fp32_solve_fits_the_model(name, nx, ny, rho, amp, s):
    p = oracle.Params(a=0.9, b=1.1, kappa=0.8, M=1.2, eta=0.6, rho=rho, gdot=0.0, dt=0.01, dx=0.9)
    phi = inputs.quench_noise(nx, ny, 5, amp)
    om = inputs.quench_noise(nx, ny, 6, 0.05) if rho > 0 else np.zeros((ny, nx))
    want = reference(phi, om, s, p)
    q = psi32_model_ratio(fp32_flow_solve(phi, om, s, p), want, s, p.dx, rho)
    assert 0.2 <= q <= PSI32_MODEL_MAX / 2, (name, q)


@pytest.mark.parametrize("name,nx,ny,rho,amp,s", CASES)
def test_model_rejects_planted_mistakes(name, nx, ny, rho, amp, s):
    p = oracle.Params(a=0.9, b=1.1, kappa=0.8, M=1.2, eta=0.6, rho=rho, gdot=0.0, dt=0.01, dx=0.9)
    phi = inputs.quench_noise(nx, ny, 5, amp)
    om = inputs.quench_noise(nx, ny, 6, 0.05) if rho > 0 else np.zeros((ny, nx))
    want = reference(phi, om, s, p)
    bad = {
        "sign of the curl": fp32_flow_solve(phi, om, s, p, flip_sign=True),
        "unsheared k": fp32_flow_solve(phi, om, s, p, s_k2=s + 0.25),
        "1e-4 perturbation": want * (1 + 1e-4),
    }
    if amp > 0.1:   # the cubic term is below FP32 resolution at quench amplitudes
        bad["dropped cubic"] = fp32_flow_solve(phi, om, s, p, drop_cubic=True)
    for what, psi in bad.items():
        q = psi32_model_ratio(psi, want, s, p.dx, rho)
        assert q > 3 * PSI32_MODEL_MAX, (name, what, q)
