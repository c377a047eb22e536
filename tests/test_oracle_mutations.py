"""The pins must catch plausible slips in the oracle.

Each case plants one mistake in the oracle (on the CPU, by monkeypatching one
function) -- a wrong sign, a dropped term, a transposed operand, a wrong index
or a wrong time level -- and runs the pins that should notice; at least one of
them must fail.  This is the evidence that the pins in test_oracle_*.py
constrain every part of the scheme rather than only re-running it.
"""
import math

import numpy as np
import pytest

from oracle import scheme
import test_oracle_spectral as tsp
import test_oracle_stencils as tst
import test_oracle_step as tstep


def _mut_dy_diag_index(f, s, h):
    vert = scheme.shifted(f, 0, 1) - scheme.shifted(f, 0, -1)
    if s >= 0.0:   # diagonal pair taken on the wrong side
        diag = scheme.shifted(f, 2, 1) - scheme.shifted(f, -2, -1)
        return ((1.0 - s / 2.0) * vert + (s / 2.0) * diag) / (2.0 * h)
    diag = scheme.shifted(f, 2, 1) - scheme.shifted(f, -2, -1)
    return ((1.0 + s / 2.0) * vert - (s / 2.0) * diag) / (2.0 * h)


def _mut_lap_cross_sign(f, s, h):
    dxx = (scheme.shifted(f, 1, 0) - 2.0 * f + scheme.shifted(f, -1, 0)) / (h * h)
    dyy = (scheme.shifted(f, 0, 1) - 2.0 * f + scheme.shifted(f, 0, -1)) / (h * h)
    dxy = (scheme.shifted(f, 1, 1) - scheme.shifted(f, 1, -1) - scheme.shifted(f, -1, 1)
           + scheme.shifted(f, -1, -1)) / (4.0 * h * h)
    return (1.0 + s * s) * dxx + 2.0 * s * dxy + dyy


def _mut_bracket_transposed(A, B, s, h):
    return scheme.d_x(A, h) * scheme.d_y_sheared(B, s, h) - scheme.d_y_sheared(A, s, h) * scheme.d_x(B, h)


def _mut_mu_no_cubic(phi, s, p):
    return -p.a * phi - p.kappa * scheme.lap_sheared(phi, s, p.dx)


def _mut_force_sign(phi, mu, s, h):
    return -(scheme.d_x(phi, h) * scheme.d_y_sheared(mu, s, h) - scheme.d_y_sheared(phi, s, h) * scheme.d_x(mu, h))


def _mut_k2_tilt_sign(QX, QY, s):
    return QX * QX + (QY + s * QX) ** 2


def _mut_strain_off_by_one(n, gdot, dt, nx, ny):
    r = nx // ny
    total = (gdot * dt) * float(n + 1)
    K = math.floor(total / r + 0.5)
    return total - K * r, K


def _mut_remap_direction(f, shift_per_row):
    out = np.empty_like(f)
    for j in range(f.shape[0]):
        out[j] = np.roll(f[j], -(j * shift_per_row) % f.shape[1])
    return out


_orig_ch = scheme.cahn_hilliard_spectral


def _mut_ch_explicit_k4(phi_half, f, s, p, QX, QY, nyquist):
    # treat the k^4 term fully explicitly (drops the Crank-Nicolson half)
    dt = p.dt
    k2 = scheme.sheared_k2(QX, QY, s)
    Phi = np.fft.fft2(phi_half)
    num = (1.0 + dt * p.a * p.M * k2 - dt * p.kappa * p.M * k2 * k2) * Phi - dt * p.b * p.M * k2 * np.fft.fft2(f)
    num[nyquist] = 0
    return np.real(np.fft.ifft2(num))


def _mut_stokes_k2(F, s, p, QX, QY, nyquist):
    k2 = scheme.sheared_k2(QX, QY, s)
    k0 = k2 == 0
    Psi = np.fft.fft2(-F / p.eta) / np.where(k0, 1.0, k2)
    Psi[k0] = 0
    Psi[nyquist] = 0
    return np.real(np.fft.ifft2(Psi))


def _mut_vort_cn_sign(omega_star, F, s, p, QX, QY, nyquist):
    dt = p.dt
    k2 = scheme.sheared_k2(QX, QY, s)
    k0 = k2 == 0
    nu = p.eta / p.rho
    W = np.fft.fft2(omega_star)
    G = np.fft.fft2(-F / p.rho)
    W_new = ((1.0 + 0.5 * dt * nu * k2) * W + dt * G) / (1.0 + 0.5 * dt * nu * k2)
    W_new[k0] = 0
    W_new[nyquist] = 0
    Psi = W_new / np.where(k0, 1.0, k2)
    Psi[k0] = 0
    return np.real(np.fft.ifft2(Psi)), np.real(np.fft.ifft2(W_new))


def _mut_tensor_unsheared(phi, s, dx=1.0):
    # laboratory y-derivative taken as the plain co-sheared d_y (tilt dropped)
    return _orig_gradient_tensor(phi, 0.0, dx)


_orig_gradient_tensor = scheme.gradient_tensor


def _run_first_failing(checks):
    for fn in checks:
        try:
            fn()
        except AssertionError:
            return True
    return False


MUTATIONS = {
    "dy_diag_index": ("d_y_sheared", _mut_dy_diag_index,
                      [lambda: tst.test_first_derivative_symbols(0.3, (3, -2))]),
    "lap_cross_sign": ("lap_sheared", _mut_lap_cross_sign,
                       [lambda: tst.test_sheared_laplacian_symbol(0.25)]),
    "bracket_transposed": ("bracket", _mut_bracket_transposed,
                           [lambda: tst.test_bracket_is_shear_invariant_in_the_continuum_limit(0.0)]),
    "mu_no_cubic": ("chemical_potential", _mut_mu_no_cubic,
                    [lambda: tst.test_chemical_potential_and_body_force_continuum(0.3)]),
    "force_sign": ("body_force_curl", _mut_force_sign,
                   [lambda: tst.test_chemical_potential_and_body_force_continuum(0.0)]),
    "k2_tilt_sign": ("sheared_k2", _mut_k2_tilt_sign,
                     [lambda: tsp.test_stokes_solve_matches_dense_biharmonic(0.21, (8, 8))]),
    "strain_off_by_one": ("strain", _mut_strain_off_by_one,
                          [tstep.test_strain_sawtooth_wraps_inclusively]),
    "remap_direction": ("remap_rows", _mut_remap_direction,
                        [tstep.test_remap_is_the_stated_permutation]),
    "ch_explicit_k4": ("cahn_hilliard_spectral", _mut_ch_explicit_k4,
                       [lambda: tsp.test_cahn_hilliard_update_matches_dense_solve(0.37, (8, 8))]),
    "stokes_k2": ("stokes_solve", _mut_stokes_k2,
                  [lambda: tsp.test_stokes_solve_matches_dense_biharmonic(0.0, (8, 8))]),
    "vort_cn_sign": ("vorticity_poisson_solve", _mut_vort_cn_sign,
                     [lambda: tsp.test_vorticity_and_poisson_match_dense_solve(0.3)]),
    "tensor_unsheared": ("gradient_tensor", _mut_tensor_unsheared,
                         [tstep.test_gradient_tensor_matches_analytic_lab_derivatives]),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pins_catch_planted_mistake(name, monkeypatch):
    attr, fn, checks = MUTATIONS[name]
    monkeypatch.setattr(scheme, attr, fn)
    assert _run_first_failing(checks), f"no pin caught the planted mistake {name}"


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_same_pins_pass_on_the_real_oracle(name):
    _, _, checks = MUTATIONS[name]
    assert not _run_first_failing(checks)
