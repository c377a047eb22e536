"""Pins of the oracle's spectral solves (Appendix B, items 1-3 and the
zero-Reynolds-number algorithm).

* Dense brute force: the co-sheared operators are built as dense real-space
  matrices from the periodic Fourier differentiation matrix (the cotangent
  formula for even N, Trefethen, "Spectral Methods in MATLAB", ch. 3), with no
  FFT and no wavenumber formula, and the semi-implicit updates are solved with
  dense linear algebra.  The even-N differentiation matrix annihilates the
  Nyquist mode, which is the oracle's Nyquist reading.
* Linear spinodal dispersion: the growth rate of a small mode tends to
  sigma = M k^2 (a - kappa k^2) (Eqs. phi1, mu1 linearised) as dt -> 0.
* Tilted-mode damping: under shear a passive mode's y-wavevector in the
  laboratory is k_y - gdot t k_x, so its hyperdiffusive decay integrates
  |k(t)|^4 over time.
* The Stokes limit of the inertial Crank-Nicolson solve.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import scheme
from paper_0710_5912_gb300 import inputs

sympy = pytest.importorskip("sympy")


def fourier_diff_matrix(N, L):
    """Periodic spectral first-derivative matrix on N (even) points of a period L."""
    h = 2 * math.pi / N
    D = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            if i != j:
                D[i, j] = 0.5 * (-1) ** (i - j) / math.tan((i - j) * h / 2)
    return D * (2 * math.pi / L)


def dense_ops(nx, ny, dx, s):
    Dx1 = fourier_diff_matrix(nx, nx * dx)
    Dy1 = fourier_diff_matrix(ny, ny * dx)
    Dx = np.kron(np.eye(ny), Dx1)      # acts on row-major flattening p = j*nx + i
    Dy = np.kron(Dy1, np.eye(nx))
    Dyc = Dy - s * Dx                  # y component of grad_c (Eq. coshearedNabluFinal)
    lapc = Dx @ Dx + Dyc @ Dyc
    return lapc


def drop_nyquist(f):
    ny, nx = f.shape
    F = np.fft.fft2(f)
    F[ny // 2, :] = 0
    F[:, nx // 2] = 0
    return np.real(np.fft.ifft2(F))


def test_differentiation_matrix_sanity():
    N, L = 8, 3.0
    D = fourier_diff_matrix(N, L)
    x = np.arange(N) * L / N
    q = 2 * math.pi / L
    assert np.allclose(D @ np.sin(q * x), q * np.cos(q * x), atol=1e-13)
    assert np.allclose(D @ np.cos(4 * q * x), 0.0, atol=1e-13)   # Nyquist annihilated


def random_field(nx, ny, seed):
    return drop_nyquist(inputs.quench_noise(nx, ny, seed, 1.0))


@pytest.mark.parametrize("s", [0.0, 0.37, -0.5])
@pytest.mark.parametrize("shape", [(8, 8), (8, 4)])
def test_cahn_hilliard_update_matches_dense_solve(s, shape):
    nx, ny = shape
    p = oracle.Params(a=0.8, b=1.1, kappa=0.9, M=0.7, dt=0.05, dx=0.9)
    phi_half = random_field(nx, ny, 1)
    f = random_field(nx, ny, 2)
    QX, QY, nyq = scheme.wavenumbers(nx, ny, p.dx)
    got = scheme.cahn_hilliard_spectral(phi_half, f, s, p, QX, QY, nyq)
    # d_t phi = M L(-a phi + b f - kappa L phi), L = lap_c: Euler on L, CN on L^2
    Lc = dense_ops(nx, ny, p.dx, s)
    I = np.eye(nx * ny)
    A = I + 0.5 * p.dt * p.kappa * p.M * Lc @ Lc
    rhs = (I - p.dt * p.a * p.M * Lc - 0.5 * p.dt * p.kappa * p.M * Lc @ Lc) @ phi_half.ravel() \
        + p.dt * p.b * p.M * Lc @ f.ravel()
    want = np.linalg.solve(A, rhs).reshape(ny, nx)
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("s", [0.0, 0.21, -0.44])
@pytest.mark.parametrize("shape", [(8, 8), (16, 8)])
def test_stokes_solve_matches_dense_biharmonic(s, shape):
    """Zero-Reynolds-number algorithm: 0 = -eta lap_c^2 psi - F, min-norm solution."""
    nx, ny = shape
    p = oracle.Params(eta=1.7, rho=0.0, dx=1.0)
    F = random_field(nx, ny, 3)
    QX, QY, nyq = scheme.wavenumbers(nx, ny, p.dx)
    got = scheme.stokes_solve(F, s, p, QX, QY, nyq)
    Lc = dense_ops(nx, ny, p.dx, s)
    want = np.linalg.lstsq(p.eta * Lc @ Lc, -F.ravel(), rcond=1e-12)[0].reshape(ny, nx)
    assert np.allclose(got, want, atol=1e-12 * np.abs(want).max())


@pytest.mark.parametrize("s", [0.0, 0.3, -0.25])
def test_vorticity_and_poisson_match_dense_solve(s):
    nx, ny = 8, 8
    p = oracle.Params(eta=0.6, rho=1.4, dt=0.1, dx=1.0)
    omega_star = random_field(nx, ny, 4)
    omega_star -= omega_star.mean()
    F = random_field(nx, ny, 5)
    QX, QY, nyq = scheme.wavenumbers(nx, ny, p.dx)
    psi, omega = scheme.vorticity_poisson_solve(omega_star, F, s, p, QX, QY, nyq)
    Lc = dense_ops(nx, ny, p.dx, s)
    I = np.eye(nx * ny)
    nu = p.eta / p.rho
    # CN on d_t omega = nu lap_c omega + g, g = -F / rho (Eqs. vortNum, G)
    w = np.linalg.solve(I - 0.5 * p.dt * nu * Lc,
                        (I + 0.5 * p.dt * nu * Lc) @ omega_star.ravel() - p.dt * F.ravel() / p.rho)
    w -= w.mean()
    ps = np.linalg.lstsq(-Lc, w, rcond=1e-12)[0]          # omega = -lap_c psi
    assert np.allclose(omega.ravel(), w, atol=1e-12 * np.abs(w).max())
    assert np.allclose(psi.ravel(), ps, atol=1e-12 * np.abs(ps).max())


@pytest.mark.parametrize("s", [0.3, -0.41])
def test_poisson_on_analytic_sheared_mode(s):
    """omega = cos(q.x) with phi = 0 (no body force): after one step psi must satisfy
    -lap_c psi = omega pointwise, lap_c applied symbolically (sympy)."""
    nx = ny = 32
    m, n = 3, -2
    gdot, dt = s, 1.0          # s^{n+1} = s after the first step (no wrap for |s| < 1/2)
    p = oracle.Params(rho=2.0, eta=0.5, gdot=gdot, dt=dt)
    omega0 = inputs.cosine_mode(nx, ny, m, n)
    zero = np.zeros((ny, nx))
    phi1, psi1, omega1 = scheme.step(zero, zero, omega0, 0, p)
    x, y = sympy.symbols("x y", real=True)
    qx, qy = 2 * sympy.pi * m / nx, 2 * sympy.pi * n / ny
    c = sympy.cos(qx * x + qy * y)
    dyc = lambda e: sympy.diff(e, y) - s * sympy.diff(e, x)
    lapc_c = sympy.simplify((sympy.diff(c, x, 2) + dyc(dyc(c))) / c)     # = -k^2
    k2 = float(-lapc_c)
    nu = p.eta / p.rho
    cn = (1 - 0.5 * dt * nu * k2) / (1 + 0.5 * dt * nu * k2)             # CN factor
    assert np.allclose(omega1, cn * omega0, atol=1e-14)
    assert np.allclose(psi1, cn * omega0 / k2, atol=1e-14)
    assert np.abs(phi1).max() == 0.0


def mode_amplitude(f, m, n):
    ny, nx = f.shape
    return 2.0 * np.fft.fft2(f)[n % ny, m % nx].real / (nx * ny)


@pytest.mark.parametrize("mn", [(2, 1), (1, 3), (0, 2)])
def test_linear_spinodal_dispersion(mn):
    """One step of a tiny mode grows by exp(sigma dt) + O(dt^2) with
    sigma = M k^2 (a - kappa k^2): the measured rate converges at first order."""
    nx = ny = 32
    A = 1e-8
    p0 = dict(a=1.0, b=1.0, kappa=1.0, M=1.0, eta=1.0, rho=0.0, gdot=0.0, dx=1.0)
    qx, qy = 2 * math.pi * mn[0] / nx, 2 * math.pi * mn[1] / ny
    k2 = qx * qx + qy * qy
    sigma = p0["M"] * k2 * (p0["a"] - p0["kappa"] * k2)
    phi0 = inputs.cosine_mode(nx, ny, *mn, amp=A)
    zero = np.zeros_like(phi0)
    errs = []
    for dt in (0.8, 0.4, 0.2):
        p = oracle.Params(dt=dt, **p0)
        phi1, psi1, _ = scheme.step(phi0, zero, zero, 0, p)
        G = mode_amplitude(phi1, *mn) / A
        errs.append(abs(math.log(G) / dt - sigma))
        # textbook IMEX amplification (Euler on lambda_e, CN on lambda_i)
        le, li = p.a * p.M * k2, -p.kappa * p.M * k2 * k2
        assert math.isclose(G, (1 + dt * le + 0.5 * dt * li) / (1 - 0.5 * dt * li), rel_tol=1e-12)
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


def test_tilted_mode_hyperdiffusion_follows_lab_wavevector():
    """Shear tilts a passive mode: its laboratory wavevector is (k_x, k_y - gdot t k_x).
    With a = b = 0 the amplitude decays as exp(-kappa M int |k(t)|^4 dt); the scheme
    reproduces the product of per-step CN factors at k(s^n) exactly and the
    continuum integral to first order in dt.  The opposite tilt sign is excluded."""
    nx = ny = 32
    m, n = 2, 1
    qx, qy = 2 * math.pi * m / nx, 2 * math.pi * n / ny
    T, gdot = 2.0, 0.2
    A = 1e-6

    def run(dt):
        p = oracle.Params(a=0.0, b=0.0, kappa=1.0, M=1.0, rho=0.0, eta=1.0, gdot=gdot, dt=dt)
        phi = inputs.cosine_mode(nx, ny, m, n, amp=A)
        zero = np.zeros_like(phi)
        prod = 1.0
        nsteps = int(round(T / dt))
        for k in range(nsteps):
            s = scheme.strain(k, gdot, dt, nx, ny)[0]
            kk = qx * qx + (qy - s * qx) ** 2
            c = 0.5 * dt * kk * kk
            prod *= (1 - c) / (1 + c)
            phi, zero, _ = scheme.step(phi, zero, np.zeros_like(phi), k, p)
        return mode_amplitude(phi, m, n) / A, prod

    def cont(sign):
        t = sympy.symbols("t", real=True)
        ky = qy + sign * gdot * t * qx
        return math.exp(-float(sympy.integrate((qx ** 2 + ky ** 2) ** 2, (t, 0, T))))

    errs = []
    for dt in (0.1, 0.05, 0.025):
        amp, prod = run(dt)
        assert math.isclose(amp, prod, rel_tol=1e-9)
        errs.append(abs(math.log(amp) - math.log(cont(-1))))
    assert 1.7 < errs[0] / errs[1] < 2.3
    wrong = abs(math.log(amp) - math.log(cont(+1)))
    assert wrong > 20 * errs[-1]


def test_inertial_solve_tends_to_stokes_solve():
    """As rho -> 0 the CN vorticity update becomes the Stokes solve: the CN average
    (omega^{n+1} + omega*)/2 tends to -lap_c psi_Stokes."""
    nx = ny = 16
    s = 0.27
    F = random_field(nx, ny, 7)
    F -= F.mean()
    omega_star = random_field(nx, ny, 8)
    omega_star -= omega_star.mean()
    QX, QY, nyq = scheme.wavenumbers(nx, ny, 1.0)
    eta = 1.3
    psi_s = scheme.stokes_solve(F, s, oracle.Params(eta=eta, rho=0.0), QX, QY, nyq)
    _, omega_new = scheme.vorticity_poisson_solve(omega_star, F, s,
                                                  oracle.Params(eta=eta, rho=1e-12, dt=0.01),
                                                  QX, QY, nyq)
    k2 = scheme.sheared_k2(QX, QY, s)
    want = np.real(np.fft.ifft2(k2 * np.fft.fft2(psi_s)))
    got = 0.5 * (omega_new + drop_nyquist(omega_star))
    assert np.allclose(got, want, atol=1e-6 * np.abs(want).max())
