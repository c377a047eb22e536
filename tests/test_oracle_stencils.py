"""Pins of the oracle's FFT convention and finite-difference stencils.

Each check compares the oracle against something fixed outside it: a naive DFT
written as explicit sums, the Fourier symbols of the Appendix B stencils
(Eq. p1y and the mu discretisation) derived by hand, and continuum derivatives
computed symbolically by sympy (second-order convergence as h -> 0).
"""
import cmath
import math

import numpy as np
import pytest

import oracle
from oracle import scheme

sympy = pytest.importorskip("sympy")


# ---------------------------------------------------------------- FFT (C-18)

def naive_dft2(f, sign=-1):
    ny, nx = f.shape
    out = np.zeros((ny, nx), dtype=complex)
    for n in range(ny):
        for m in range(nx):
            acc = 0j
            for j in range(ny):
                for i in range(nx):
                    acc += f[j, i] * cmath.exp(sign * 2j * math.pi * (m * i / nx + n * j / ny))
            out[n, m] = acc
    return out


@pytest.mark.parametrize("shape", [(4, 8), (8, 8), (16, 8)])
def test_fft_matches_naive_dft_and_parseval(shape):
    rng = np.random.default_rng(1)
    f = rng.standard_normal(shape)
    F = scheme.fft2(f)
    assert np.allclose(F, naive_dft2(f), atol=1e-12, rtol=0)
    # inverse carries the 1/(Nx Ny) factor and returns the real field
    assert np.allclose(scheme.ifft2_real(F), f, atol=1e-14, rtol=0)
    # Parseval: sum |f|^2 = sum |F|^2 / (Nx Ny)
    assert math.isclose(np.sum(f ** 2), np.sum(np.abs(F) ** 2) / f.size, rel_tol=1e-13)


def test_wavenumber_order_and_nyquist_mask():
    QX, QY, nyq = scheme.wavenumbers(8, 4, 0.5)
    # numpy order: m = 0, 1, 2, 3, -4, -3, -2, -1 ; q = 2 pi m / (N dx)
    m = np.array([0, 1, 2, 3, -4, -3, -2, -1])
    assert np.allclose(QX[0], 2 * math.pi * m / (8 * 0.5))
    n = np.array([0, 1, -2, -1])
    assert np.allclose(QY[:, 0], 2 * math.pi * n / (4 * 0.5))
    assert nyq[:, 4].all() and nyq[2, :].all()
    assert nyq.sum() == 4 + 8 - 1


# ------------------------------------------------ stencil symbols (Eq. p1y)

def mode(nx, ny, m, n, h):
    X, Y = np.meshgrid(np.arange(nx) * h, np.arange(ny) * h)
    qx, qy = 2 * math.pi * m / (nx * h), 2 * math.pi * n / (ny * h)
    return np.exp(1j * (qx * X + qy * Y)), qx, qy


@pytest.mark.parametrize("s", [0.0, 0.3, -0.45, 1.0, -1.0])
@pytest.mark.parametrize("mn", [(1, 0), (3, -2), (-5, 7), (7, 7)])
def test_first_derivative_symbols(s, mn):
    nx, ny, h = 16, 16, 0.7
    e, qx, qy = mode(nx, ny, *mn, h)
    # D_x e^{i q.x} = i sin(q_x h)/h e^{i q.x}
    assert np.allclose(scheme.d_x(e, h), 1j * math.sin(qx * h) / h * e, atol=1e-13)
    # D_y^s: vertical pair gives 2i sin(q_y h); the diagonal pair (i-2, j+1) - (i+2, j-1)
    # gives 2i sin(q_y h - 2 q_x h) for s >= 0, and (i+2, j+1) - (i-2, j-1) gives
    # 2i sin(q_y h + 2 q_x h) for s < 0.
    if s >= 0:
        sym = ((1 - s / 2) * math.sin(qy * h) + (s / 2) * math.sin(qy * h - 2 * qx * h)) / h
    else:
        sym = ((1 + s / 2) * math.sin(qy * h) - (s / 2) * math.sin(qy * h + 2 * qx * h)) / h
    assert np.allclose(scheme.d_y_sheared(e, s, h), 1j * sym * e, atol=1e-13)


@pytest.mark.parametrize("s", [0.0, 0.25, -0.5])
def test_sheared_laplacian_symbol(s):
    nx, ny, h = 16, 8, 1.3
    e, qx, qy = mode(nx, ny, 3, -1, h)
    dxx = -(2 - 2 * math.cos(qx * h)) / h ** 2
    dyy = -(2 - 2 * math.cos(qy * h)) / h ** 2
    dxy = -math.sin(qx * h) * math.sin(qy * h) / h ** 2
    sym = (1 + s * s) * dxx - 2 * s * dxy + dyy
    assert np.allclose(scheme.lap_sheared(e, s, h), sym * e, atol=1e-13)


@pytest.mark.parametrize("s", [0.0, 0.4, -0.3])
def test_stencil_symbols_tend_to_sheared_gradient(s):
    """As h -> 0 the symbols tend to i q_x, i (q_y - s q_x) and -(q_x^2 + (q_y - s q_x)^2):
    the stencils discretise grad_c of Eq. coshearedNabluFinal (second order)."""
    errs = []
    for N in (32, 64, 128):
        L = 2 * math.pi
        h = L / N
        e, qx, qy = mode(N, N, 2, 3, h)
        dy = scheme.d_y_sheared(e, s, h) / e
        lap = scheme.lap_sheared(e, s, h) / e
        err = abs(dy[0, 0] - 1j * (qy - s * qx)) + abs(lap[0, 0] + qx ** 2 + (qy - s * qx) ** 2)
        errs.append(err)
    assert errs[0] / errs[1] > 3.6 and errs[1] / errs[2] > 3.6


# ---------------------------------------- continuum limits via sympy (2nd order)

X_, Y_ = sympy.symbols("x y", real=True)
PHI_EXPR = sympy.Rational(3, 10) * sympy.cos(X_ + 2 * Y_) + sympy.Rational(1, 5) * sympy.sin(3 * X_ - Y_)
PSI_EXPR = sympy.Rational(1, 2) * sympy.sin(2 * X_ + Y_) - sympy.Rational(1, 4) * sympy.cos(X_ - 3 * Y_)


def sample(expr, N):
    f = sympy.lambdify((X_, Y_), expr, "numpy")
    h = 2 * math.pi / N
    X, Y = np.meshgrid(np.arange(N) * h, np.arange(N) * h)
    return np.asarray(f(X, Y), dtype=float) * np.ones_like(X), h


def convergence(errfun):
    errs = [errfun(N) for N in (32, 64, 128)]
    return errs, errs[0] / errs[1], errs[1] / errs[2]


@pytest.mark.parametrize("s", [0.0, 0.35, -0.2])
def test_bracket_is_shear_invariant_in_the_continuum_limit(s):
    """Section V: the s terms of (d_y - s d_x) cancel inside the advective bracket,
    so the discrete bracket with any s tends to d_y psi d_x phi - d_x psi d_y phi."""
    exact = sympy.diff(PSI_EXPR, Y_) * sympy.diff(PHI_EXPR, X_) - sympy.diff(PSI_EXPR, X_) * sympy.diff(PHI_EXPR, Y_)

    def err(N):
        phi, h = sample(PHI_EXPR, N)
        psi, _ = sample(PSI_EXPR, N)
        ex, _ = sample(exact, N)
        return np.abs(scheme.bracket(psi, phi, s, h) - ex).max()

    errs, r1, r2 = convergence(err)
    assert errs[-1] < 2e-2
    assert 3.5 < r1 < 4.5 and 3.5 < r2 < 4.5


def test_advection_moves_pattern_downstream():
    """Eq. advective with v = curl(psi z) = (d_y psi, -d_x psi): for psi = A sin(y) the
    flow is v_x = A cos(y), and one Euler step must equal phi - dt v.grad(phi)."""
    A = 0.3
    psi_e = A * sympy.sin(Y_)
    phi_e = sympy.cos(2 * X_)
    vgrad = sympy.diff(psi_e, Y_) * sympy.diff(phi_e, X_) - sympy.diff(psi_e, X_) * sympy.diff(phi_e, Y_)
    p = oracle.Params(dt=0.01)

    def err(N):
        phi, h = sample(phi_e, N)
        psi, _ = sample(psi_e, N)
        vg, _ = sample(vgrad, N)
        p2 = oracle.Params(dt=p.dt, dx=h)
        return np.abs((scheme.advect(phi, psi, 0.0, p2) - phi) / p.dt + vg).max()

    errs, r1, r2 = convergence(err)
    assert errs[-1] < 5e-3 and r1 > 3.5 and r2 > 3.5
    # sign: at x = pi/4 (d_x phi = -2), y = 0 (v_x = A > 0) phi must increase
    # (the crest upstream at x = 0 moves in the +x direction).
    N = 64
    phi, h = sample(phi_e, N)
    psi, _ = sample(psi_e, N)
    d = scheme.advect(phi, psi, 0.0, oracle.Params(dt=0.01, dx=h)) - phi
    assert d[0, N // 8] > 0


@pytest.mark.parametrize("s", [0.0, 0.3, -0.4])
def test_chemical_potential_and_body_force_continuum(s):
    """mu = -a phi + b phi^3 - kappa lap_c phi (Eq. mu1 with grad_c) and
    F = [curl(phi grad mu)].z = d_x phi d_y mu - d_y phi d_x mu (Eq. vorticity):
    both converge at second order, and the s terms cancel in F (Section V)."""
    a, b, kappa = 0.7, 1.3, 0.9
    def dyc(e):  # the y component of grad_c, Eq. coshearedNabluFinal
        return sympy.diff(e, Y_) - s * sympy.diff(e, X_)
    lapc = sympy.diff(PHI_EXPR, X_, 2) + dyc(dyc(PHI_EXPR))
    mu_e = -a * PHI_EXPR + b * PHI_EXPR ** 3 - kappa * lapc
    # the curl of phi grad mu, taken literally and symbolically
    Fx = PHI_EXPR * sympy.diff(mu_e, X_)
    Fy = PHI_EXPR * sympy.diff(mu_e, Y_)
    curl = sympy.diff(Fy, X_) - sympy.diff(Fx, Y_)
    # the co-sheared frame writes the same quantity with grad_c; it is s-independent
    # only after the cancellation, so compare against the lab-frame curl of the
    # co-sheared mu (the form of Eq. equation2).
    def err_mu(N):
        phi, h = sample(PHI_EXPR, N)
        ex, _ = sample(mu_e, N)
        p = oracle.Params(a=a, b=b, kappa=kappa, dx=h)
        return np.abs(scheme.chemical_potential(phi, s, p) - ex).max()

    def err_F(N):
        phi, h = sample(PHI_EXPR, N)
        mu, _ = sample(mu_e, N)
        ex, _ = sample(curl, N)
        return np.abs(scheme.body_force_curl(phi, mu, s, h) - ex).max()

    for fn in (err_mu, err_F):
        errs, r1, r2 = convergence(fn)
        assert 3.2 < r1 < 4.8 and 3.6 < r2 < 4.4, (fn.__name__, errs)
