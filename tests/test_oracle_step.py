"""Pins of the oracle's full time step and diagnostics.

* an independent loop-by-loop restatement of one step on tiny grids (explicit
  stencil indices of Eq. p1y, explicit DFT sums) -- catches index, roll-direction
  and ordering slips in the vectorised oracle;
* exact invariants: conservation of the mean of phi (Eq. phi1 is a conservation
  law; D_x and D_y^s are commuting antisymmetric operators, so the bracket sums
  to zero), the phi -> -phi symmetry of model H (bit-exact in IEEE arithmetic);
* the strain sawtooth of Section V and the remap that keeps the laboratory field
  continuous across a wrap (the laboratory wavevector of a frozen mode follows
  k_y - gdot t k_x through the wrap);
* second-order self-convergence under grid refinement with dt ~ h^2;
* structure-factor moments of a single mode in closed form (Eq. L_structure).
"""
import cmath
import math

import numpy as np
import pytest

import oracle
from oracle import scheme
from paper_0710_5912_gb300 import inputs


# ------------------------------------------------------------------ strain

def test_strain_sawtooth_wraps_inclusively():
    gd = 2.0 ** -6          # gdot*dt exact: the wrap falls exactly on step 32
    for n, s_want, K_want in [(0, 0.0, 0), (31, 31 / 64, 0), (32, -0.5, 1), (33, -31 / 64, 1),
                              (96, -0.5, 2), (100, -0.4375, 2)]:
        s, K = scheme.strain(n, 1.0, gd, 64, 64)
        assert (s, K) == (s_want, K_want)
    # Lx = 2 Ly: the strain wraps at 1 by 2
    assert scheme.strain(64, 1.0, gd, 128, 64) == (-1.0, 1)
    assert scheme.strain(63, 1.0, gd, 128, 64) == (63 / 64, 0)
    # negative shear rate wraps the other way; s stays in [-r/2, r/2)
    for n in range(0, 500, 7):
        s, K = scheme.strain(n, -0.013, 0.7, 64, 64)
        assert -0.5 <= s < 0.5
        assert math.isclose(s + K, -0.013 * 0.7 * n, abs_tol=1e-12)


# ------------------------------------------------- loop-by-loop restatement

def loop_step(phi, psi, omega, n, p, remap=True):
    """One step written point by point (explicit indices, explicit DFT sums)."""
    ny, nx = len(phi), len(phi[0])
    h, dt = p.dx, p.dt
    r = nx // ny

    def strain(k):
        tot = (p.gdot * p.dt) * k
        K = math.floor(tot / r + 0.5)
        return tot - K * r, K

    def at(f, i, j):
        return f[j % ny][i % nx]

    def dx_(f, i, j):
        return (at(f, i + 1, j) - at(f, i - 1, j)) / (2 * h)

    def dy_(f, i, j, s):
        if s >= 0:
            return ((1 - s / 2) * (at(f, i, j + 1) - at(f, i, j - 1))
                    + s / 2 * (at(f, i - 2, j + 1) - at(f, i + 2, j - 1))) / (2 * h)
        return ((1 + s / 2) * (at(f, i, j + 1) - at(f, i, j - 1))
                - s / 2 * (at(f, i + 2, j + 1) - at(f, i - 2, j - 1))) / (2 * h)

    def dft(f, sign):
        out = [[0j] * nx for _ in range(ny)]
        for nn in range(ny):
            for mm in range(nx):
                acc = 0j
                for j in range(ny):
                    for i in range(nx):
                        acc += f[j][i] * cmath.exp(sign * 2j * math.pi * (mm * i / nx + nn * j / ny))
                out[nn][mm] = acc if sign < 0 else acc / (nx * ny)
        return out

    def k2(mm, nn, s):
        ms = mm if mm < nx // 2 else mm - nx
        ns = nn if nn < ny // 2 else nn - ny
        qx, qy = 2 * math.pi * ms / (nx * h), 2 * math.pi * ns / (ny * h)
        return qx * qx + (qy - s * qx) ** 2, (mm == nx // 2) or (nn == ny // 2)

    s0, K0 = strain(n)
    s1, K1 = strain(n + 1)
    half = [[phi[j][i] - dt * (dy_(psi, i, j, s0) * dx_(phi, i, j) - dx_(psi, i, j) * dy_(phi, i, j, s0))
             for i in range(nx)] for j in range(ny)]
    wstar = [[omega[j][i] - dt * (dy_(psi, i, j, s0) * dx_(omega, i, j) - dx_(psi, i, j) * dy_(omega, i, j, s0))
              for i in range(nx)] for j in range(ny)]
    cube = [[(phi[j][i] * phi[j][i]) * phi[j][i] for i in range(nx)] for j in range(ny)]
    P, C = dft(half, -1), dft(cube, -1)
    for nn in range(ny):
        for mm in range(nx):
            kk, nyq = k2(mm, nn, s0)
            if nyq:
                P[nn][mm] = 0
                continue
            c4 = 0.5 * dt * p.kappa * p.M * kk * kk
            P[nn][mm] = ((1 + dt * p.a * p.M * kk - c4) * P[nn][mm] - dt * p.b * p.M * kk * C[nn][mm]) / (1 + c4)
    new = [[v.real for v in row] for row in dft(P, +1)]
    if K1 != K0 and remap:
        sh = (K1 - K0) * r
        new = [[new[j][(i - j * sh) % nx] for i in range(nx)] for j in range(ny)]
        wstar = [[wstar[j][(i - j * sh) % nx] for i in range(nx)] for j in range(ny)]
    lap = lambda f, i, j, s: ((1 + s * s) * (at(f, i + 1, j) - 2 * at(f, i, j) + at(f, i - 1, j)) / h ** 2
                              - 2 * s * (at(f, i + 1, j + 1) - at(f, i + 1, j - 1) - at(f, i - 1, j + 1)
                                         + at(f, i - 1, j - 1)) / (4 * h * h)
                              + (at(f, i, j + 1) - 2 * at(f, i, j) + at(f, i, j - 1)) / h ** 2)
    mu = [[-p.a * new[j][i] + p.b * (new[j][i] * new[j][i]) * new[j][i] - p.kappa * lap(new, i, j, s1)
           for i in range(nx)] for j in range(ny)]
    F = [[dx_(new, i, j) * dy_(mu, i, j, s1) - dy_(new, i, j, s1) * dx_(mu, i, j)
          for i in range(nx)] for j in range(ny)]
    if p.rho > 0:
        nu = p.eta / p.rho
        W, G = dft(wstar, -1), dft([[-v / p.rho for v in row] for row in F], -1)
        Psi = [[0j] * nx for _ in range(ny)]
        for nn in range(ny):
            for mm in range(nx):
                kk, nyq = k2(mm, nn, s1)
                if nyq or kk == 0:
                    W[nn][mm] = 0
                    continue
                W[nn][mm] = ((1 - 0.5 * dt * nu * kk) * W[nn][mm] + dt * G[nn][mm]) / (1 + 0.5 * dt * nu * kk)
                Psi[nn][mm] = W[nn][mm] / kk
        return (np.array(new), np.array([[v.real for v in r_] for r_ in dft(Psi, +1)]),
                np.array([[v.real for v in r_] for r_ in dft(W, +1)]))
    G = dft([[-v / p.eta for v in row] for row in F], -1)
    for nn in range(ny):
        for mm in range(nx):
            kk, nyq = k2(mm, nn, s1)
            G[nn][mm] = 0 if (nyq or kk == 0) else G[nn][mm] / (kk * kk)
    return np.array(new), np.array([[v.real for v in r_] for r_ in dft(G, +1)]), np.zeros((ny, nx))


@pytest.mark.parametrize("rho", [0.0, 0.8])
@pytest.mark.parametrize("shape,gdot,n0", [((8, 8), 0.13, 3), ((8, 4), 0.4, 2), ((8, 8), 0.0, 0),
                                           ((8, 8), 0.5, 0)])
def test_step_matches_loop_restatement(rho, shape, gdot, n0):
    nx, ny = shape
    p = oracle.Params(a=0.9, b=1.2, kappa=0.8, M=1.1, eta=0.7, rho=rho, gdot=gdot, dt=0.2, dx=1.1)
    phi = inputs.quench_noise(nx, ny, 11, 0.6)
    psi = inputs.quench_noise(nx, ny, 12, 0.3)
    omega = inputs.quench_noise(nx, ny, 13, 0.3) if rho > 0 else np.zeros((ny, nx))
    got = scheme.step(phi, psi, omega, n0, p)
    want = loop_step(phi.tolist(), psi.tolist(), omega.tolist(), n0, p)
    for g, w in zip(got, want):
        assert np.allclose(g, w, atol=1e-12 * max(1.0, np.abs(w).max()))


# ----------------------------------------------------------------- invariants

@pytest.mark.parametrize("rho", [0.0, 1.0])
def test_mean_of_phi_is_conserved(rho):
    p = oracle.Params(rho=rho, gdot=0.01, dt=0.005)
    phi0 = inputs.quench_noise(64, 64, 0)
    m0 = scheme.mean_phi(phi0)
    phi, psi, om = phi0, np.zeros_like(phi0), np.zeros_like(phi0)
    for n in range(200):
        phi, psi, om = scheme.step(phi, psi, om, n, p)
    assert abs(scheme.mean_phi(phi) - m0) < 1e-15


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_phi_sign_symmetry_is_bit_exact(rho):
    """Model H is invariant under phi -> -phi (mu is odd, F is even in phi)."""
    p = oracle.Params(rho=rho, gdot=0.03, dt=0.01)
    phi, psi, om = inputs.quench_state(32, 32, 5, 0.3)
    a = (phi, psi, om)
    b = (-phi, psi, om)
    for n in range(40):
        a = scheme.step(*a, n, p)
        b = scheme.step(*b, n, p)
    assert np.array_equal(a[0], -b[0])
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_remap_is_the_stated_permutation():
    nx, ny = 8, 4
    idx = np.arange(nx * ny, dtype=float).reshape(ny, nx)
    out = scheme.remap_rows(idx, nx // ny)
    for j in range(ny):
        for i in range(nx):
            assert out[j, i] == idx[j, (i - j * 2) % nx]
    assert np.array_equal(np.sort(out.ravel()), np.sort(idx.ravel()))


@pytest.mark.parametrize("shape", [(32, 32), (64, 32)])
def test_frozen_mode_keeps_lab_wavevector_through_wraps(shape):
    """With no dynamics (M = 0, b = 0, tiny amplitude) the co-sheared field is frozen
    except for the remap, and its laboratory wavevector (q_x, q_y - s q_x) must equal
    (k_x, k_y - gdot t k_x) at every step, across several wraps (Sections III and V)."""
    nx, ny = shape
    r = nx // ny
    m, n = 2, 1
    gd = 2.0 ** -5                      # gdot*dt: a wrap every 16*r steps
    p = oracle.Params(a=1.0, b=0.0, kappa=1.0, M=0.0, rho=0.0, gdot=1.0, dt=gd)
    phi = inputs.cosine_mode(nx, ny, m, n, amp=1e-9)
    zero = np.zeros_like(phi)
    kx = 2 * math.pi * m / nx
    ky0 = 2 * math.pi * n / ny
    for step_i in range(80 * r):
        phi, psi, _ = scheme.step(phi, zero, zero, step_i, p)
        F = np.fft.fft2(phi)
        nn, mm = np.unravel_index(np.argmax(np.abs(F[:, : nx // 2])), F[:, : nx // 2].shape)
        assert mm == m
        qy = 2 * math.pi * (nn if nn < ny // 2 else nn - ny) / ny
        s, K = scheme.strain(step_i + 1, 1.0, gd, nx, ny)
        t = gd * (step_i + 1)
        assert math.isclose(qy - s * kx, ky0 - t * kx, abs_tol=1e-12)
        assert math.isclose(np.abs(F).max() * 2 / (nx * ny), 1e-9, rel_tol=1e-9)
    assert K >= 2


def test_no_remap_mode_leaves_fields_untouched_at_wrap():
    nx = ny = 16
    p = oracle.Params(b=0.0, M=0.0, rho=0.0, gdot=1.0, dt=0.25)
    phi = inputs.cosine_mode(nx, ny, 1, 1, amp=1e-9)
    zero = np.zeros_like(phi)
    a = scheme.step(phi, zero, zero, 1, p, remap=scheme.REMAP_NONE)[0]   # wraps at n = 2
    b = scheme.step(phi, zero, zero, 1, p, remap=scheme.REMAP_SHIFT)[0]
    assert np.allclose(a, phi, atol=1e-20)
    assert np.allclose(b, scheme.remap_rows(phi, 1), atol=1e-20)


# --------------------------------------------------------- grid refinement

def test_second_order_self_convergence():
    """Smooth state, fixed physical box and time, dt ~ h^2: the error against the
    finest grid falls by ~ (1 - 1/16)/(1/4 - 1/16) = 5 from N=16 to N=32."""
    L, T = 2 * math.pi, 0.1
    base = dict(a=1.0, b=1.0, kappa=0.05, M=0.2, eta=0.5, rho=1.0, gdot=0.2)
    sols = {}
    for N in (16, 32, 64):
        dx = L / N
        dt = 0.02 * (16 / N) ** 2
        p = oracle.Params(dx=dx, dt=dt, **base)
        phi = inputs.smooth_blobs(N, N, dx, seed=3, nmodes=2, amp=0.6)
        psi = 0.3 * inputs.smooth_blobs(N, N, dx, seed=4, nmodes=2, amp=1.0)
        omega = np.zeros_like(phi)
        # start with a consistent (omega, psi) pair: omega = -lap psi, spectrally
        QX, QY, _ = scheme.wavenumbers(N, N, dx)
        omega = np.real(np.fft.ifft2((QX ** 2 + QY ** 2) * np.fft.fft2(psi)))
        steps = int(round(T / dt))
        phi, psi, omega = scheme.run(phi, psi, omega, steps, p)
        sols[N] = phi
    e16 = np.abs(sols[16] - sols[64][::4, ::4]).max()
    e32 = np.abs(sols[32] - sols[64][::2, ::2]).max()
    assert 3.5 < e16 / e32 < 6.5, (e16, e32)


# ----------------------------------------------------------- diagnostics

@pytest.mark.parametrize("s", [0.0, 0.2, -0.35])
def test_structure_factor_of_single_mode(s):
    nx, ny, dx = 32, 16, 1.5
    A = 0.7
    m, n = 3, 1
    phi = inputs.cosine_mode(nx, ny, m, n, amp=A, dx=dx)
    S0, S1, Sm1, L1, Ls = scheme.structure_factor_moments(phi, s, dx)
    qx, qy = 2 * math.pi * m / (nx * dx), 2 * math.pi * n / (ny * dx)
    k = math.hypot(qx, qy - s * qx)
    assert math.isclose(S0, A * A / 2, rel_tol=1e-12)        # Parseval: <phi^2> = A^2/2
    assert math.isclose(L1, 2 * math.pi / k, rel_tol=1e-12)
    assert math.isclose(Ls, 1 / k, rel_tol=1e-12)
    bins = scheme.structure_factor_binned(phi, s, 16, dx)
    dk = 2 * math.pi / (ny * dx)
    assert math.isclose(bins[int(k // dk)], A * A / 2, rel_tol=1e-12)
    assert math.isclose(bins.sum(), A * A / 2, rel_tol=1e-12)


def test_mean_phi_is_correctly_rounded():
    vals = np.array([1e16, 1.0, -1e16, 1.0])
    assert scheme.mean_phi(vals.reshape(2, 2)) == 0.5


@pytest.mark.parametrize("s", [0.0, 0.37, -0.5])
def test_gradient_tensor_of_modes_is_the_closed_form(s):
    """Eq. L_matrix by Parseval: for orthogonal plane waves a_i cos(theta_i) the
    tensor is sum a_i^2/2 q_i q_i^T / (c^2 + sum a_i^2/2), with q the laboratory
    wavevector (q_x, q_y - s q_x) of each co-sheared grid mode and c the mean."""
    nx, ny, dx = 32, 16, 0.8
    modes = [(3, 1, 0.7, 0.3), (-2, 3, 0.4, 1.1)]          # (m, n, amplitude, phase)
    c = 0.25
    phi = c + sum(inputs.cosine_mode(nx, ny, m, n, amp=a, dx=dx, phase=ph) for m, n, a, ph in modes)
    G = scheme.gradient_tensor(phi, s, dx)
    num = np.zeros((2, 2))
    den = c * c
    for m, n, a, _ in modes:
        q = np.array([2 * math.pi * m / (nx * dx), 2 * math.pi * n / (ny * dx) - s * 2 * math.pi * m / (nx * dx)])
        num += a * a / 2 * np.outer(q, q)
        den += a * a / 2
    want = num / den
    assert np.allclose([G[0], G[1], G[2]], [want[0, 0], want[0, 1], want[1, 1]], rtol=1e-12, atol=1e-14)


def test_gradient_tensor_matches_analytic_lab_derivatives():
    """A smooth lab-frame field f(x, y) sampled on the co-sheared grid at strain s
    (lab x = x' + s y'): the tensor is the mean of grad f grad f^T over the box
    divided by the mean of f^2, with the exact derivatives of f."""
    nx, ny, dx, s = 48, 24, 0.5, 0.375
    Lx, Ly = nx * dx, ny * dx
    Xp, Yp = inputs.grid_coords(nx, ny, dx)
    # f = cos(a x + b y) + 0.5 sin(c x + d y) with (a, b), (c, d) lab wavevectors whose
    # co-sheared components (a, b + s a) are grid modes
    a, b = 2 * math.pi * 2 / Lx, 2 * math.pi * 1 / Ly - s * 2 * math.pi * 2 / Lx
    c, d = 2 * math.pi * -1 / Lx, 2 * math.pi * 3 / Ly - s * 2 * math.pi * -1 / Lx
    X, Y = Xp + s * Yp, Yp
    f = np.cos(a * X + b * Y) + 0.5 * np.sin(c * X + d * Y)
    fx = -a * np.sin(a * X + b * Y) + 0.5 * c * np.cos(c * X + d * Y)
    fy = -b * np.sin(a * X + b * Y) + 0.5 * d * np.cos(c * X + d * Y)
    den = np.mean(f * f)
    want = (np.mean(fx * fx) / den, np.mean(fx * fy) / den, np.mean(fy * fy) / den)
    assert np.allclose(scheme.gradient_tensor(f, s, dx), want, rtol=1e-12, atol=1e-13)


def test_principal_lengths_are_reciprocal_eigenvalues():
    G = (2.0, 0.5, 1.0)
    ev = np.linalg.eigvalsh(np.array([[2.0, 0.5], [0.5, 1.0]]))
    Lpar, Lperp = scheme.principal_lengths(G, 0.5)
    assert math.isclose(Lpar, 1 / (0.5 * ev[0]), rel_tol=1e-14)
    assert math.isclose(Lperp, 1 / (0.5 * ev[1]), rel_tol=1e-14)
    assert scheme.principal_lengths((1.0, 0.0, 0.0), 1.0) == (float("inf"), 1.0)
