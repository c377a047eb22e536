"""FP64 CPU oracle of the sheared model-H time step (test infrastructure only).

THIS PACKAGE IS TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py`` (its ``cpu_baseline`` leg and ``--impl reference``) may import or
run it.  The CUDA library never calls into it and it never calls the CUDA library.

It restates, slowly and in the paper's order, the mixed finite-difference /
pseudo-spectral scheme of Fielding, "The need for inertia in nonequilibrium
steady states of sheared binary fluids" (arXiv:0710.5912), Appendix B, on the
co-sheared frame of Section V / Appendix A.  All arithmetic is float64; numpy's
FFT is used as a library primitive (forward sign e^{-i}, inverse e^{+i}/(NxNy)).

Model (Section II, Eqs. vorticity/stream/streamVort/phi1/mu1, in the generalised
form mu = -a phi + b phi^3 - kappa lap phi; the paper's case is a = b = 1,
kappa = M = l^2 in its units, Section IV):

    d_t phi + J(psi, phi) = M lap_c mu,
    rho (d_t omega + J(psi, omega)) = eta lap_c omega - F,   F = curl(phi grad mu).z
    omega = -lap_c psi;   Stokes (rho = 0):  0 = -eta lap_c^2 psi - F.

Co-sheared gradient (Eq. coshearedNabluFinal): grad_c = (d_x, d_y - s(t) d_x),
with the sawtooth strain s(t) of Section V.

Readings of points the paper leaves open (each used below, named by tag):

  [s-timing]  stage 1 (advection + phi update) uses s^n; stages 2-3 (mu, F,
              omega, psi), whose results carry the label n+1, use s^{n+1}.
  [remap]     at a wrap (s jumps by -Lx/Ly) the stored fields are relabelled so
              the laboratory field stays continuous: row j shifts by j*Nx/Ny
              cells (mode "shift", default); mode "none" leaves them untouched.
  [cubic]     f = (phi^n)^3, the pre-advection field.
  [nyquist]   every mode on the lines m = -Nx/2 or n = -Ny/2 of phi^{n+1},
              omega^{n+1}, psi^{n+1} is set to zero (the sheared multipliers
              break Hermitian symmetry there when s != 0).
  [k0]        the k = 0 mode of phi passes unchanged; psi(k=0) = omega(k=0) = 0.
  [stokes]    Stokes source: psi_hat = -F_hat / (eta k^4).
  [omega*]    the Crank-Nicolson omega^n is the post-advection omega*.
  [wavenum]   spectral wavenumbers are the continuous q = 2 pi m / L.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

REMAP_SHIFT = 0
REMAP_NONE = 1


@dataclass(frozen=True)
class Params:
    """Run parameters in grid units (set_params(a, b, kappa, M, eta, rho, gdot, dt))."""
    a: float = 1.0
    b: float = 1.0
    kappa: float = 1.0
    M: float = 1.0
    eta: float = 1.0
    rho: float = 1.0      # rho == 0 selects the zero-Reynolds-number (Stokes) algorithm
    gdot: float = 0.0
    dt: float = 0.005
    dx: float = 1.0


# ---------------------------------------------------------------------------
# Strain sawtooth (Section V, paragraph on the shift s -> s - Lx/Ly)
# ---------------------------------------------------------------------------

def strain(n: int, gdot: float, dt: float, nx: int, ny: int):
    """s(t^n) and the wrap count K_n.

    The accumulated strain gdot*t^n is computed from the integer step n, never
    accumulated.  Whenever it reaches Lx/(2Ly) the strain is shifted down by
    Lx/Ly, so s lies in [-Lx/(2Ly), Lx/(2Ly)) (the wrap is inclusive).
    Lx/Ly = Nx/Ny exactly because dx = dy.
    """
    r = nx // ny
    total = (gdot * dt) * float(n)
    K = math.floor(total / r + 0.5)
    return total - K * r, K


# ---------------------------------------------------------------------------
# Finite-difference stencils (Appendix B, Eq. p1y and the mu discretisation)
# ---------------------------------------------------------------------------

def shifted(f: np.ndarray, di: int, dj: int) -> np.ndarray:
    """Periodic neighbour: result[j, i] = f[(j + dj) mod Ny, (i + di) mod Nx]."""
    return np.roll(f, (-dj, -di), axis=(0, 1))


def d_x(f, h):
    """Central first difference in x (Eq. p1y, first line)."""
    return (shifted(f, 1, 0) - shifted(f, -1, 0)) / (2.0 * h)


def d_y_sheared(f, s, h):
    """Sheared y-derivative (Eq. p1y): the vertical central difference blended,
    with weight s/2, with the difference along the diagonal pair two cells
    across; it approximates d_y - s d_x.  The branch follows the sign of s
    (s = 0 takes the first branch, where it reduces to the central difference).
    """
    vert = shifted(f, 0, 1) - shifted(f, 0, -1)
    if s >= 0.0:
        diag = shifted(f, -2, 1) - shifted(f, 2, -1)
        return ((1.0 - s / 2.0) * vert + (s / 2.0) * diag) / (2.0 * h)
    diag = shifted(f, 2, 1) - shifted(f, -2, -1)
    return ((1.0 + s / 2.0) * vert - (s / 2.0) * diag) / (2.0 * h)


def lap_sheared(f, s, h):
    """(1 + s^2) d_xx - 2 s d_xy + d_yy with 3-point second differences and the
    4-point cross difference (Appendix B, item 2, discretisation of mu)."""
    dxx = (shifted(f, 1, 0) - 2.0 * f + shifted(f, -1, 0)) / (h * h)
    dyy = (shifted(f, 0, 1) - 2.0 * f + shifted(f, 0, -1)) / (h * h)
    dxy = (shifted(f, 1, 1) - shifted(f, 1, -1) - shifted(f, -1, 1)
           + shifted(f, -1, -1)) / (4.0 * h * h)
    return (1.0 + s * s) * dxx - 2.0 * s * dxy + dyy


def bracket(A, B, s, h):
    """Advective bracket d_y A d_x B - d_x A d_y B with the Eq. p1y stencils
    (Eq. advective: v = curl(psi z) = (d_y psi, -d_x psi))."""
    return d_y_sheared(A, s, h) * d_x(B, h) - d_x(A, h) * d_y_sheared(B, s, h)


def cube(phi):
    """phi^3 as the product (phi*phi)*phi, which is exactly odd in IEEE arithmetic
    (a library power routine need not be), so the phi -> -phi symmetry of the
    model holds bit for bit."""
    return (phi * phi) * phi


def chemical_potential(phi, s, p: Params):
    """mu = -a phi + b phi^3 - kappa * lap_c phi (Eq. mu1 with the sheared
    Laplacian of the Appendix B mu formula)."""
    return -p.a * phi + p.b * cube(phi) - p.kappa * lap_sheared(phi, s, p.dx)


def body_force_curl(phi, mu, s, h):
    """F = d_x phi d_y mu - d_y phi d_x mu = [curl(phi grad mu)].z (Eq. G without
    its -1/rho factor); first derivatives as in Eq. p1y."""
    return d_x(phi, h) * d_y_sheared(mu, s, h) - d_y_sheared(phi, s, h) * d_x(mu, h)


# ---------------------------------------------------------------------------
# Spectral helpers (Appendix B, the D2 / D4 / C / E operators as complex
# multipliers: grad_c^2 acting on exp(i q.x) gives -k^2 with
# k^2 = q_x^2 + (q_y - s q_x)^2; the 4x4 real blocks of the paper are the same
# operator written on (rr, ir, ri, ii) components)
# ---------------------------------------------------------------------------

def wavenumbers(nx, ny, dx):
    """Signed q_x[j, i], q_y[j, i] in numpy FFT order, plus a Nyquist-line mask."""
    m = np.fft.fftfreq(nx, d=1.0 / nx)          # 0..nx/2-1, -nx/2..-1
    n = np.fft.fftfreq(ny, d=1.0 / ny)
    qx = 2.0 * np.pi * m / (nx * dx)
    qy = 2.0 * np.pi * n / (ny * dx)
    QX, QY = np.meshgrid(qx, qy)
    MM, NN = np.meshgrid(m, n)
    nyquist = (MM == -nx // 2) | (NN == -ny // 2)
    return QX, QY, nyquist


def sheared_k2(QX, QY, s):
    """|q_c|^2 with q_c = (q_x, q_y - s q_x), the symbol of -lap_c."""
    return QX * QX + (QY - s * QX) ** 2


def fft2(f):
    return np.fft.fft2(f)


def ifft2_real(F):
    return np.real(np.fft.ifft2(F))


def remap_rows(f, shift_per_row: int):
    """Exact relabelling at a strain wrap: new[j, i] = old[(i - j*shift) mod Nx, j].

    A shift of s by -Lx/Ly moves the laboratory point under a fixed co-sheared
    cell by -(Lx/Ly) y; re-indexing row j by j*Nx/Ny cells keeps the laboratory
    field unchanged (a pure permutation of the stored values).
    """
    out = np.empty_like(f)
    nx = f.shape[1]
    for j in range(f.shape[0]):
        out[j] = np.roll(f[j], (j * shift_per_row) % nx)
    return out


# ---------------------------------------------------------------------------
# One time step (Appendix B, items 1-3; "Algorithm at zero Reynolds number")
# ---------------------------------------------------------------------------

def advect(field, psi, s, p: Params):
    """Explicit Euler advection by the stream function (Eq. advective):
    field^{n+1/2} = field^n - dt * (d_y psi d_x field - d_x psi d_y field).
    Item 1 applies it to phi; item 2 applies it to omega in the same pass."""
    return field - p.dt * bracket(psi, field, s, p.dx)


def cahn_hilliard_spectral(phi_half, f, s, p: Params, QX, QY, nyquist):
    """Item 1, diffusive part: d_t phi = M lap_c(-a phi + b f - kappa lap_c phi)
    in Fourier space, explicit Euler on the lap_c terms and Crank-Nicolson on
    lap_c^2, which rearranges per mode to

        (1 + dt kappa M k^4 / 2) phi' = (1 + dt a M k^2 - dt kappa M k^4 / 2) phi_half
                                        - dt b M k^2 f_hat.
    """
    dt = p.dt
    k2 = sheared_k2(QX, QY, s)
    k4 = k2 * k2
    Phi = fft2(phi_half)
    Fc = fft2(f)
    num = (1.0 + dt * p.a * p.M * k2 - 0.5 * dt * p.kappa * p.M * k4) * Phi \
        - dt * p.b * p.M * k2 * Fc
    Phi_new = num / (1.0 + 0.5 * dt * p.kappa * p.M * k4)
    Phi_new[nyquist] = 0.0                                # [nyquist]
    return ifft2_real(Phi_new)


def vorticity_poisson_solve(omega_star, F, s, p: Params, QX, QY, nyquist):
    """Items 2-3 (rho > 0): Crank-Nicolson on d_t omega = nu lap_c omega + g,
    nu = eta / rho, g = -F / rho (Eqs. vortNum, G), then psi from
    omega = -lap_c psi (Eq. streamVort).  Returns (psi, omega)."""
    dt = p.dt
    k2 = sheared_k2(QX, QY, s)
    k0 = (k2 == 0.0)
    nu = p.eta / p.rho
    W = fft2(omega_star)                                  # [omega*]
    G = fft2(-F / p.rho)
    W_new = ((1.0 - 0.5 * dt * nu * k2) * W + dt * G) / (1.0 + 0.5 * dt * nu * k2)
    W_new[k0] = 0.0                                       # [k0]
    W_new[nyquist] = 0.0                                  # [nyquist]
    Psi = W_new / np.where(k0, 1.0, k2)
    Psi[k0] = 0.0
    return ifft2_real(Psi), ifft2_real(W_new)


def stokes_solve(F, s, p: Params, QX, QY, nyquist):
    """Zero-Reynolds-number algorithm: 0 = -eta lap_c^2 psi - F, i.e.
    psi_hat = -F_hat / (eta k^4) for k != 0 [stokes]; psi(k=0) = 0."""
    k2 = sheared_k2(QX, QY, s)
    k0 = (k2 == 0.0)
    safe = np.where(k0, 1.0, k2)
    Psi = fft2(-F / p.eta) / (safe * safe)
    Psi[k0] = 0.0                                         # [k0]
    Psi[nyquist] = 0.0                                    # [nyquist]
    return ifft2_real(Psi)


def flow_substep(phi_new, omega_star, s, p: Params, QX, QY, nyquist):
    """Items 2-3, or the zero-Reynolds-number algorithm when rho = 0, at phi^{n+1}
    and s = s^{n+1}: mu, the body-force curl F, then the spectral solve.
    Returns (psi^{n+1}, omega^{n+1}); omega is identically zero for Stokes."""
    mu = chemical_potential(phi_new, s, p)
    F = body_force_curl(phi_new, mu, s, p.dx)
    if p.rho > 0.0:
        return vorticity_poisson_solve(omega_star, F, s, p, QX, QY, nyquist)
    return stokes_solve(F, s, p, QX, QY, nyquist), np.zeros_like(phi_new)


def step(phi, psi, omega, n: int, p: Params, remap: int = REMAP_SHIFT):
    """Advance (phi^n, psi^n, omega^n) at step index n to step n+1."""
    ny, nx = phi.shape
    QX, QY, nyq = wavenumbers(nx, ny, p.dx)
    s_n, K_n = strain(n, p.gdot, p.dt, nx, ny)            # [s-timing]
    s_1, K_1 = strain(n + 1, p.gdot, p.dt, nx, ny)
    phi_half = advect(phi, psi, s_n, p)                   # item 1, advective part
    f = cube(phi)                                         # [cubic]
    phi_new = cahn_hilliard_spectral(phi_half, f, s_n, p, QX, QY, nyq)
    omega_star = advect(omega, psi, s_n, p) if p.rho > 0.0 else omega
    if K_1 != K_n and remap == REMAP_SHIFT:               # [remap]
        shift = (K_1 - K_n) * (nx // ny)
        phi_new = remap_rows(phi_new, shift)
        omega_star = remap_rows(omega_star, shift)
    psi_new, omega_new = flow_substep(phi_new, omega_star, s_1, p, QX, QY, nyq)
    return phi_new, psi_new, omega_new


def run(phi, psi, omega, nsteps: int, p: Params, n0: int = 0,
        remap: int = REMAP_SHIFT, callback=None):
    """nsteps successive steps starting at step index n0."""
    for k in range(nsteps):
        phi, psi, omega = step(phi, psi, omega, n0 + k, p, remap)
        if callback is not None:
            callback(n0 + k + 1, phi, psi, omega)
    return phi, psi, omega


# ---------------------------------------------------------------------------
# Diagnostics (Section VI, Eq. L_structure; mass of phi)
# ---------------------------------------------------------------------------

def mean_phi(phi) -> float:
    """Correctly rounded mean of phi (math.fsum is exact before the division)."""
    return math.fsum(phi.ravel().tolist()) / phi.size


def structure_factor_moments(phi, s: float, dx: float = 1.0):
    """S(q) = |phi_hat(q)|^2 / (Nx Ny)^2 on the laboratory wavevectors
    q_c = (q_x, q_y - s q_x); k = 0 and the Nyquist lines are excluded.

    Returns (sum S, sum k S, sum S / k, L_1 = 2 pi sum S / sum k S,
    L_s = sum S/k / sum S), L_s being Eq. L_structure written as a sum.
    """
    ny, nx = phi.shape
    QX, QY, nyq = wavenumbers(nx, ny, dx)
    k = np.sqrt(sheared_k2(QX, QY, s))
    S = np.abs(fft2(phi)) ** 2 / float(nx * ny) ** 2
    keep = (~nyq) & (k > 0.0)
    S0 = math.fsum(S[keep].tolist())
    S1 = math.fsum((k[keep] * S[keep]).tolist())
    Sm1 = math.fsum((S[keep] / k[keep]).tolist())
    L1 = 2.0 * math.pi * S0 / S1 if S1 > 0 else float("nan")
    Ls = Sm1 / S0 if S0 > 0 else float("nan")
    return S0, S1, Sm1, L1, Ls


def gradient_tensor(phi, s: float, dx: float = 1.0):
    """The anisotropy tensor of Eq. L_matrix without its prefactor l:
    G_ab = int d_a phi d_b phi / int phi^2 with laboratory derivatives
    (d_x, d_y - s d_x) of the trigonometric interpolant, i.e. by Parseval
    G_ab = sum q_ca q_cb |phi_hat|^2 / sum |phi_hat|^2 over the modes off the
    Nyquist lines (k = 0 included in the denominator), q_c = (q_x, q_y - s q_x).
    Returns (G_xx, G_xy, G_yy)."""
    ny, nx = phi.shape
    QX, QY, nyq = wavenumbers(nx, ny, dx)
    KY = QY - s * QX
    P = np.abs(fft2(phi)) ** 2
    P[nyq] = 0.0
    den = math.fsum(P.ravel().tolist())
    gxx = math.fsum((QX * QX * P).ravel().tolist()) / den
    gxy = math.fsum((QX * KY * P).ravel().tolist()) / den
    gyy = math.fsum((KY * KY * P).ravel().tolist()) / den
    return gxx, gxy, gyy


def principal_lengths(G, ell: float):
    """L_par, L_perp of Eq. L_matrix: the reciprocals of the eigenvalues of
    D = ell G (smallest eigenvalue -> the long axis L_par); infinite where an
    eigenvalue is zero."""
    gxx, gxy, gyy = G
    half_tr = 0.5 * (gxx + gyy)
    rad = math.hypot(0.5 * (gxx - gyy), gxy)
    lam_max, lam_min = half_tr + rad, half_tr - rad
    inv = lambda lam: 1.0 / (ell * lam) if lam > 0 else float("inf")
    return inv(lam_min), inv(lam_max)


def structure_factor_binned(phi, s: float, nbins: int, dx: float = 1.0):
    """Radially binned S: bin b sums S over the kept modes (as in
    structure_factor_moments) with b <= k / dk < b + 1, where the bin width is
    the box's fundamental wavenumber dk = 2 pi / (Ny dx); modes beyond the last
    bin are left out."""
    ny, nx = phi.shape
    QX, QY, nyq = wavenumbers(nx, ny, dx)
    k = np.sqrt(sheared_k2(QX, QY, s))
    S = np.abs(fft2(phi)) ** 2 / float(nx * ny) ** 2
    dk = 2.0 * math.pi / (ny * dx)
    out = np.zeros(nbins)
    keep = (~nyq) & (k > 0.0)
    b = np.floor(k / dk).astype(np.int64)
    ok = keep & (b < nbins)
    np.add.at(out, b[ok], S[ok])
    return out
