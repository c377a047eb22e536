"""Seeded synthetic inputs for the sheared model-H step.

This module only *generates* initial states; it contains none of the scheme's
arithmetic, so both the CUDA path (through the C ABI) and the FP64 oracle can
be fed from it without sharing any code of the method itself.

Quench state (Section VII, "initial condition"): each grid value of phi is
drawn from a flat distribution on [-amp, +amp] (the paper uses amp = 0.01);
psi and omega start at zero.  The draw is SplitMix64 (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014): the generator
state starts at ``seed``, is advanced by the golden-gamma constant once per
draw, and the mixed 64-bit output ``z`` becomes ``u = (z >> 11) * 2**-53`` in
[0, 1), then ``phi = amp * (2u - 1)``.  Draws run over the grid in row-major
order (row j = y index outer, column i = x index inner).  Because SplitMix64
is counter based, draw k is a pure function of ``seed + (k + 1) * gamma``,
which is what ``splitmix64`` below evaluates, vectorised.

Single Fourier modes (cosines on the grid) serve the dispersion, tilting and
Poisson checks.
"""
from __future__ import annotations

import numpy as np

GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of SplitMix64 seeded with ``seed``."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int) -> np.ndarray:
    """u = (z >> 11) * 2^-53, exactly representable doubles in [0, 1)."""
    z = splitmix64(seed, count)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def quench_noise(nx: int, ny: int, seed: int, amp: float = 0.01) -> np.ndarray:
    """phi^0 of shape (ny, nx): amp * (2u - 1), row-major draw order."""
    u = uniform01(seed, nx * ny)
    return (amp * (2.0 * u - 1.0)).reshape(ny, nx)


def quench_state(nx: int, ny: int, seed: int, amp: float = 0.01):
    """(phi, psi, omega) for a deep quench: noisy phi, zero flow."""
    phi = quench_noise(nx, ny, seed, amp)
    return phi, np.zeros_like(phi), np.zeros_like(phi)


def grid_coords(nx: int, ny: int, dx: float = 1.0):
    """Cell coordinates x_i = i*dx, y_j = j*dx as (ny, nx) arrays."""
    x = np.arange(nx, dtype=np.float64) * dx
    y = np.arange(ny, dtype=np.float64) * dx
    return np.meshgrid(x, y)  # X[j, i], Y[j, i]


def cosine_mode(nx: int, ny: int, m: int, n: int, amp: float = 1.0,
                dx: float = 1.0, phase: float = 0.0) -> np.ndarray:
    """amp * cos(q_x x + q_y y + phase) with q = (2 pi m / (nx dx), 2 pi n / (ny dx))."""
    X, Y = grid_coords(nx, ny, dx)
    qx = 2.0 * np.pi * m / (nx * dx)
    qy = 2.0 * np.pi * n / (ny * dx)
    return amp * np.cos(qx * X + qy * Y + phase)


def smooth_blobs(nx: int, ny: int, dx: float, seed: int, nmodes: int = 4,
                 amp: float = 0.5) -> np.ndarray:
    """A smooth, band-limited random field (a few low modes) for refinement checks.

    Only modes with |m|, |n| <= nmodes are populated, so the field is resolved
    on every grid of the refinement sequence.
    """
    rng_u = uniform01(seed, 4 * (2 * nmodes + 1) ** 2)
    X, Y = grid_coords(nx, ny, dx)
    Lx, Ly = nx * dx, ny * dx
    out = np.zeros((ny, nx))
    c = 0
    total = 0.0
    for m in range(-nmodes, nmodes + 1):
        for n in range(-nmodes, nmodes + 1):
            a = rng_u[c] - 0.5
            ph = 2.0 * np.pi * rng_u[c + 1]
            c += 4
            if m == 0 and n == 0:
                continue
            total += abs(a)
            out += a * np.cos(2 * np.pi * m * X / Lx + 2 * np.pi * n * Y / Ly + ph)
    # normalised by the sum of |coefficients| (a bound on the maximum), which does
    # not depend on the grid, so every grid samples the same continuous field
    return out * (amp / total)


def coarsened_state(phi_noise: np.ndarray) -> np.ndarray:
    """A domain-like state (phi ~ +-1) built from noise by sign + smoothing.

    Used only as a second timing state (interfaces everywhere): throughput does
    not depend on the data, but this checks that claim on real domain patterns.
    """
    s = np.sign(phi_noise)
    s[s == 0] = 1.0
    k = np.fft.fft2(s)
    ny, nx = s.shape
    m = np.fft.fftfreq(nx)[None, :]
    n = np.fft.fftfreq(ny)[:, None]
    filt = np.exp(-((m ** 2 + n ** 2) * (nx / 8.0) ** 2))
    sm = np.real(np.fft.ifft2(k * filt))
    return np.tanh(4.0 * sm / max(np.abs(sm).max(), 1e-300))
