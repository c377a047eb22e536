"""Error model of FP32 psi, shared by the GPU parity tests and pinned on the
CPU in test_fp32_model.py.  Test infrastructure only."""
import numpy as np

import oracle

EPS32 = 2.0 ** -24      # unit roundoff of IEEE binary32
PSI32_MODEL_MAX = 8.0   # allowed RMS of |error| / envelope for FP32 psi (measured 1.7-2.8)


def psi32_model_ratio(got, want, s, dx, rho):
    """FP32 psi against the FP64 oracle through an error model of FP32 arithmetic.

    psi comes from a division by L(k) = k^2 (inertial: psi_hat = omega_hat / k^2)
    or k^4 (Stokes: psi_hat = g_hat / (eta k^4)), k from the sheared wavevector at
    s.  Its right-hand side (omega, or the body-force curl g) is formed and
    transformed in FP32, so every mode of it carries rounding of about eps times
    its RMS over modes -- but the spectrum of the finite-difference curl of
    Appendix B vanishes like k^2 at small k, so at the lowest modes that rounding
    is a large relative error, and 1/L(k) makes those modes dominate psi.  The
    error of each mode is therefore modelled as
        envelope(k) = eps * (rms(L psi_hat_ref) / L(k) + rms(psi_hat_ref)),
    the second term being psi's own FP32 storage and inverse transform.  Returns
    the RMS over the solved modes (k != 0, off the Nyquist lines) of
    |psi_hat_gpu - psi_hat_ref| / envelope.  A wrong term, sign or index gives
    errors of order |psi_hat| and ratios of 1e3 and more."""
    ny, nx = want.shape
    QX, QY, nyq = oracle.wavenumbers(nx, ny, dx)
    k2 = oracle.sheared_k2(QX, QY, s)
    L = k2 * k2 if rho == 0 else k2
    solved = (k2 > 0) & ~nyq
    R = np.fft.fft2(want)
    E = np.fft.fft2(got) - R
    rhs_rms = np.sqrt(np.mean(np.abs(L * R)[solved] ** 2))
    psi_rms = np.sqrt(np.mean(np.abs(R) ** 2))
    env = EPS32 * (rhs_rms / np.where(solved, L, 1.0) + psi_rms)
    return float(np.sqrt(np.mean((np.abs(E) / env)[solved] ** 2)))
