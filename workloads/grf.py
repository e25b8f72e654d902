"""Seeded periodic Gaussian random fields (synthetic initial velocities).

Input generation only.  Recipe: white noise from numpy's PCG64 with the given
seed, filtered in Fourier space by exp(-|kappa|^2 ell^2 / 4) (kappa in radians
per cell), so that the power spectrum is exp(-|kappa|^2 ell^2 / 2) and the
covariance is Gaussian, exp(-r^2 / (2 ell^2)), with correlation length ell
cells; then shifted to zero mean and scaled to the requested standard deviation.
Derivatives are spectral (exact for the band-limited periodic field).
"""
from __future__ import annotations

import numpy as np


def _wavenumbers(nx: int, ny: int):
    kx = 2.0 * np.pi * np.fft.rfftfreq(nx)      # rad / cell
    ky = 2.0 * np.pi * np.fft.fftfreq(ny)
    return kx[None, :], ky[:, None]


def gaussian_random_field(nx: int, ny: int, ell: float, std: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((ny, nx))
    W = np.fft.rfft2(w)
    kx, ky = _wavenumbers(nx, ny)
    W *= np.exp(-(kx * kx + ky * ky) * (ell * ell) / 4.0)
    W[0, 0] = 0.0
    f = np.fft.irfft2(W, s=(ny, nx))
    s = float(np.std(f))
    return f * (std / s) if s > 0 else f


def spectral_gradient(f: np.ndarray, dx: float):
    """(d/dx f, d/dy f) of a periodic field sampled with spacing dx."""
    ny, nx = f.shape
    F = np.fft.rfft2(f)
    kx, ky = _wavenumbers(nx, ny)
    # the Nyquist modes carry no derivative information for a real field
    kxn = kx.copy()
    if nx % 2 == 0:
        kxn[..., -1] = 0.0
    kyn = ky.copy()
    if ny % 2 == 0:
        kyn[ny // 2, ...] = 0.0
    dfx = np.fft.irfft2(F * (1j * kxn / dx), s=(ny, nx))
    dfy = np.fft.irfft2(F * (1j * kyn / dx), s=(ny, nx))
    return dfx, dfy
