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


def gaussian_random_field_torch(nx: int, ny: int, ell: float, std: float, seed: int, device="cuda"):
    """The recipe of :func:`gaussian_random_field` with the FFTs on a torch device.

    The white noise is the same numpy PCG64 stream, so the field equals the
    numpy one up to FFT rounding.  Returns (field, d/dx, d/dy) as float64 tensors
    for a spacing of 1 (divide the derivatives by dx).
    """
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    w = torch.from_numpy(rng.standard_normal((ny, nx))).to(device)
    W = torch.fft.rfft2(w)
    kx = torch.from_numpy(2.0 * np.pi * np.fft.rfftfreq(nx)).to(device)[None, :]
    ky = torch.from_numpy(2.0 * np.pi * np.fft.fftfreq(ny)).to(device)[:, None]
    W = W * torch.exp(-(kx * kx + ky * ky) * (ell * ell) / 4.0)
    W[0, 0] = 0.0
    f = torch.fft.irfft2(W, s=(ny, nx))
    scale = std / float(torch.std(f, unbiased=False))
    W = W * scale
    f = f * scale
    kxn = kx.clone()
    if nx % 2 == 0:
        kxn[..., -1] = 0.0
    kyn = ky.clone()
    if ny % 2 == 0:
        kyn[ny // 2, ...] = 0.0
    fx = torch.fft.irfft2(W * (1j * kxn), s=(ny, nx))
    fy = torch.fft.irfft2(W * (1j * kyn), s=(ny, nx))
    return f, fx, fy


def batch_lattice_inputs_torch(spec, dx: float, std: float = 1e-3, device="cuda"):
    """U0, dU0/dx, dU0/dy ([5, ny, nx] float64 tensors) of one batch lattice: GRF
    velocities with correlation length spec.ell (seeds spec.seed, spec.seed + 7919),
    windowed by sin(pi x/Lx) sin(pi y/Ly) for Dirichlet lattices, u0 = 0."""
    import torch
    nx, ny = spec.nx, spec.ny
    out = [torch.zeros((5, ny, nx), dtype=torch.float64, device=device) for _ in range(3)]
    for comp, seed in enumerate((spec.seed, spec.seed + 7919)):
        f, fx, fy = gaussian_random_field_torch(nx, ny, spec.ell, std, seed, device)
        fx, fy = fx / dx, fy / dx
        if spec.dirichlet:
            xs = (torch.arange(nx, dtype=torch.float64, device=device) + 0.5) / nx
            ys = (torch.arange(ny, dtype=torch.float64, device=device) + 0.5) / ny
            wx, wy = torch.sin(np.pi * xs)[None, :], torch.sin(np.pi * ys)[:, None]
            dwx = (np.pi / (nx * dx)) * torch.cos(np.pi * xs)[None, :]
            dwy = (np.pi / (ny * dx)) * torch.cos(np.pi * ys)[:, None]
            win = wy * wx
            fx, fy = fx * win + f * wy * dwx, fy * win + f * dwy * wx
            f = f * win
        out[0][comp], out[1][comp], out[2][comp] = f, fx, fy
    return out
