"""Isotropised 1-D spectra of a 2-D periodic field (Sec. 5, Fig. 5): the energy of
the Fourier modes in unit-width shells of k_perp = |(kx, ky)|, and the slope of a
power-law fit over a range of k_perp.  Analysis of outputs, not part of the step."""
import numpy as np


def shell_spectrum(fields):
    """fields: sequence of [ny, nx] arrays (components); returns (k, E(k)) with
    E(k) = sum over |k'| in [k - 1/2, k + 1/2) of sum_c |f_c(k')|^2 / N^2."""
    ny, nx = fields[0].shape
    kx = np.fft.fftfreq(nx) * nx
    ky = np.fft.fftfreq(ny) * ny
    kk = np.sqrt(kx[None, :] ** 2 + ky[:, None] ** 2)
    shell = np.rint(kk).astype(np.int64)
    e = np.zeros_like(kk)
    for f in fields:
        F = np.fft.fft2(f - f.mean()) / (nx * ny)
        e += np.abs(F) ** 2
    kmax = min(nx, ny) // 2
    E = np.bincount(shell.ravel(), weights=e.ravel(), minlength=kmax + 1)[:kmax + 1]
    return np.arange(kmax + 1), E


def slope(k, E, kmin, kmax):
    """least-squares slope of log E against log k over kmin <= k <= kmax"""
    sel = (k >= kmin) & (k <= kmax) & (E > 0)
    return float(np.polyfit(np.log(k[sel]), np.log(E[sel]), 1)[0])
