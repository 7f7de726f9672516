"""Spectral (Fourier) restriction and prolongation between a fine n^3 and a
coarse m^3 periodic grid, m = n / r -- numpy FFT, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2.2 lets the coarse propagator run on a coarser spatial mesh, which
needs transfer operators between the meshes whose order affects the
convergence.  The spectral pair keeps exactly the Fourier modes both grids
represent and drops the others:

  restriction    (R u)(X) = sum_{k in K_m} u_hat(k) exp(2 pi i k.X)   at the coarse points,
  prolongation   (P c)(x) = sum_{k in K_m} c_hat(k) exp(2 pi i k.x)   at the fine points,

with u_hat, c_hat the Fourier coefficients of the fine and the coarse field
(fftn divided by the number of points) and K_m the integer wavevectors with
|k_d| <= m/2 - 1 on every axis.  The coarse grid's Nyquist wavenumber m/2 has
no symmetric partner on the coarse grid and is dropped.  Coarse point I sits
on fine point I r (cell-vertex grids, x_i = i / n).
"""
import numpy as np


def _kept(m):
    """Integer wavenumbers kept by the transfers between any grid and m^3."""
    return np.arange(-(m // 2 - 1), m // 2)


def _index_maps(n, m):
    w = _kept(m)
    return w % n, w % m          # fftn positions of the kept wavenumbers on each grid


def restrict_spectral(u, r):
    """R u: fine [n][n][n] field -> coarse [m][m][m] field, m = n / r."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[0]
    m = n // r
    fi, ci = _index_maps(n, m)
    U = np.fft.fftn(u) / n ** 3
    C = np.zeros((m, m, m), dtype=np.complex128)
    C[np.ix_(ci, ci, ci)] = U[np.ix_(fi, fi, fi)]
    return np.real(np.fft.ifftn(C) * m ** 3)


def prolong_spectral(c, r):
    """P c: coarse [m][m][m] field -> fine [n][n][n] field, n = m r."""
    c = np.asarray(c, dtype=np.float64)
    m = c.shape[0]
    n = m * r
    fi, ci = _index_maps(n, m)
    Cc = np.fft.fftn(c) / m ** 3
    U = np.zeros((n, n, n), dtype=np.complex128)
    U[np.ix_(fi, fi, fi)] = Cc[np.ix_(ci, ci, ci)]
    return np.real(np.fft.ifftn(U) * n ** 3)


def kept_mask(n, m):
    """Boolean [n][n][n] mask (fftn order) of the fine modes the transfers keep."""
    f = np.abs(np.fft.fftfreq(n, d=1.0 / n)) <= m // 2 - 1
    return f[:, None, None] & f[None, :, None] & f[None, None, :]
