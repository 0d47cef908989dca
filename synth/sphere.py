"""Sphere geometry and real spherical harmonics used to synthesise smooth fields.

Grid convention (Sec. 2.2, collocated lon/lat grid): nx longitudes
lambda_i = i * dlam, dlam = 2*pi/nx, periodic; ny latitudes
phi_j = -pi/2 + (j + 1/2) * dphi, dphi = pi/ny (rows half a cell from the poles).
"""
from __future__ import annotations

import math

import numpy as np


def grid_coords(nx: int, ny: int):
    """Return (lam[nx], phi[ny], dlam, dphi) for the collocated lon/lat grid."""
    dlam = 2.0 * math.pi / nx
    dphi = math.pi / ny
    lam = np.arange(nx, dtype=np.float64) * dlam
    phi = -0.5 * math.pi + (np.arange(ny, dtype=np.float64) + 0.5) * dphi
    return lam, phi, dlam, dphi


def _assoc_legendre(l: int, m: int, x: np.ndarray) -> np.ndarray:
    """Unnormalised associated Legendre function P_l^m(x), m >= 0, without the
    Condon-Shortley phase, by the standard three-term recurrence in l."""
    if m > l:
        return np.zeros_like(x)
    somx2 = np.sqrt(np.maximum(0.0, 1.0 - x * x))
    pmm = np.ones_like(x)
    fact = 1.0
    for _ in range(m):
        pmm = pmm * fact * somx2
        fact += 2.0
    if l == m:
        return pmm
    pmmp1 = x * (2 * m + 1) * pmm
    if l == m + 1:
        return pmmp1
    pll = pmmp1
    for ll in range(m + 2, l + 1):
        pll = ((2 * ll - 1) * x * pmmp1 - (ll + m - 1) * pmm) / (ll - m)
        pmm, pmmp1 = pmmp1, pll
    return pll


def real_sh(l: int, m: int, lam: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Orthonormal real spherical harmonic Y_lm(lam, phi) evaluated on the
    outer grid (phi rows x lam columns).  m > 0 -> cos(m lam), m < 0 -> sin(|m| lam).

    It is an eigenfunction of the unit-sphere Laplacian with eigenvalue
    -l(l+1); the operator tests rely on that property."""
    am = abs(m)
    norm = math.sqrt((2 * l + 1) / (4.0 * math.pi)
                     * math.factorial(l - am) / math.factorial(l + am))
    p = _assoc_legendre(l, am, np.sin(phi))[:, None]
    if m == 0:
        ang = np.ones_like(lam)[None, :]
    elif m > 0:
        ang = math.sqrt(2.0) * np.cos(m * lam)[None, :]
    else:
        ang = math.sqrt(2.0) * np.sin(am * lam)[None, :]
    return norm * p * ang


def sh_modes(lmin: int, lmax: int):
    """All (l, m) with lmin <= l <= lmax, -l <= m <= l, in a fixed order."""
    return [(l, m) for l in range(lmin, lmax + 1) for m in range(-l, l + 1)]


def random_sh_field(lam, phi, coeffs: np.ndarray, modes) -> np.ndarray:
    """Sum_k coeffs[k] * Y_{modes[k]} on the grid, evaluated separably: the
    latitude factors are summed per zonal wavenumber first, then one small
    matrix product with the longitude factors gives the field."""
    mmax = max(abs(m) for _, m in modes)
    lat = np.zeros((phi.size, 2 * mmax + 1))
    for c, (l, m) in zip(coeffs, modes):
        am = abs(m)
        norm = math.sqrt((2 * l + 1) / (4.0 * math.pi)
                         * math.factorial(l - am) / math.factorial(l + am))
        if m != 0:
            norm *= math.sqrt(2.0)
        lat[:, m + mmax] += c * norm * _assoc_legendre(l, am, np.sin(phi))
    lon = np.empty((2 * mmax + 1, lam.size))
    for m in range(-mmax, mmax + 1):
        lon[m + mmax] = np.cos(m * lam) if m > 0 else (np.sin(-m * lam) if m < 0 else 1.0)
    return lat @ lon
