"""Teter-Payne-Allan (TPA) preconditioner on a real-space grid (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Section 5.3 solves its Hamiltonian problems with the preconditioner of Teter,
Payne and Allan (Phys. Rev. B 40, 12255, 1989): a positive diagonal matrix in
the plane-wave basis, so T is symmetric positive definite and cheap.  For a
plane wave G the published factor is

    K(x) = (27 + 18 x + 12 x^2 + 8 x^3) / (27 + 18 x + 12 x^2 + 8 x^3 + 16 x^4),

with x the wave's kinetic energy over a reference kinetic energy E.  On the
finite-difference grid the readings taken are:

* the "plane waves" are the eigenvectors of the grid's own kinetic operator
  -1/2 Lap_h: Fourier modes on a periodic grid, sine modes on a Dirichlet grid,
  and the kinetic energy of a mode is its eigenvalue of -1/2 Lap_h, so T
  commutes with -1/2 Lap_h;
* E is one fixed positive number for all columns (the paper applies T as a
  fixed diagonal matrix); by default E = sigma - min V (an upper bound of the
  kinetic energy of a state at energy sigma) when that is positive, otherwise
  the mean kinetic energy of the grid's modes, d / h^2;
* T = F^T diag(K(x)) F with F the orthonormal transform to those modes.

Here the transforms are numpy/scipy FFTs (library primitives, one step each).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def tpa_factor(x):
    x = np.asarray(x, dtype=np.float64)
    num = 27.0 + 18.0 * x + 12.0 * x**2 + 8.0 * x**3
    return num / (num + 16.0 * x**4)


def kinetic_symbol(dims, h: float, periodic: bool, scale: float = 0.5):
    """Eigenvalues of scale * (-Lap_h) per mode (scale 1/2: the kinetic operator), as an array shaped (nz, ny, nx) for
    dims = (nx, ny, nz) (reversed order), in the mode order of numpy's fftn
    (periodic) or scipy's type-I DST (Dirichlet, modes 1..N)."""
    axes = []
    for N in reversed(dims):
        m = np.arange(N)
        if periodic:
            mu = (2.0 - 2.0 * np.cos(2.0 * np.pi * m / N)) / h**2
        else:
            mu = (2.0 - 2.0 * np.cos((m + 1) * np.pi / (N + 1))) / h**2
        axes.append(mu)
    grids = np.meshgrid(*axes, indexing="ij")
    return scale * sum(grids)


def default_energy(sigma: float, V, dims, h: float, scale: float = 0.5) -> float:
    """sigma - min V when positive, else the mean of the kinetic symbol
    (scale * 2 d / h^2)."""
    e = sigma - float(np.min(V)) if V is not None and np.size(V) else sigma
    return e if e > 0 else scale * 2.0 * len(dims) / h**2


class TPA:
    """x -> T x on blocks (n x c, rows ordered x fastest)."""

    def __init__(self, dims, h: float, energy: float, periodic: bool = True, scale: float = 0.5):
        if not energy > 0:
            raise ValueError("energy must be positive")
        self.dims = tuple(dims)
        self.shape = tuple(reversed(self.dims))
        self.periodic = periodic
        self.energy = energy
        self.factor = tpa_factor(kinetic_symbol(dims, h, periodic, scale) / energy)

    def _one(self, x):
        X = x.reshape(self.shape)
        if self.periodic:
            return np.real(np.fft.ifftn(self.factor * np.fft.fftn(X))).ravel()
        Y = sfft.dstn(X, type=1, norm="ortho")
        return sfft.idstn(self.factor * Y, type=1, norm="ortho").ravel()

    def __call__(self, R):
        R = np.asarray(R, dtype=np.float64)
        if R.ndim == 1:
            return self._one(R)
        return np.stack([self._one(R[:, c]) for c in range(R.shape[1])], axis=1)
