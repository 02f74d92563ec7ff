"""ORACLE (test infrastructure only): planewave discretisation of a periodic cell.

The paper works at the Gamma point with a planewave basis cut off at
|G|^2/2 <= Ecut (Sec. 3.1; Sec. 4 sets the cutoff to 10 Ha).
Orbitals are stored as basis coefficients c(G) with

    psi(r) = Omega^{-1/2} sum_G c(G) exp(i G.r),      sum_G |c(G)|^2 = <psi|psi>,

and are taken to a real-space grid of n0 x n1 x n2 points (row-major, axis 2
fastest) by a dense inverse FFT. G = 2 pi (m0/a0, m1/a1, m2/a2) with the
integer frequencies m in FFT index order. The basis is the set of grid
frequencies inside the cutoff sphere listed by increasing flat grid index.
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

# Threads scipy.fft may use (the CPU-baseline timing raises this; tests keep 1).
FFT_WORKERS = 1


def fftn(x):
    """Unnormalised forward DFT over the last three axes: sum_r x(r) exp(-2 pi i m.r/n)."""
    return sfft.fftn(x, axes=(-3, -2, -1), workers=FFT_WORKERS)


def ifftn(x):
    """Inverse DFT over the last three axes with the 1/N factor (numpy convention)."""
    return sfft.ifftn(x, axes=(-3, -2, -1), workers=FFT_WORKERS)


def integer_frequencies(n: int) -> np.ndarray:
    """m for FFT index k: k for k < n/2, k - n above (index n/2 maps to -n/2)."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


class Grid:
    """Cell, real-space grid, reciprocal vectors and the planewave basis."""

    def __init__(self, n, cell, ecut: float):
        self.n = tuple(int(v) for v in n)
        self.cell = np.asarray(cell, dtype=np.float64)
        self.ecut = float(ecut)
        self.volume = float(np.prod(self.cell))
        self.N = int(np.prod(self.n))
        self.dV = self.volume / self.N
        self.m = [integer_frequencies(nk) for nk in self.n]
        self.g = [2.0 * np.pi * self.m[k] / self.cell[k] for k in range(3)]
        g0, g1, g2 = np.meshgrid(*self.g, indexing="ij")
        self.gvec = np.stack([g0, g1, g2], axis=-1)          # (n0, n1, n2, 3)
        self.g2 = g0 ** 2 + g1 ** 2 + g2 ** 2                 # |G|^2 on the grid
        # basis: 0.5 |G|^2 <= ecut, increasing flat index
        self.basis = np.flatnonzero(0.5 * self.g2.reshape(-1) <= self.ecut)
        self.npw = self.basis.size

    # -- basis data ---------------------------------------------------------
    def g2_basis(self) -> np.ndarray:
        return self.g2.reshape(-1)[self.basis]

    def gvec_basis(self) -> np.ndarray:
        return self.gvec.reshape(-1, 3)[self.basis]

    def alias_free(self) -> bool:
        """True when every pair product of basis functions is resolved on the grid.

        Pair densities hold frequencies up to twice the cutoff radius; with
        m_c the largest |m_k| in the basis, the grid must satisfy n_k > 4 m_c,k
        so that neither the pair density nor its product with an orbital folds
        back into the basis sphere.
        """
        mb = np.stack([np.abs(self.m[k])[np.unravel_index(self.basis, self.n)[k]] for k in range(3)], axis=-1)
        mc = mb.max(axis=0)
        return bool(np.all(np.asarray(self.n) > 4 * mc))

    # -- transforms -------------------------------------------------------
    def to_real(self, c: np.ndarray) -> np.ndarray:
        """Basis coefficients (..., npw) -> psi on the grid (..., n0, n1, n2)."""
        c = np.asarray(c, dtype=np.complex128)
        full = np.zeros(c.shape[:-1] + (self.N,), dtype=np.complex128)
        full[..., self.basis] = c
        full = full.reshape(c.shape[:-1] + self.n)
        return ifftn(full) * (self.N / np.sqrt(self.volume))

    def to_basis(self, f: np.ndarray) -> np.ndarray:
        """Grid function (..., n0, n1, n2) -> its planewave-basis components (..., npw).

        d(G) = Omega^{-1/2} * integral exp(-i G.r) f(r) dr, by the grid sum with weight dV.
        """
        f = np.asarray(f, dtype=np.complex128)
        F = fftn(f).reshape(f.shape[:-3] + (self.N,))
        return F[..., self.basis] * (np.sqrt(self.volume) / self.N)

    def r_coords(self) -> np.ndarray:
        """Cartesian coordinates of the grid points in [0, a), shape (n0, n1, n2, 3)."""
        axes = [np.arange(self.n[k]) * (self.cell[k] / self.n[k]) for k in range(3)]
        r0, r1, r2 = np.meshgrid(*axes, indexing="ij")
        return np.stack([r0, r1, r2], axis=-1)
