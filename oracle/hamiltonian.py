"""ORACLE (test infrastructure only): the Hamiltonian of Eq. 2 and observables.

H = -1/2 Laplacian + V_ext + V_Hxc[P] + V_X[P]   (Eq. 2)

Readings used here (the paper's pseudopotentials, HSE06 and laser are not
reproducible without their data files; the test cells use these stand-ins):

* V_ext: a periodic sum of Gaussian wells -D exp(-|r - R_a|^2 / (2 sigma^2)),
  defined by its Fourier series
  Vhat(G) = -D (2 pi sigma^2)^{3/2} / Omega * sum_a exp(-i G.R_a) exp(-sigma^2 |G|^2 / 2).
* External field: a velocity-gauge kick kappa (plus, when switched on, the
  laser vector potential A(t) of the PT-CN model), so the kinetic term is
  |G + kappa|^2 / 2 on each basis vector (the phases of the length-gauge
  kick exp(i kappa.r) are not periodic on the cell).
* V_Hxc: Hartree 4 pi rhohat(G)/|G|^2 with the G = 0 term removed
  (neutralising background) plus (1 - alpha) times Slater exchange
  v_x = -(3 rho / pi)^{1/3}; Fock exchange carries weight alpha.
* Spin is omitted as in Sec. 2: every orbital is doubly occupied, rho = 2 sum |psi_i|^2,
  and V_X sums over the N_e orbitals of one spin.
* Energy: E = 2 sum_i <psi_i| -Lap/2 |psi_i> + int V_ion rho + 1/2 int V_H rho
  + (1 - alpha) E_x^LDA[rho] + tr(Psi^H V_X Psi), with
  E_x^LDA = -3/4 (3/pi)^{1/3} int rho^{4/3}.
* Dipole: d = -dV sum_r r rho(r), r the grid coordinates in [0, a) (a fixed
  functional of rho used for comparison; the periodic dipole is not unique).
"""
from __future__ import annotations

import numpy as np

from .discretization import Grid, fftn, ifftn


def density(grid: Grid, psi_r: np.ndarray) -> np.ndarray:
    """rho(r) = 2 sum_i |psi_i(r)|^2 (Sec. 3.4, with double occupation)."""
    return 2.0 * np.sum(np.abs(psi_r) ** 2, axis=0)


def ion_potential(grid: Grid, atoms_frac: np.ndarray, depth: float, sigma: float) -> np.ndarray:
    """Gaussian-well external potential on the grid, from its Fourier series."""
    m = grid.m
    frac = np.asarray(atoms_frac, dtype=np.float64).reshape(-1, 3)
    sf = np.zeros(grid.n, dtype=np.complex128)
    for f in frac:
        p0 = np.exp(-2j * np.pi * m[0] * f[0])
        p1 = np.exp(-2j * np.pi * m[1] * f[1])
        p2 = np.exp(-2j * np.pi * m[2] * f[2])
        sf += p0[:, None, None] * p1[None, :, None] * p2[None, None, :]
    vhat = (-depth * (2.0 * np.pi * sigma * sigma) ** 1.5 / grid.volume) * sf * np.exp(-0.5 * sigma * sigma * grid.g2)
    # V(r) = sum_G Vhat(G) exp(i G.r) = N * ifftn(Vhat); real up to the (negligible) Nyquist terms.
    return np.real(ifftn(vhat) * grid.N)


def hartree_potential(grid: Grid, rho: np.ndarray) -> np.ndarray:
    """V_H = ifftn(4 pi / |G|^2 * fftn(rho)), G = 0 removed."""
    g2 = grid.g2
    fac = np.zeros_like(g2)
    nz = g2 > 0.0
    fac[nz] = 4.0 * np.pi / g2[nz]
    return np.real(ifftn(fac * fftn(rho.astype(np.complex128))))


SLATER_C = 0.75 * (3.0 / np.pi) ** (1.0 / 3.0)


def lda_exchange_potential(rho: np.ndarray) -> np.ndarray:
    """Slater exchange potential -(3 rho / pi)^{1/3}."""
    return -np.cbrt(3.0 * rho / np.pi)


def lda_exchange_energy(grid: Grid, rho: np.ndarray) -> float:
    """-3/4 (3/pi)^{1/3} int rho^{4/3}."""
    return float(-SLATER_C * grid.dV * np.sum(np.cbrt(rho) * rho))


def kinetic_diagonal(grid: Grid, kick) -> np.ndarray:
    """|G + kappa|^2 / 2 on the basis vectors."""
    gk = grid.gvec_basis() + np.asarray(kick, dtype=np.float64)[None, :]
    return 0.5 * np.sum(gk * gk, axis=1)


class LocalModel:
    """Everything of Eq. 2 except V_X: kinetic diagonal, V_ion, switches for Hartree / LDA."""

    def __init__(self, grid: Grid, atoms_frac, depth, sigma, kick, alpha, use_hartree=True, use_lda=True):
        self.grid = grid
        self.kick = np.asarray(kick, dtype=np.float64)
        self.kin = kinetic_diagonal(grid, kick)
        self.v_ion = ion_potential(grid, atoms_frac, depth, sigma)
        self.alpha = float(alpha)
        self.use_hartree = bool(use_hartree)
        self.use_lda = bool(use_lda)

    def local_potential(self, rho: np.ndarray) -> np.ndarray:
        v = self.v_ion.copy()
        if self.use_hartree:
            v = v + hartree_potential(self.grid, rho)
        if self.use_lda:
            v = v + (1.0 - self.alpha) * lda_exchange_potential(rho)
        return v

    def kin_at(self, a_field) -> np.ndarray:
        """Kinetic diagonal |G + kappa + A|^2 / 2 for a vector potential A (velocity gauge)."""
        return kinetic_diagonal(self.grid, self.kick + np.asarray(a_field, dtype=np.float64))

    def apply_local(self, vloc: np.ndarray, X: np.ndarray, kin=None) -> np.ndarray:
        """Kinetic + local part of H on the columns of X (npw, m); kin defaults to the kick's."""
        g = self.grid
        k = self.kin if kin is None else kin
        return k[:, None] * X + g.to_basis(vloc[None] * g.to_real(X.T)).T

    def energy_terms(self, C: np.ndarray, rho: np.ndarray, exx: float, kin=None) -> dict:
        g = self.grid
        k = self.kin if kin is None else kin
        e = dict(kinetic=float(2.0 * np.sum(k[:, None] * np.abs(C) ** 2)),
                 ion=float(g.dV * np.sum(self.v_ion * rho)),
                 hartree=0.0, xc=0.0, fock=float(exx))
        if self.use_hartree:
            e["hartree"] = float(0.5 * g.dV * np.sum(hartree_potential(g, rho) * rho))
        if self.use_lda:
            e["xc"] = (1.0 - self.alpha) * lda_exchange_energy(g, rho)
        e["total"] = e["kinetic"] + e["ion"] + e["hartree"] + e["xc"] + e["fock"]
        return e


def dipole(grid: Grid, rho: np.ndarray) -> np.ndarray:
    """d = -dV sum_r r rho(r) with r in [0, a)."""
    r = grid.r_coords()
    return -grid.dV * np.einsum("abcx,abc->x", r, rho)
