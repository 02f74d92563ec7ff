"""ORACLE (test infrastructure only): Fock exchange, Eq. 3, and its ACE form.

Eq. 3 applies the exchange operator to an orbital psi_j as

    (V_X psi_j)(r) = - sum_i psi_i(r) * integral K(r - r') psi_i^*(r') psi_j(r') dr',

one Poisson-like solve per pair (i, j), N_e^2 of them (Sec. 2; Alg. 2 loops
over i and j). The kernel is the screened interaction of the range-separated
hybrid, with the mixing fraction alpha of Sec. 2 (whose operator kernel is
-alpha P(r,r') K(r,r')) kept in front. Reading: Eq. 3 drops alpha; it is
restored here, as the operator kernel of Sec. 2 has it.

The screened Coulomb kernel is K(r) = erfc(w r)/r, whose Fourier transform is

    Khat(G) = 4 pi (1 - exp(-|G|^2 / (4 w^2))) / |G|^2,   Khat(0) = pi / w^2

(the G -> 0 limit, equal to the integral of erfc(w r)/r over space). With
rho_ij(r) = psi_i^*(r) psi_j(r) on the grid the convolution is exactly

    v_ij = ifftn(Khat * fftn(rho_ij))          (numpy normalisation, no other factor).

ACE (the compression the paper cites in Sec. 1; its formulas are not printed
in the paper): with W = V_X Psi, M = Psi^H W, -M = L L^H (Cholesky),
xi = W L^{-H}, the compressed operator is K_ACE X = -xi (xi^H X), which agrees
with V_X on the span of Psi.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .discretization import Grid, fftn, ifftn


def screened_kernel(grid: Grid, omega: float) -> np.ndarray:
    """Khat(G) on the FFT grid for the erfc(w r)/r interaction (G = 0 -> pi / w^2)."""
    g2 = grid.g2
    out = np.empty_like(g2)
    nz = g2 > 0.0
    out[nz] = 4.0 * np.pi * (-np.expm1(-g2[nz] / (4.0 * omega * omega))) / g2[nz]
    out[~nz] = np.pi / (omega * omega)
    return out


def poisson_like(rho_r: np.ndarray, khat: np.ndarray) -> np.ndarray:
    """Periodic convolution of a grid function with K: ifftn(Khat * fftn(rho)) (Eq. 3 integral)."""
    return ifftn(khat * fftn(rho_r))


def apply_vx_real(psi_r: np.ndarray, phi_r: np.ndarray, khat: np.ndarray, alpha: float) -> np.ndarray:
    """V_X[P] phi_j on the grid for P = sum_i psi_i psi_i^*, by the N_e x m pair loop of Alg. 2.

    psi_r: (N_e, n0, n1, n2) orbitals that define the density matrix.
    phi_r: (m, n0, n1, n2) functions to apply the operator to.
    Returns (m, n0, n1, n2). For each target j the i loop is batched into one
    array FFT (a library primitive); every pair (i, j) is solved on its own.
    """
    out = np.zeros_like(phi_r, dtype=np.complex128)
    for j in range(phi_r.shape[0]):
        rho = np.conj(psi_r) * phi_r[j][None]            # rho_ij(r) = psi_i^*(r) phi_j(r), all i
        v = poisson_like(rho, khat[None])                 # v_ij(r)
        out[j] = np.sum(psi_r * v, axis=0)                # sum_i psi_i(r) v_ij(r)
    return -alpha * out


def apply_vx(grid: Grid, khat: np.ndarray, alpha: float, C: np.ndarray, X: np.ndarray) -> np.ndarray:
    """Basis coefficients of V_X[P] x for columns x of X (npw, m), P built from columns of C (npw, N_e)."""
    psi_r = grid.to_real(C.T)
    phi_r = psi_r if X is C else grid.to_real(X.T)
    return grid.to_basis(apply_vx_real(psi_r, phi_r, khat, alpha)).T


def build_ace(grid: Grid, khat: np.ndarray, alpha: float, C: np.ndarray):
    """ACE from the orbitals C (npw, N_e): returns (W, M, L, xi).

    W = V_X C (exact, Eq. 3), M = C^H W, -M = L L^H, xi = W L^{-H}.
    """
    W = apply_vx(grid, khat, alpha, C, C)
    M = C.conj().T @ W
    L = np.linalg.cholesky(-M)                           # raises if -M is not positive definite
    xi = sla.solve_triangular(L.conj(), W.T, lower=True).T   # xi L^H = W  <=>  conj(L) xi^T = W^T
    return W, M, L, xi


def apply_ace(xi: np.ndarray, X: np.ndarray) -> np.ndarray:
    """K_ACE X = -xi (xi^H X)."""
    return -(xi @ (xi.conj().T @ X))
