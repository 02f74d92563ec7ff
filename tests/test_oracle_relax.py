"""Pins of the oracle's start-state relaxation (``Model.relax``).

The paper propagates from a ground state (Sec. 4); the synthetic start orbitals
are random, so both paths first relax them by preconditioned steepest descent
on the local Hamiltonian with a Kerker-mixed density. That procedure is the
builder's reading, not the paper's, so it is pinned here by what its fixed
point must be, computed without the procedure itself:

* Linear H (alpha = 0, no Hartree, no LDA): the Kerker mixing is inert and the
  iteration must converge to the span of the lowest n_orb eigenvectors of the
  dense Hamiltonian matrix (``numpy.linalg.eigh``); the projector defect falls
  geometrically with the iteration count, the sum of the band energies reaches
  the sum of the lowest eigenvalues, and the orbitals stay orthonormal.
* Hartree + Slater LDA on: the fixed point is the self-consistent aufbau state
  -- its residual H[rho(Psi)] Psi - Psi (Psi^H H[rho(Psi)] Psi) with the
  density of Psi itself (not the mixed one) falls towards zero, and Psi spans
  the lowest n_orb eigenvectors of its own dense H[rho(Psi)].

A sign error in the descent or in the Kerker update, a wrong preconditioner
(one that does not keep the step a descent direction) or a missing
re-orthonormalisation fails one of these.
"""
import numpy as np

import synthetic as syn
from oracle import ptcn as pc

N_ORB = 7   # a gap of 0.14 Ha follows the 7th eigenvalue of the tiny cell's linear H


def model(**kw):
    cell, frac = syn.diamond_supercell(1)
    base = dict(n=(12, 12, 12), cell=tuple(cell), ecut=1.5, atoms=frac, n_orb=N_ORB, relax_iters=0)
    base.update(kw)
    return pc.Model(pc.Params(**base))


def dense_h(m, rho):
    eye = np.eye(m.grid.npw, dtype=complex)
    H = m.local.apply_local(m.local.local_potential(rho), eye)
    return 0.5 * (H + H.conj().T)


def start(m):
    C0 = syn.initial_coefficients(m.grid.g2_basis(), N_ORB, seed=3)
    return pc.orthonormalize(C0.T)


def test_relax_reaches_lowest_eigenspace_of_linear_h():
    m = model(alpha=0.0, use_hartree=False, use_lda=False)
    H = dense_h(m, np.zeros(m.grid.N))
    w, V = np.linalg.eigh(H)
    assert w[N_ORB] - w[N_ORB - 1] > 0.1
    P_eig = V[:, :N_ORB] @ V[:, :N_ORB].conj().T
    Psi0 = start(m)
    defects = []
    Psi = Psi0
    for iters in (40, 80, 160, 320):
        Psi = m.relax(Psi0, iters, 1.0)
        defects.append(np.linalg.norm(Psi @ Psi.conj().T - P_eig))
        assert np.max(np.abs(Psi.conj().T @ Psi - np.eye(N_ORB))) < 1e-13
    assert all(b < 0.1 * a for a, b in zip(defects, defects[1:])), defects
    assert defects[-1] < 1e-10, defects
    band = np.real(np.trace(Psi.conj().T @ H @ Psi))
    assert abs(band - np.sum(w[:N_ORB])) < 1e-12


def test_relax_reaches_self_consistent_aufbau_state():
    m = model(alpha=0.0)          # Hartree and Slater LDA on
    Psi0 = start(m)
    resid = []
    Psi = Psi0
    for iters in (40, 80, 160, 320):
        Psi = m.relax(Psi0, iters, 1.0)
        rho = m.density(Psi)
        HP = m.local.apply_local(m.local.local_potential(rho), Psi)
        resid.append(np.linalg.norm(HP - Psi @ (Psi.conj().T @ HP)))
    assert all(b < 0.1 * a for a, b in zip(resid, resid[1:])), resid
    assert resid[-1] < 1e-12, resid
    w, V = np.linalg.eigh(dense_h(m, m.density(Psi)))
    assert w[N_ORB] - w[N_ORB - 1] > 0.1
    P_eig = V[:, :N_ORB] @ V[:, :N_ORB].conj().T
    assert np.linalg.norm(Psi @ Psi.conj().T - P_eig) < 1e-11
