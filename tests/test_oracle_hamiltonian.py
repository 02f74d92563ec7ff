"""Pins of the oracle's Hamiltonian pieces (Eq. 2) and energy.

* Gaussian wells: the oracle builds V_ion from its Fourier series; here it is
  summed directly in real space over atoms and periodic images.
* Hartree: a neutral pair of concentric Gaussians (widths s1, s2) has the
  potential sum_R [erf(d/(sqrt2 s1)) - erf(d/(sqrt2 s2))]/d, compared after
  removing the mean (the G = 0 term is dropped by the solver).
* Energy and Hamiltonian are consistent: for any direction D,
  dE(Psi + eps D)/d eps = 4 Re tr(D^H H[Psi] Psi) (double occupation; the
  Fock term contributes twice V_X psi as every orbital appears twice in E_X).
  A wrong 1/2 in Hartree, a wrong 3/4 or 4/3 in LDA, a wrong Fock weight or a
  sign anywhere fails this.
* Slater exchange constant (3/4)(3/pi)^{1/3} = 0.7385587663820224 (textbook).
"""
import numpy as np
import pytest
from scipy.special import erf

import synthetic as syn
from oracle.discretization import Grid
from oracle import hamiltonian as hm
from oracle import ptcn as pc


def test_ion_potential_matches_real_space_sum():
    cell = np.array([8.0, 9.0, 7.5])
    grid = Grid((24, 24, 20), cell, 2.0)
    atoms = np.array([[0.1, 0.2, 0.3], [0.6, 0.55, 0.9], [0.35, 0.8, 0.05]])
    D, sig = 2.0, 1.2
    v = hm.ion_potential(grid, atoms, D, sig)
    rng = np.random.default_rng(5)
    idx = rng.integers(0, grid.N, size=200)
    pts = grid.r_coords().reshape(-1, 3)[idx]
    ref = np.zeros(len(idx))
    for f in atoms:
        for i in range(-3, 4):
            for j in range(-3, 4):
                for k in range(-3, 4):
                    d = pts - (f * cell + np.array([i, j, k]) * cell)
                    ref += -D * np.exp(-np.sum(d * d, axis=1) / (2 * sig * sig))
    assert np.max(np.abs(v.reshape(-1)[idx] - ref)) < 1e-12 * np.max(np.abs(ref))


def test_hartree_neutral_gaussian_pair():
    cell = np.array([12.0, 12.0, 13.0])
    grid = Grid((40, 40, 44), cell, 2.0)
    c = np.array([0.4, 0.55, 0.45]) * cell
    s1, s2 = 0.9, 1.4
    r = grid.r_coords()

    def gauss(s):
        out = np.zeros(grid.n)
        for i in range(-1, 2):
            for j in range(-1, 2):
                for k in range(-1, 2):
                    d = r - (c + np.array([i, j, k]) * cell)
                    out += np.exp(-np.sum(d * d, axis=-1) / (2 * s * s))
        return out / (2 * np.pi * s * s) ** 1.5

    rho = gauss(s1) - gauss(s2)
    v = hm.hartree_potential(grid, rho)
    d = np.linalg.norm(r - c, axis=-1)
    ref = np.zeros(grid.n)
    for i in range(-2, 3):
        for j in range(-2, 3):
            for k in range(-2, 3):
                d = np.linalg.norm(r - (c + np.array([i, j, k]) * cell), axis=-1)
                small = d < 1e-12
                dd = np.where(small, 1.0, d)
                val = (erf(dd / (np.sqrt(2) * s1)) - erf(dd / (np.sqrt(2) * s2))) / dd
                ref += np.where(small, np.sqrt(2 / np.pi) * (1 / s1 - 1 / s2), val)
    ref -= ref.mean()
    assert np.max(np.abs(v - ref)) < 1e-10 * np.max(np.abs(ref))


def test_slater_constant():
    assert hm.SLATER_C == pytest.approx(0.7385587663820224, rel=1e-15)
    rho = np.array([0.3])
    # v_x = d e_x / d rho for e_x = -C rho^{4/3}
    assert hm.lda_exchange_potential(rho)[0] == pytest.approx(-(4.0 / 3.0) * hm.SLATER_C * rho[0] ** (1 / 3), rel=1e-14)


@pytest.mark.parametrize("fock_mode", ["exact"])
def test_energy_gradient_matches_hamiltonian(fock_mode):
    cell, frac = syn.diamond_supercell(1)
    p = pc.Params(n=(16, 16, 16), cell=tuple(cell), ecut=2.0, atoms=frac, n_orb=3,
                  kick=(0.02, -0.01, 0.005), fock_mode=fock_mode, relax_iters=0)
    m = pc.Model(p)
    Psi = syn.gaussian_vectors((m.grid.npw, 3), seed=21) * 0.1
    D = syn.gaussian_vectors((m.grid.npw, 3), seed=22) * 0.1

    def energy(P):
        W = m.vx(P, P)
        return m.observables(P, P.conj().T @ W)[0]

    eps = 1e-4
    fd = (energy(Psi + eps * D) - energy(Psi - eps * D)) / (2 * eps)
    HP = m.apply_h(Psi, Psi, "exact")
    an = 4.0 * np.real(np.sum(np.conj(D) * HP))
    assert fd == pytest.approx(an, rel=1e-7)


def test_dipole_of_point_like_density():
    grid = Grid((16, 16, 16), (10.0, 10.0, 10.0), 1.0)
    rho = np.zeros(grid.n)
    rho[4, 8, 2] = 1.0 / grid.dV
    d = hm.dipole(grid, rho)
    assert np.allclose(d, -np.array([4 * 10 / 16, 8 * 10 / 16, 2 * 10 / 16]), rtol=0, atol=1e-14)
