"""Pins of the oracle's Fock exchange (Eq. 3) and its ACE compression.

* FFT-free check: on a tiny non-cubic cell the operator is evaluated as a
  direct double sum in reciprocal space,
      rho_ij(q) = Omega^{-1} sum_G c_i^*(G) c_j(G + q),
      d_j(G'')  = -alpha sum_i sum_q c_i(G'' - q) Khat(q) rho_ij(q),
  which is exact for band-limited orbitals. With an alias-free grid the FFT
  pair loop must give the same basis components.
* Grid invariance: two alias-free grids give identical basis components.
* Structure: <a|V_X b> is Hermitian and negative semidefinite (Khat > 0), and
  tr(Psi^H V_X Psi) is real.
* ACE: K_ACE Psi = V_X Psi, xi^H Psi = -L^H, K_ACE Hermitian and NSD.
* Fock grid (the paper's wavefunction grid): on a grid that holds the orbitals
  but aliases their pair products, the FFT pair loop equals the same double
  sum with every frequency folded modulo the grid.
"""
import numpy as np
import pytest

import synthetic as syn
from oracle.discretization import Grid
from oracle import exchange as ex

CELL = (6.1, 7.3, 5.6)
ECUT = 2.5
ALPHA = 0.25
OMEGA = 0.3


def direct_vx(grid, C, X, alpha, omega):
    """Reciprocal-space double sum, independent of every FFT in the oracle."""
    gv = grid.gvec_basis()
    m = np.stack(np.unravel_index(grid.basis, grid.n), axis=-1)
    m = np.where(m < (np.asarray(grid.n) + 1) // 2, m, m - np.asarray(grid.n))
    keys = [tuple(v) for v in m]
    index = {k: a for a, k in enumerate(keys)}
    cellv = np.asarray(grid.cell)

    def khat(q):
        g = 2 * np.pi * np.asarray(q) / cellv
        g2 = float(g @ g)
        if g2 == 0.0:
            return np.pi / omega ** 2
        return 4 * np.pi * (1 - np.exp(-g2 / (4 * omega ** 2))) / g2

    qs = sorted({tuple(np.subtract(b, a)) for a in keys for b in keys})
    kq = {q: khat(q) for q in qs}
    ne = C.shape[1]
    out = np.zeros_like(X)
    for j in range(X.shape[1]):
        for i in range(ne):
            rho = {}
            for q in qs:
                s = 0j
                for a, G in enumerate(keys):
                    b = index.get((G[0] + q[0], G[1] + q[1], G[2] + q[2]))
                    if b is not None:
                        s += np.conj(C[a, i]) * X[b, j]
                rho[q] = s / grid.volume
            for a2, G2 in enumerate(keys):
                s = 0j
                for q in qs:
                    b = index.get((G2[0] - q[0], G2[1] - q[1], G2[2] - q[2]))
                    if b is not None:
                        s += C[b, i] * kq[q] * rho[q]
                out[a2, j] += -alpha * s
    return out


@pytest.fixture(scope="module")
def tiny():
    grid = Grid((12, 16, 10), CELL, ECUT)
    assert grid.alias_free()
    C = syn.gaussian_vectors((grid.npw, 3), seed=11)
    X = syn.gaussian_vectors((grid.npw, 2), seed=12)
    return grid, C, X


def test_vx_equals_direct_reciprocal_sum(tiny):
    grid, C, X = tiny
    khat = ex.screened_kernel(grid, OMEGA)
    got = ex.apply_vx(grid, khat, ALPHA, C, X)
    ref = direct_vx(grid, C, X, ALPHA, OMEGA)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))


def test_vx_grid_invariance(tiny):
    grid, C, X = tiny
    big = Grid((16, 20, 16), CELL, ECUT)
    assert big.alias_free() and big.npw == grid.npw
    # map basis vectors of one grid onto the other by their G vectors
    order_small = np.lexsort(grid.gvec_basis().T)
    order_big = np.lexsort(big.gvec_basis().T)
    assert np.allclose(grid.gvec_basis()[order_small], big.gvec_basis()[order_big])
    perm = np.empty(grid.npw, int)
    perm[order_big] = order_small           # big basis index -> small basis index
    Cb, Xb = C[perm], X[perm]
    a = ex.apply_vx(grid, ex.screened_kernel(grid, OMEGA), ALPHA, C, X)
    b = ex.apply_vx(big, ex.screened_kernel(big, OMEGA), ALPHA, Cb, Xb)
    assert np.max(np.abs(a[perm] - b)) < 1e-12 * np.max(np.abs(a))


def test_vx_hermitian_negative_semidefinite(tiny):
    grid, C, _ = tiny
    khat = ex.screened_kernel(grid, OMEGA)
    V = syn.gaussian_vectors((grid.npw, 6), seed=13)
    A = V.conj().T @ ex.apply_vx(grid, khat, ALPHA, C, V)
    assert np.max(np.abs(A - A.conj().T)) < 1e-12 * np.max(np.abs(A))
    ev = np.linalg.eigvalsh(0.5 * (A + A.conj().T))
    assert ev.max() < 1e-12 * np.abs(ev).max()
    M = C.conj().T @ ex.apply_vx(grid, khat, ALPHA, C, C)
    assert abs(np.imag(np.trace(M))) < 1e-12 * abs(np.trace(M))
    assert np.real(np.trace(M)) < 0


def test_ace_reproduces_exchange_on_orbitals(tiny):
    grid, C, _ = tiny
    khat = ex.screened_kernel(grid, OMEGA)
    W, M, L, xi = ex.build_ace(grid, khat, ALPHA, C)
    assert np.max(np.abs(ex.apply_ace(xi, C) - W)) < 1e-12 * np.max(np.abs(W))
    assert np.max(np.abs(xi.conj().T @ C + L.conj().T)) < 1e-12 * np.max(np.abs(L))
    V = syn.gaussian_vectors((grid.npw, 5), seed=14)
    A = V.conj().T @ ex.apply_ace(xi, V)
    assert np.max(np.abs(A - A.conj().T)) < 1e-12 * np.max(np.abs(A))
    assert np.linalg.eigvalsh(0.5 * (A + A.conj().T)).max() < 1e-12 * np.abs(A).max()


def test_ace_on_si_cell_uses_symmetric_pairs():
    """W from the full N_e^2 loop obeys the pair symmetry v_ji = conj(v_ij) the GPU path exploits."""
    grid = Grid((16, 16, 16), (10.26,) * 3, 2.0)
    C = syn.gaussian_vectors((grid.npw, 4), seed=15)
    psi = grid.to_real(C.T)
    khat = ex.screened_kernel(grid, 0.106)
    v01 = ex.poisson_like(np.conj(psi[0]) * psi[1], khat)
    v10 = ex.poisson_like(np.conj(psi[1]) * psi[0], khat)
    assert np.max(np.abs(v10 - np.conj(v01))) < 1e-13 * np.max(np.abs(v01))


def direct_vx_folded(grid_c, C, X, alpha, omega):
    """The same double sum on a grid that does not hold the pair products: every frequency
    is taken modulo the grid (its representative in the FFT range), as the grid's DFT does."""
    n = np.asarray(grid_c.n)
    m = np.stack(np.unravel_index(grid_c.basis, grid_c.n), axis=-1)
    m = np.where(m < (n + 1) // 2, m, m - n)
    keys = [tuple(v) for v in m]
    cellv = np.asarray(grid_c.cell)

    def rep(q):                                  # representative of q modulo the grid
        q = np.mod(np.asarray(q), n)
        return tuple(np.where(q < (n + 1) // 2, q, q - n))

    def khat(q):
        g = 2 * np.pi * np.asarray(q) / cellv
        g2 = float(g @ g)
        if g2 == 0.0:
            return np.pi / omega ** 2
        return 4 * np.pi * (1 - np.exp(-g2 / (4 * omega ** 2))) / g2

    ne = C.shape[1]
    out = np.zeros_like(X)
    for j in range(X.shape[1]):
        for i in range(ne):
            rho = {}
            for a, G in enumerate(keys):          # rho_ij(q) = Omega^-1 sum c_i^*(G) x_j(G'), G' - G = q mod n
                for b, G1 in enumerate(keys):
                    q = rep(np.subtract(G1, G))
                    rho[q] = rho.get(q, 0j) + np.conj(C[a, i]) * X[b, j] / grid_c.volume
            for q in rho:
                rho[q] *= khat(q)
            for a, G in enumerate(keys):          # W_j(G'') += c_i(G) v_ij(q), G + q = G'' mod n
                for q, v in rho.items():
                    g2 = rep(np.add(G, q))
                    if g2 in keys:
                        out[keys.index(g2), j] += -alpha * C[a, i] * v
    return out


def test_vx_on_an_aliasing_fock_grid():
    """Eq. 3 on a grid that holds the orbitals but not their pair products (the paper's
    choice of evaluating the exchange on the wavefunction grid): the FFT pair loop equals
    the folded reciprocal-space double sum, and differs from the alias-free result."""
    fine = Grid((12, 16, 10), CELL, ECUT)
    coarse = Grid((6, 6, 4), CELL, ECUT)
    assert fine.alias_free() and not coarse.alias_free()
    assert np.array_equal(coarse.gvec_basis(), fine.gvec_basis())
    C = syn.gaussian_vectors((fine.npw, 2), seed=21)
    X = syn.gaussian_vectors((fine.npw, 2), seed=22)
    got = ex.apply_vx(coarse, ex.screened_kernel(coarse, OMEGA), ALPHA, C, X)
    ref = direct_vx_folded(coarse, C, X, ALPHA, OMEGA)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(ref))
    exact = ex.apply_vx(fine, ex.screened_kernel(fine, OMEGA), ALPHA, C, X)
    assert np.max(np.abs(got - exact)) > 1e-3 * np.max(np.abs(exact))


def test_fock_grid_must_hold_the_sphere():
    from oracle import ptcn as pc
    base = dict(n=(12, 16, 10), cell=CELL, ecut=ECUT, atoms=np.zeros((1, 3)), n_orb=2, relax_iters=0)
    pc.Model(pc.Params(fock_grid=(6, 6, 4), **base))
    with pytest.raises(ValueError):
        pc.Model(pc.Params(fock_grid=(4, 4, 4), **base))
