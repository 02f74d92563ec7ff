"""Pins of the oracle's screened-Coulomb solve (the Poisson-like problem of Eq. 3).

The convolution ifftn(Khat * fftn(rho)) is checked against the analytic
potential of a periodic Gaussian charge, which the oracle never evaluates:
a normalised Gaussian of width s under erfc(w r)/r gives

    V(d) = [erf(d / (sqrt(2) s)) - erf(d / sqrt(2 s^2 + 1/w^2))] / d,
    V(0) = sqrt(2/pi) (1/s - 1/sqrt(s^2 + 1/(2 w^2))),

summed over periodic images (the screened kernel decays like erfc(w d)/d, so
images out to ~60 bohr suffice at w = 0.106). A wrong 4 pi, a missing
1/(4 w^2), a wrong G = 0 value or a stray FFT normalisation all fail here.
"""
import numpy as np
import pytest
from scipy.special import erf

from oracle.discretization import Grid
from oracle.exchange import poisson_like, screened_kernel


def periodic_gaussian(grid, center, s):
    r = grid.r_coords()
    rho = np.zeros(grid.n)
    cell = grid.cell
    nimg = [int(np.ceil(8 * s / cell[k])) + 1 for k in range(3)]
    for i in range(-nimg[0], nimg[0] + 1):
        for j in range(-nimg[1], nimg[1] + 1):
            for k in range(-nimg[2], nimg[2] + 1):
                d = r - (np.asarray(center) + np.array([i, j, k]) * cell)
                rho += np.exp(-np.sum(d * d, axis=-1) / (2 * s * s))
    return rho / (2 * np.pi * s * s) ** 1.5


def screened_gaussian_potential(points, center, cell, s, w, rmax):
    out = np.zeros(len(points))
    nimg = [int(np.ceil(rmax / cell[k])) + 1 for k in range(3)]
    a = np.sqrt(2.0) * s
    b = np.sqrt(2.0 * s * s + 1.0 / (w * w))
    v0 = np.sqrt(2.0 / np.pi) * (1.0 / s - 1.0 / np.sqrt(s * s + 1.0 / (2.0 * w * w)))
    for i in range(-nimg[0], nimg[0] + 1):
        for j in range(-nimg[1], nimg[1] + 1):
            for k in range(-nimg[2], nimg[2] + 1):
                d = np.linalg.norm(points - (np.asarray(center) + np.array([i, j, k]) * cell), axis=1)
                small = d < 1e-12
                dd = np.where(small, 1.0, d)
                val = (erf(dd / a) - erf(dd / b)) / dd
                out += np.where(small, v0, val)
    return out


@pytest.mark.parametrize("w,n,cell,rmax", [
    (0.106, (32, 36, 30), (10.26, 11.5, 9.8), 70.0),
    (0.5, (24, 24, 28), (8.0, 8.0, 9.0), 20.0),
])
def test_screened_poisson_matches_erf_closed_form(w, n, cell, rmax):
    s = 1.0
    grid = Grid(n, cell, ecut=1.0)
    center = np.array([0.31, 0.47, 0.22]) * np.asarray(cell)
    rho = periodic_gaussian(grid, center, s)
    v = np.real(poisson_like(rho.astype(complex), screened_kernel(grid, w)))
    rng = np.random.default_rng(3)
    idx = rng.integers(0, grid.N, size=300)
    pts = grid.r_coords().reshape(-1, 3)[idx]
    ref = screened_gaussian_potential(pts, center, np.asarray(cell), s, w, rmax)
    got = v.reshape(-1)[idx]
    assert np.max(np.abs(got - ref)) < 1e-11 * np.max(np.abs(ref))


def test_kernel_g0_is_limit():
    grid = Grid((8, 8, 8), (1e4, 1e4, 1e4), ecut=1.0)   # huge cell: smallest |G| ~ 6e-4
    k = screened_kernel(grid, 0.3)
    assert k[0, 0, 0] == pytest.approx(np.pi / 0.09, rel=1e-14)
    assert k[1, 0, 0] == pytest.approx(np.pi / 0.09, rel=1e-5)
    assert np.all(k > 0)
