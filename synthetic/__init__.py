"""Seeded synthetic inputs shared by the oracle-side tests and the CUDA-side callers.

This module only draws random numbers and lays out the silicon-like test cells.
It holds none of the method's arithmetic (no Hamiltonian, no FFT, no exchange,
no propagation): every quantity the method computes is computed separately by
``oracle/`` and by the CUDA library.

Workload recipe (the paper's test system, Sec. 4, is a silicon supercell built
from simple-cubic 8-atom diamond cells with lattice constant 5.43 Angstrom,
10 Ha planewave cutoff and a 50 as time step; the pseudopotential and the laser
of the paper are replaced by Gaussian wells and a velocity-gauge kick):

* cell: ``reps`` x ``reps`` x ``reps`` cubic diamond cells of edge 10.26 bohr;
* atoms: the 8 diamond sites of each cell (fractional positions below);
* orbitals: two electrons per atom, so ``n_orb = 4 * n_atoms / 2 = 16 reps**3``
  doubly occupied orbitals (Si has 4 valence electrons);
* initial coefficients: ``c_b(G) = (g1 + i g2) exp(-|G|^2 / 4)`` with ``g1, g2``
  standard normal from ``numpy.random.Generator(PCG64(seed))``, drawn band by
  band over the basis vectors in the order given by the caller (the basis is
  the set of grid frequencies with |G|^2/2 <= ecut, listed by increasing
  row-major flat grid index); these are NOT orthonormal, each side
  orthonormalises them itself.
"""
from __future__ import annotations

import numpy as np

BOHR_PER_ANGSTROM = 1.8897261254578281
# Simple-cubic diamond cell of the paper's test system (Sec. 4): 5.43 Angstrom.
SI_CUBIC_CELL_BOHR = 10.26
# 50 attoseconds in atomic time units (1 a.u. = 24.188843 as), as the configs round it.
DT_50AS = 2.07

# Fractional positions of the 8 atoms of the conventional cubic diamond cell:
# the 4 fcc sites and the same sites shifted by (1/4, 1/4, 1/4).
_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
DIAMOND_SITES = np.concatenate([_FCC, _FCC + 0.25])


def diamond_supercell(reps: int) -> tuple[np.ndarray, np.ndarray]:
    """Return (cell edge lengths in bohr, fractional atom positions) of a reps^3 supercell."""
    reps = int(reps)
    shifts = np.array([[i, j, k] for i in range(reps) for j in range(reps) for k in range(reps)], dtype=float)
    frac = (DIAMOND_SITES[None, :, :] + shifts[:, None, :]).reshape(-1, 3) / reps
    cell = np.full(3, SI_CUBIC_CELL_BOHR * reps)
    return cell, frac


# Named workloads: grid points per edge, supercell repetitions, orbitals.
SI_CONFIGS = {
    "si8": dict(n=(32, 32, 32), reps=1, n_orb=16),
    "si64": dict(n=(64, 64, 64), reps=2, n_orb=128),
    "si216": dict(n=(96, 96, 96), reps=3, n_orb=432),
}

# Physical parameters common to every workload (Gaussian wells of depth 2 Ha and
# width 1.2 bohr, screened exchange with w = 0.106 / bohr and mixing 0.25, 10 Ha
# cutoff, kick 0.01 / bohr along x, dt = 50 as).
COMMON = dict(
    ecut=10.0,
    well_depth=2.0,
    well_sigma=1.2,
    omega=0.106,
    alpha=0.25,
    dt=DT_50AS,
    kick=(0.01, 0.0, 0.0),
    anderson_dim=20,
    anderson_beta=1.0,
    scf_tol=1e-6,
    scf_max=50,
    scf_fixed_iters=0,
    # mixed precision: below this SCF tolerance the late iterations run in FP64
    # (no effect at the paper's tolerance 1e-6)
    scf_fp64_below=1e-7,
)


def si_workload(name: str, **overrides) -> dict:
    """Full parameter dictionary of a named silicon workload (cell, atoms, grid, physics)."""
    cfg = SI_CONFIGS[name]
    cell, frac = diamond_supercell(cfg["reps"])
    out = dict(COMMON)
    out.update(n=tuple(cfg["n"]), cell=tuple(cell), atoms=frac, n_orb=cfg["n_orb"], seed=0)
    out.update(overrides)
    return out


def initial_coefficients(g2_basis: np.ndarray, n_orb: int, seed: int) -> np.ndarray:
    """Random initial orbital coefficients, shape (n_orb, n_basis), complex128.

    ``g2_basis`` is |G|^2 of each basis vector in basis order (supplied by the
    caller). Row b is orbital b. The envelope exp(-|G|^2/4) keeps the start
    state smooth; the rows are not orthonormal.
    """
    g2 = np.asarray(g2_basis, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    z = rng.standard_normal((int(n_orb), g2.size, 2))
    return (z[..., 0] + 1j * z[..., 1]) * np.exp(-g2 / 4.0)[None, :]


_GOLDEN = np.uint64(0x9E3779B97F4A7C15)


def splitmix64(seed: int, k: np.ndarray) -> np.ndarray:
    """Outputs k (0, 1, ...) of SplitMix64 (Steele, Lea and Flood, 2014) started from the
    state `seed`: state_k = seed + (k + 1) * golden (mod 2^64), mixed by the variant-13
    finaliser (shifts 30, 27, 31; multipliers 0xBF58476D1CE4E5B9, 0x94D049BB133111EB).
    Counter-based: each output depends only on seed and k."""
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) % (1 << 64)) + (k + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def counter_coefficients(g2_basis: np.ndarray, n_orb: int, seed: int) -> np.ndarray:
    """The start coefficients the library generates when it is given no orbitals
    (pt_seeded_coefficients), shape (n_orb, n_basis), complex128: coefficient m of band b
    is (g1 + i g2) exp(-|G_m|^2 / 4), (g1, g2) the Box-Muller normals of the uniforms
    u1 = U(2j), u2 = U(2j + 1), j = b n_basis + m, U(k) = ((x_k >> 11) + 1/2) 2^-53 from
    SplitMix64 output x_k. Rows are not orthonormal."""
    g2 = np.asarray(g2_basis, dtype=np.float64)
    j = np.arange(int(n_orb) * g2.size, dtype=np.uint64)
    u = lambda x: ((x >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    u1, u2 = u(splitmix64(seed, 2 * j)), u(splitmix64(seed, 2 * j + np.uint64(1)))
    r, t = np.sqrt(-2.0 * np.log(u1)), 2.0 * np.pi * u2
    z = (r * np.cos(t) + 1j * r * np.sin(t)).reshape(int(n_orb), g2.size)
    return z * np.exp(-g2 / 4.0)[None, :]


def batched_kicks(count: int, seed: int = 1) -> np.ndarray:
    """Kick vectors for a batch of trajectories: axis uniform over x/y/z, size U[0.005, 0.02]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    axes = rng.integers(0, 3, size=count)
    mags = rng.uniform(0.005, 0.02, size=count)
    k = np.zeros((count, 3))
    k[np.arange(count), axes] = mags
    return k


def gaussian_vectors(shape, seed: int) -> np.ndarray:
    """Plain complex standard-normal array (for operator tests on arbitrary vectors)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    z = rng.standard_normal(tuple(shape) + (2,))
    return z[..., 0] + 1j * z[..., 1]


def basis_g2(flat_index: np.ndarray, n, cell) -> np.ndarray:
    """|G|^2 of grid frequencies given by row-major flat indices (input-envelope helper)."""
    flat = np.asarray(flat_index, dtype=np.int64)
    idx = np.unravel_index(flat, tuple(int(v) for v in n))
    out = np.zeros(flat.shape, dtype=np.float64)
    for k in range(3):
        nk = int(n[k])
        m = np.where(idx[k] < (nk + 1) // 2, idx[k], idx[k] - nk)
        g = 2.0 * np.pi * m / float(cell[k])
        out += g * g
    return out


def request_stream(count: int, rate_per_s: float, seed: int = 2, workloads=("si8", "si64", "si216"),
                   steps=(5, 50)) -> list:
    """A Poisson stream of propagation requests: exponential inter-arrival times of mean
    1 / rate_per_s seconds, workload uniform over ``workloads``, step count uniform over
    the integers steps[0]..steps[1], orbital seed = request index. Returns dictionaries
    with keys rid, arrival_s, workload, steps, seed."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    gaps = rng.exponential(1.0 / float(rate_per_s), size=count)
    arrival = np.cumsum(gaps) - gaps[0]          # the first request arrives at t = 0
    kinds = rng.integers(0, len(workloads), size=count)
    nsteps = rng.integers(int(steps[0]), int(steps[1]) + 1, size=count)
    return [dict(rid=k, arrival_s=float(arrival[k]), workload=workloads[int(kinds[k])], steps=int(nsteps[k]), seed=k)
            for k in range(count)]
