"""The workload constants against the parameters the paper prints (Sec. 4).

The fixture tests/golden/paper_parameters.json holds the paper's values. The
synthetic cells use the same lattice constant, cutoff, time step, tolerance,
Anderson depth and two orbitals per atom. The paper evaluates exchange on the
wavefunction grid (15 points per cubic-cell edge), which folds pair densities;
the workloads use 32 points per edge (the density grid is 30), which is
alias-free. Both facts are checked with the oracle's grid.
"""
import json
import os

import numpy as np

import synthetic as syn
from oracle.discretization import Grid

HERE = os.path.dirname(os.path.abspath(__file__))


def load():
    with open(os.path.join(HERE, "golden", "paper_parameters.json")) as f:
        return json.load(f)


def test_workload_constants_follow_paper():
    g = load()
    assert abs(g["lattice_constant_angstrom"] * syn.BOHR_PER_ANGSTROM - syn.SI_CUBIC_CELL_BOHR) < 2e-3
    assert abs(g["dt_attoseconds"] / 24.188843265857 - syn.DT_50AS) < 5e-3
    assert syn.COMMON["ecut"] == g["ecut_hartree"]
    assert syn.COMMON["scf_tol"] == g["density_tolerance"]
    assert syn.COMMON["anderson_dim"] == g["anderson_dim"]
    assert g["largest_supercell_orbitals"] == 2 * g["largest_supercell_atoms"]
    assert int(np.prod(g["largest_supercell_cells"])) * g["atoms_per_cubic_cell"] == g["largest_supercell_atoms"]
    for name, cfg in syn.SI_CONFIGS.items():
        cell, frac = syn.diamond_supercell(cfg["reps"])
        assert len(frac) == g["atoms_per_cubic_cell"] * cfg["reps"] ** 3
        assert cfg["n_orb"] == 2 * len(frac)


def test_grid_reading():
    g = load()
    per_edge_wf = [n // c for n, c in zip(g["wavefunction_grid_largest"], g["largest_supercell_cells"])]
    per_edge_rho = [n // c for n, c in zip(g["density_grid_largest"], g["largest_supercell_cells"])]
    assert per_edge_wf == [15, 15, 15] and per_edge_rho == [30, 30, 30]
    a = syn.SI_CUBIC_CELL_BOHR
    assert not Grid((16, 16, 16), (a, a, a), g["ecut_hartree"]).alias_free()
    assert Grid((32, 32, 32), (a, a, a), g["ecut_hartree"]).alias_free()
