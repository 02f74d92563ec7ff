"""Parity at the bench workload's full size (Si216: 3x3x3 cell, 96^3 grid,
432 orbitals, 93,528 pairs per exchange), in the configuration bench.py
times, on sampled outputs the oracle computes one by one.

Both sides orthonormalise the same seeded coefficients (no relaxation, which
the oracle could not afford at this size). The GPU applies the exchange to
all 432 orbitals with the pair pipeline; the oracle computes six sampled
columns V_X psi_j (every i, summed over chunks of orbitals) with dense FFTs:
the first, both sides of a pair-tile edge (orbitals 3 and 4), one from the
middle and the last two (the last tile).
Tolerances as in test_gpu_parity: 2e-5 (mixed) and 1e-10 (FP64).
"""
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import discretization as dz
from oracle import exchange as ex
from oracle import ptcn as pc

pytestmark = pytest.mark.gpu

SAMPLES = (0, 3, 4, 217, 430, 431)


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


@pytest.fixture(scope="module")
def reference():
    dz.FFT_WORKERS = max(1, len(os.sched_getaffinity(0)))
    w = syn.si_workload("si216", relax_iters=0)
    grid = dz.Grid(w["n"], w["cell"], w["ecut"])
    C0 = syn.initial_coefficients(grid.g2_basis(), w["n_orb"], seed=0)
    Psi = pc.orthonormalize(C0.T)                     # (npw, 432)
    khat = ex.screened_kernel(grid, w["omega"])
    psi_r = grid.to_real(Psi.T)                       # (432, 96, 96, 96)
    cols = {}
    for j in SAMPLES:
        acc = np.zeros(grid.n, dtype=np.complex128)
        for c0 in range(0, w["n_orb"], 48):
            acc += ex.apply_vx_real(psi_r[c0:c0 + 48], psi_r[j:j + 1], khat, w["alpha"])[0]
        cols[j] = grid.to_basis(acc)
    dz.FFT_WORKERS = 1
    return w, C0, cols


@pytest.mark.parametrize("precision,tol", [("mixed", 2e-5), ("fp64", 1e-10)])
def test_si216_exchange_sampled_columns(pkg, reference, precision, tol):
    w, C0, cols = reference
    s = pkg.System(dict(w, precision=precision, fock_mode="ace"), C0)
    W = s.exchange().cpu().numpy()
    for j in SAMPLES:
        ref = cols[j]
        assert np.max(np.abs(W[j] - ref)) < tol * np.max(np.abs(ref)), j
    s.close()
