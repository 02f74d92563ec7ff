"""Mixed precision against the FP64 oracle over a 20-step trajectory (the accuracy target).

Target: the mixed-precision path keeps the dipole within 1e-6 a.u. and the total
energy within 1e-6 Ha per atom of the FP64 result over 20 PT-CN steps. The
reference is the FP64 oracle's Si8 trajectory (tests/golden/, written by
make_si8_trajectory.py, which calls only oracle/): 40 relaxation steps from the
seed-0 start orbitals, then 20 steps of dt = 2.07 a.u. (50 as) with ACE built once
per step (Eq. 5, Alg. 1). Both sides iterate the SCF to a density change of 1e-9,
far below the paper's 1e-6 (Sec. 4): at 1e-6 the stopping point of the fixed-point
iteration alone moves the dipole by ~2e-5 a.u. in FP64, so the comparison would
measure the tolerance, not the arithmetic. The mixed path runs its pair FFTs in
FP32 and its ACE and projection products on the tensor cores (3xTF32); its SCF
iterations run in FP32 until the density change falls below 1e-7 and in FP64 after
(iterative refinement, scf_fp64_below), since the FP32 iteration stalls near 1e-8.
"""
import json
import os

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
GOLDEN = os.path.join(HERE, "golden", "si8_ace_tol1e-09_trajectory.json")


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


def test_mixed_trajectory_within_target_of_fp64_oracle(pkg):
    ref = json.load(open(GOLDEN))
    assert ref["steps"] == 20 and all(ref["converged"])
    w = syn.si_workload("si8", precision="mixed", fock_mode="ace", scf_tol=ref["scf_tol"], scf_max=400)
    assert w["scf_fp64_below"] > ref["scf_tol"]
    g2 = syn.basis_g2(pkg.pt_basis_indices(pkg.make_params(w)), w["n"], w["cell"])
    s = pkg.System(w, syn.initial_coefficients(g2, w["n_orb"], seed=ref["seed"]))
    n_atoms = ref["n_atoms"]
    e0, d0 = s.observables()
    de = [abs(e0 - ref["energy"][0]) / n_atoms]
    dd = [float(np.max(np.abs(np.asarray(d0) - ref["dipole"][0])))]
    for k in range(ref["steps"]):
        st, info = s.step()
        assert info["converged"], k
        de.append(abs(info["energy"] - ref["energy"][k + 1]) / n_atoms)
        dd.append(float(np.max(np.abs(info["dipole"] - np.asarray(ref["dipole"][k + 1])))))
    s.close()
    print(f"mixed vs FP64 oracle over 20 steps: max |dE|/atom {max(de):.2e} Ha, max |d dipole| {max(dd):.2e} a.u.")
    assert max(de) <= 1e-6, de
    assert max(dd) <= 1e-6, dd
