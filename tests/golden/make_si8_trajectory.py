"""Write the FP64 oracle's Si8 trajectory used by the mixed-precision accuracy test.

Calls only ``oracle/`` (and the seeded inputs of ``synthetic``): the Si8 workload
(8-atom cubic diamond cell of 10.26 bohr, 16 orbitals, 32^3 grid, 10 Ha cutoff,
Gaussian wells, screened exchange w = 0.106 with mixing 0.25, velocity-gauge kick
0.01 / bohr along x, dt = 2.07 a.u. = 50 as; Sec. 4's system with the stand-ins of
the input recipe), start orbitals from seed 0 relaxed by 40 steps, then 20 PT-CN
steps (Eq. 5, Alg. 1) with ACE built once per step, at an SCF density tolerance
far below the paper's 1e-6 so that the stopping point of the iteration is not what
the test measures. Output: the energy and dipole of the start state and after each
step, and the SCF iteration counts.

    python tests/golden/make_si8_trajectory.py [--tol 1e-9] [--steps 20] [--fock-mode ace]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--fock-mode", default="ace", choices=["ace", "exact"])
    ap.add_argument("--out", default=None)
    args = ap.parse_args(argv)

    import numpy as np
    import synthetic as syn
    from oracle import ptcn as pc

    w = syn.si_workload("si8", scf_tol=args.tol, scf_max=400, fock_mode=args.fock_mode)
    m = pc.Model(pc.Params.from_dict(w))
    C0 = syn.initial_coefficients(m.grid.g2_basis(), w["n_orb"], seed=0)
    t0 = time.time()
    st = m.init_state(C0)
    energy, dipole, iters, conv = [st.energy], [list(map(float, st.dipole))], [], []
    for _ in range(args.steps):
        st, info = m.step(st)
        energy.append(float(info.energy))
        dipole.append(list(map(float, info.dipole)))
        iters.append(int(info.scf_iters))
        conv.append(bool(info.converged))
    out = {
        "what": "FP64 oracle trajectory, Si8 workload, PT-CN (Eq. 5, Alg. 1)",
        "writer": "tests/golden/make_si8_trajectory.py (calls oracle/ only)",
        "workload": "si8", "seed": 0, "relax_iters": int(m.p.relax_iters), "fock_mode": args.fock_mode,
        "scf_tol": args.tol, "dt": w["dt"], "steps": args.steps, "n_atoms": int(len(w["atoms"])),
        "energy": energy, "dipole": dipole, "scf_iters": iters, "converged": conv,
        "oracle_seconds": time.time() - t0,
    }
    path = args.out or os.path.join(HERE, f"si8_{args.fock_mode}_tol{args.tol:.0e}_trajectory.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path, out["oracle_seconds"])


if __name__ == "__main__":
    main()
