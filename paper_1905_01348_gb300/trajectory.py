"""Propagate one workload and log every step as a JSON line; checkpoint to disk.

Each PT-CN step (Eq. 5, Alg. 1) through the C ABI writes one line with the
step index, the time (a.u. and fs), total energy, dipole, SCF iterations,
whether the SCF met its tolerance, the final residual norm and density change,
the wall time of the step and the pair solves per second it reached. With
`--checkpoint PATH` the state (orbitals Psi_n, their exchange W_n and the step
index n; see pt_get_state) is written to PATH (.npz) every `--checkpoint-every`
steps and at the end; `--resume PATH` starts from such a file instead of the
seeded start orbitals, and the run continues exactly where it stopped.

    python -m paper_1905_01348_gb300.trajectory --workload si8 --steps 20 --out si8.jsonl
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

FS_AU = 41.341374575751   # atomic units of time per femtosecond


def save_checkpoint(path: str, psi: np.ndarray, w: np.ndarray, step: int) -> None:
    """Write a state taken by pt_get_state (written to a temporary name, then renamed)."""
    import os
    tmp = path + ".tmp.npz"
    np.savez(tmp, psi=psi, w=w, step=np.int64(step))
    os.replace(tmp, path)


def load_checkpoint(path: str):
    with np.load(path) as d:
        return (np.ascontiguousarray(d["psi"], dtype=np.complex128), np.ascontiguousarray(d["w"], dtype=np.complex128),
                int(d["step"]))


def step_record(step: int, info: dict, dt: float, wall_s: float, pairs: int) -> dict:
    """One log line for the state after step `step` (index of the new state)."""
    return {"step": step, "time_au": step * dt, "time_fs": step * dt / FS_AU, "energy": float(info["energy"]),
            "dipole": [float(v) for v in info["dipole"]], "scf_iters": int(info["scf_iters"]),
            "converged": bool(info["converged"]), "resid_norm": float(info["resid_norm"]),
            "drho": float(info["drho"]), "wall_ms": wall_s * 1e3,
            "pair_solves_per_s": pairs / wall_s if wall_s > 0 else None}


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="si8", choices=["si8", "si64", "si216"])
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fock-mode", default="ace", choices=["ace", "exact"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--laser-amp", type=float, default=0.0, help="A0 of the laser pulse (a.u.); 0: kick only")
    ap.add_argument("--out", default="-", help="JSONL file ('-': standard output)")
    ap.add_argument("--checkpoint", default="")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default="")
    args = ap.parse_args(argv)

    import synthetic as syn
    from . import _native as nat
    from . import System, make_params

    nat.load()
    w = syn.si_workload(args.workload, precision=args.precision, fock_mode=args.fock_mode, laser_amp=args.laser_amp)
    p = make_params(w)
    g2 = syn.basis_g2(nat.pt_basis_indices(p), w["n"], w["cell"])
    c0 = syn.initial_coefficients(g2, w["n_orb"], seed=args.seed)
    pairs = w["n_orb"] * (w["n_orb"] + 1) // 2
    s = System(w, c0)
    step = 0
    if args.resume:
        psi, wx, step = load_checkpoint(args.resume)
        s.set_state(psi, wx, step)
    out = sys.stdout if args.out == "-" else open(args.out, "a" if args.resume else "w")
    try:
        for _ in range(args.steps):
            t0 = time.perf_counter()
            _, info = s.step()
            step += 1
            out.write(json.dumps(step_record(step, info, w["dt"], time.perf_counter() - t0, pairs)) + "\n")
            out.flush()
            if args.checkpoint and args.checkpoint_every > 0 and step % args.checkpoint_every == 0:
                save_checkpoint(args.checkpoint, *s.get_state())
        if args.checkpoint:
            save_checkpoint(args.checkpoint, *s.get_state())
    finally:
        if out is not sys.stdout:
            out.close()
        s.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
