"""Wall time per femtosecond: PT-CN against explicit RK4 on one workload.

The paper (Sec. 5) compares PT-CN at 50 as with RK4 at 0.5 as, about the
largest step RK4's stability allows, for a 50 as simulation. This runs
`--steps` PT-CN steps at the workload's dt and `--rk4-steps` RK4 steps at
dt / 100 on the same start state (after `--warmup` steps of each), times them
with CUDA events on the system's stream, and prints one JSON object with the
wall seconds per fs of each integrator and their ratio.

    python -m paper_1905_01348_gb300.compare_rk4 --workload si216 --steps 2 --rk4-steps 2
"""
from __future__ import annotations

import argparse
import json

FS_AU = 41.341374575751   # atomic units of time per femtosecond


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="si8", choices=["si8", "si64", "si216"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fock-mode", default="ace", choices=["ace", "exact"])
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--rk4-steps", type=int, default=3)
    ap.add_argument("--rk4-ratio", type=int, default=100, help="PT-CN dt / RK4 dt")
    ap.add_argument("--warmup", type=int, default=1)
    args = ap.parse_args(argv)

    import torch
    import synthetic as syn
    from . import _native as nat
    from . import System, make_params

    nat.load()
    w = syn.si_workload(args.workload, precision=args.precision, fock_mode=args.fock_mode)
    p = make_params(w)
    g2 = syn.basis_g2(nat.pt_basis_indices(p), w["n"], w["cell"])
    C0 = syn.initial_coefficients(g2, w["n_orb"], seed=0)

    def timed(params, step_fn, nwarm, nsteps):
        s = System(params, C0)
        for _ in range(nwarm):
            step_fn(s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        for _ in range(nsteps):
            step_fn(s)
        e1.record(s.stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        s.close()
        return ms

    dt_pt = w["dt"]
    dt_rk = dt_pt / args.rk4_ratio
    ms_pt = timed(w, lambda s: s.step(), args.warmup, args.steps)
    ms_rk = timed(dict(w, dt=dt_rk), lambda s: s.rk4_step(), args.warmup, args.rk4_steps)
    s_per_fs_pt = ms_pt / 1e3 * FS_AU / dt_pt
    s_per_fs_rk = ms_rk / 1e3 * FS_AU / dt_rk
    print(json.dumps({"workload": args.workload, "precision": args.precision, "fock_mode": args.fock_mode,
                      "ptcn_dt_as": dt_pt / FS_AU * 1e3, "rk4_dt_as": dt_rk / FS_AU * 1e3,
                      "ptcn_ms_per_step": ms_pt, "rk4_ms_per_step": ms_rk,
                      "ptcn_wall_s_per_fs": s_per_fs_pt, "rk4_wall_s_per_fs": s_per_fs_rk,
                      "rk4_over_ptcn": s_per_fs_rk / s_per_fs_pt}))


if __name__ == "__main__":
    main()
