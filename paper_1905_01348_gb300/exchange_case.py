"""Run one exchange application V_X Psi (Eq. 3, pair loop of Alg. 2) on a
workload's cell and grid with a chosen number of orbitals.

A small, self-contained case for kernel profilers and quick timing: it
builds a system from seeded synthetic orbitals (no start-state relaxation),
calls pt_exchange `--repeats` times on the system's stream and exits. With
`--time` it first runs `--warmup` untimed applications, then prints the
CUDA-event time of the timed ones (on the system's stream) and the library's
own pair-pipeline time. Every launch goes through the C ABI; nothing here
computes.

    python -m paper_1905_01348_gb300.exchange_case --workload si216 --n-orb 16
    python -m paper_1905_01348_gb300.exchange_case --workload si216 --n-orb 64 --time --repeats 5
"""
from __future__ import annotations

import argparse


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="si216", choices=["si8", "si64", "si216"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n-orb", type=int, default=16)
    ap.add_argument("--repeats", type=int, default=1)
    ap.add_argument("--time", action="store_true")
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--tiles-per-launch", type=int, default=0, help="cap on pair tiles per launch group (0: auto)")
    ap.add_argument("--fock-grid", type=int, default=0, help="edge of a cubic Fock grid for the pair FFTs (0: the grid)")
    args = ap.parse_args(argv)

    import torch
    import synthetic as syn
    from . import _native as nat
    from . import System, make_params

    nat.load()
    w = syn.si_workload(args.workload, precision=args.precision, relax_iters=0, n_orb=args.n_orb)
    w["pair_tiles_per_launch"] = args.tiles_per_launch
    if args.fock_grid:
        w["fock_grid"] = (args.fock_grid,) * 3
    p = make_params(w)
    g2 = syn.basis_g2(nat.pt_basis_indices(p), w["n"], w["cell"])
    C0 = syn.initial_coefficients(g2, w["n_orb"], seed=0)
    s = System(w, C0)
    out = torch.empty((w["n_orb"], s.npw), dtype=torch.complex128, device="cuda:0")
    if args.time:
        for _ in range(args.warmup):
            nat.pt_exchange(s.handle, out.data_ptr())
        nat.pt_set_timing(s.handle, 1)
        nat.pt_get_timing(s.handle, reset=True)
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(s.stream)
    for _ in range(args.repeats):
        nat.pt_exchange(s.handle, out.data_ptr())
    if args.time:
        ev1.record(s.stream)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(torch.view_as_real(out)).all())
    msg = f"exchange {args.workload} n_orb={args.n_orb} {args.precision}: ok"
    if args.time:
        ms = ev0.elapsed_time(ev1) / args.repeats
        pair_ms, pairs, groups = nat.pt_get_timing(s.handle)
        npairs = args.n_orb * (args.n_orb + 1) // 2
        msg += (f"; {ms:.3f} ms per application, {npairs / ms * 1e3:.0f} pairs/s;"
                f" pair pipeline {pair_ms / args.repeats:.3f} ms, {pairs / pair_ms * 1e3:.0f} pairs/s")
    s.close()
    print(msg)


if __name__ == "__main__":
    main()
