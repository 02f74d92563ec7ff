"""Autotuner of the batched pair pipeline: picks, per workload, the pair-tile edge and
the launch-group size (tiles per launch) of a batch's merged pair kernels by measuring
them, and keeps the choice in tuning.json next to this module.

For each candidate shape it builds a batch of `--systems` systems of the workload
(seeded random orbitals, no relaxation: the pair pipeline's cost does not depend on
the orbital values), runs `--warmup` batched exchanges, then times `--repeats` of
them with the library's CUDA events around the merged pair kernels (pt_batch_*_timing,
graph replays on the batch stream), and records unordered pair solves per second.
Candidates: pair_tile in {2, 3, 4} (orbitals per tile edge: the FP32 cubic kernels
have a fused path for full 4 x 4 tiles) and tiles_per_launch in {whole merged round,
1/2, 1/4, 1/8 of it}. Every launch goes through the C ABI; nothing here computes.

    python -m paper_1905_01348_gb300.autotune --workload si8 --systems 12 --write
"""
from __future__ import annotations

import argparse
import json
import os

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = os.path.join(HERE, "tuning.json")


def candidates(n_orb_max: int, nsys: int):
    """(pair_tile, tiles_per_launch) shapes to measure; tiles_per_launch 0 = whole merged rounds."""
    out = []
    for tile in [t for t in (4, 3, 2) if t <= n_orb_max] or [max(1, n_orb_max)]:
        full = nsys * ((n_orb_max + tile - 1) // tile)          # tiles of the largest merged round
        tpls = sorted({0} | {max(1, full // d) for d in (2, 4, 8)})
        out += [(tile, t) for t in tpls]
    return out


def measure(workload: str, precision: str, nsys: int, tile: int, tpl: int, warmup: int, repeats: int) -> dict:
    import torch
    import synthetic as syn
    from . import _native as nat
    from .system import Batch, System

    systems = []
    for k in range(nsys):
        w = syn.si_workload(workload, precision=precision, relax_iters=0, fock_mode="ace", pair_tile=tile)
        g2 = syn.basis_g2(nat.pt_basis_indices(nat.make_params(w)), w["n"], w["cell"])
        systems.append(System(w, syn.initial_coefficients(g2, w["n_orb"], seed=k), stream=torch.cuda.Stream()))
    b = Batch(systems, pair_tile=tile, tiles_per_launch=tpl)
    for _ in range(warmup):
        b.exchange()
    nat.pt_batch_set_timing(b.handle, True)
    nat.pt_batch_get_timing(b.handle, reset=True)
    for _ in range(repeats):
        b.exchange()
    ms, pairs, groups = nat.pt_batch_get_timing(b.handle, reset=True)
    b.close()
    for s in systems:
        s.close()
    torch.cuda.empty_cache()
    return {"pair_tile": tile, "tiles_per_launch": tpl, "pair_ms": ms / repeats,
            "pairs_per_s": pairs / (ms / 1e3) if ms > 0 else None, "launch_groups": groups // repeats}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="si8", choices=["si8", "si64", "si216"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--systems", type=int, default=12)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--write", action="store_true", help="store the best shape in tuning.json")
    args = ap.parse_args(argv)

    import synthetic as syn
    from . import _native as nat
    nat.load()
    n_orb = syn.si_workload(args.workload)["n_orb"]
    rows = [measure(args.workload, args.precision, args.systems, t, tpl, args.warmup, args.repeats)
            for t, tpl in candidates(n_orb, args.systems)]
    best = max(rows, key=lambda r: r["pairs_per_s"] or 0.0)
    entry = {"systems": args.systems, "best": {"pair_tile": best["pair_tile"],
                                               "tiles_per_launch": best["tiles_per_launch"]},
             "measured": rows}
    if args.write:
        table = {}
        if os.path.exists(TABLE):
            with open(TABLE) as f:
                table = json.load(f)
        table[f"{args.workload}-{args.precision}"] = entry
        with open(TABLE + ".tmp", "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(TABLE + ".tmp", TABLE)
    print(json.dumps({"workload": args.workload, "precision": args.precision, **entry}))


if __name__ == "__main__":
    main()
