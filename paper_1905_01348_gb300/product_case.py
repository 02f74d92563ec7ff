"""Time the tensor-core complex products of ACE and the PT projection at a
workload's sizes (a case for kernel profilers and quick timing).

Two products of seeded complex64 operands through pt_complex_product:
  * "ahb": C = A^H B, n_orb x n_orb over the basis (M = Psi^H W, xi^H X, Psi^H H Psi);
  * "nn":  C = C - A Z, basis x n_orb over n_orb (-xi (xi^H X), H Psi - Psi S).
Each is run `--warmup` times untimed and `--repeats` times between CUDA events;
the line printed gives ms per product and TFLOP/s counted as 8 M N K (one
complex multiply-add = 8 real flops; the tensor cores do three TF32 passes of it).
Every launch goes through the C ABI; nothing here computes.

    python -m paper_1905_01348_gb300.product_case --workload si216 --time
"""
from __future__ import annotations

import argparse


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--workload", default="si216", choices=["si8", "si64", "si216"])
    ap.add_argument("--which", default="both", choices=["ahb", "nn", "both"])
    ap.add_argument("--repeats", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=2)
    ap.add_argument("--time", action="store_true")
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    import synthetic as syn
    from . import _native as nat

    nat.load()
    w = syn.si_workload(args.workload)
    p = nat.make_params(w)
    npw, ne = nat.pt_basis_size(p), w["n_orb"]
    dev = "cuda:0"
    A = torch.from_numpy(syn.gaussian_vectors((ne, npw), 1).astype(np.complex64)).to(dev)
    B = torch.from_numpy(syn.gaussian_vectors((ne, npw), 2).astype(np.complex64)).to(dev)
    Z = torch.from_numpy(syn.gaussian_vectors((ne, ne), 3).astype(np.complex64)).to(dev)
    S = torch.zeros((ne, ne), dtype=torch.complex128, device=dev)
    Y = torch.zeros((ne, npw), dtype=torch.complex128, device=dev)
    ws = torch.empty(16 * ne * ne * 16 + 256, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    cases = {
        "ahb": lambda: nat.pt_complex_product(1, 0, ne, ne, npw, 1.0, A.data_ptr(), npw, B.data_ptr(), npw, 0.0,
                                              S.data_ptr(), ne, False, ws.data_ptr(), ws.numel(), stream),
        "nn": lambda: nat.pt_complex_product(0, 0, npw, ne, ne, -1.0, A.data_ptr(), npw, Z.data_ptr(), ne, 1.0,
                                             Y.data_ptr(), npw, False, ws.data_ptr(), ws.numel(), stream),
    }
    sizes = {"ahb": (ne, ne, npw), "nn": (npw, ne, ne)}
    for name in (["ahb", "nn"] if args.which == "both" else [args.which]):
        f = cases[name]
        for _ in range(args.warmup if args.time else 0):
            f()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(args.repeats):
            f()
        ev1.record()
        torch.cuda.synchronize()
        M, N, K = sizes[name]
        msg = f"{name} {args.workload} M={M} N={N} K={K}: ok"
        if args.time:
            ms = ev0.elapsed_time(ev1) / args.repeats
            msg += f"; {ms:.3f} ms per product, {8.0 * M * N * K / ms / 1e9:.1f} TFLOP/s (8MNK)"
        print(msg)


if __name__ == "__main__":
    main()
