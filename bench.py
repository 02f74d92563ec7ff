#!/usr/bin/env python3
"""Benchmark: Fock pair-FFT solves/s (and wall-s per fs) of PT-CN steps on the
Si216 workload (3x3x3 diamond supercell, a = 30.78 bohr, 432 doubly occupied
orbitals, 96^3 grid, 10 Ha cutoff, Gaussian wells, HSE-like screened exchange
w = 0.106 / bohr with mixing 0.25, ACE rebuilt once per step, dt = 50 as).

A step is one PT-CN step (Eq. 5, Alg. 1) through the C ABI: the exchange of
the new orbitals over all 93,528 unordered orbital pairs (pair product, 3D
FFT, screened-kernel multiply, inverse FFT, accumulate), the ACE build
(M = Psi^H W, Cholesky of -M, xi = W L^{-H}), and the SCF loop (local H,
ACE apply, PT residual, per-band Anderson mixing, density) to the 1e-6
density tolerance, then Cholesky orthonormalisation. value = unordered pair
solves per second over the timed steps (all ranks), inputs resident in HBM.

Multi-GPU: the path runs replicas only (independent trajectories per rank,
no data-path collective); value sums the ranks' pairs over the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Fock pair-FFT solves/s (Si216 PT-CN steps, mixed precision)"


def metric_name(workload: str, precision: str) -> str:
    """The metric string of the JSON line (the default run is METRIC)."""
    names = {"si8": "Si8", "si64": "Si64", "si216": "Si216"}
    prec = "mixed precision" if precision == "mixed" else "FP64"
    return f"Fock pair-FFT solves/s ({names[workload]} PT-CN steps, {prec})"
UNIT = "pair-solves/s"
STEPS_PER_FS = 20   # 50 as per step


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="si216", choices=["si8", "si64", "si216"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fock-grid", type=int, default=0,
                    help="edge of a cubic Fock grid for the pair FFTs (0: the workload grid, the headline)")
    ap.add_argument("--ref-sample-s", type=float, default=5.0,
                    help="host seconds of oracle work per reference-arm step")
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="timed steps of the FP64 leg (0: no FP64 leg); it starts from the mixed run's state")
    ap.add_argument("--fp64-warmup", type=int, default=1)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def pairs_per_exchange(n_orb: int) -> int:
    return n_orb * (n_orb + 1) // 2


def workload_config(workload: str, precision: str, world: int, fock_grid: int = 0) -> dict:
    """The `config` object of the JSON line (both arms report the same one)."""
    import synthetic as syn
    w = syn.si_workload(workload, precision=precision, fock_mode="ace")
    extra = {"fock_grid": [fock_grid] * 3} if fock_grid else {}
    return {"workload": workload, "grid": list(w["n"]), **extra, "n_orb": w["n_orb"],
            "pairs_per_step": pairs_per_exchange(w["n_orb"]), "fock_mode": "ace", "precision": precision,
            "scf_tol": w["scf_tol"], "dt_au": w["dt"],
            "l2": "inputs larger than L2 (orbitals and pair intermediates are GBs)",
            "parallelism": f"replicas x{world}"}


def reduce_max(x: float, device) -> float:
    """Max of a per-rank float over the process group (the timing rule: slowest rank)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank: float, world: int, t_max_s: float) -> float:
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / t_max_s


def measured_peaks() -> dict:
    """HBM GB/s and bf16 TFLOP/s measured on this machine, else the stated fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# FP64 peak of GB300: 1.25 TFLOP/s (the pool's nominal figure; a register-FMA probe of this
# library's own measured 1.19 TFLOP/s, DMMA 1.05). FP64 runs at 1/64 of the FP32 rate here.
FP64_PEAK_TFLOPS = 1.25


def pair_fft_flops(n) -> float:
    """Algorithmic FLOPs per unordered pair of the FP64 pair pipeline: one forward and
    one inverse complex 3D FFT, 5 N log2 N each (the usual radix-2 count)."""
    import math
    N = int(n[0]) * int(n[1]) * int(n[2])
    return 2.0 * 5.0 * N * math.log2(N)


def live_fraction(basis_idx, n) -> float:
    """Fraction of axis-2 frequency slabs a pair product can reach.

    Products of two basis functions reach |G2| <= 2 max|g2| over the basis;
    the other slabs are exactly zero and the FP32 cubic pair kernels skip them.
    """
    import numpy as np
    n2 = int(n[2])
    i2 = np.asarray(basis_idx) % n2
    f = np.where(i2 < (n2 + 1) // 2, i2, i2 - n2)
    reach = 2 * int(np.max(np.abs(f)))
    return 1.0 if 2 * reach + 1 >= n2 else (2 * reach + 1) / n2


def pair_pipeline_bytes(n, mixed: bool, tile: int = 4, live: float = 1.0) -> float:
    """Algorithmic HBM bytes per unordered pair of the pair pipeline.

    Four passes over the live part of the pair intermediate (F1 write, F2
    read + write, F3 read) of live * N complex values, plus orbital reads and
    W accumulation amortised over a tile of `tile` x `tile` pairs:
    (4 live + 4 / tile) * N * sizeof(complex).
    """
    N = int(n[0]) * int(n[1]) * int(n[2])
    cs = 8 if mixed else 16
    return (4.0 * live + 4.0 / tile) * N * cs


def traffic_per_launch(workload: str, precision: str):
    """DRAM bytes per launch group from the committed ncu summary, if one matches."""
    path = os.path.join(ROOT, "profiles", "fock_pair_pipeline_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return d.get(f"{workload}-{precision}")
    except Exception:
        return None


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
def cpu_oracle_pairs_per_s(workload: str, budget_s: float = 15.0, seed: int = 0) -> dict:
    """The FP64 oracle's pair loop timed on the host cores on a bounded sample.

    Sample: m target orbitals against M occupied orbitals of the workload's
    grid (random coefficients), i.e. M * m pair solves of the oracle's
    apply_vx_real (each: product, dense FFT, kernel multiply, inverse FFT,
    accumulate), repeated until the time budget is used.
    """
    import numpy as np
    import synthetic as syn
    from oracle import discretization as dz
    from oracle import exchange as ex
    cores = len(os.sched_getaffinity(0))
    dz.FFT_WORKERS = cores
    w = syn.si_workload(workload)
    grid = dz.Grid(w["n"], w["cell"], w["ecut"])
    khat = ex.screened_kernel(grid, w["omega"])
    M = min(w["n_orb"], 2 * cores)
    C = syn.initial_coefficients(grid.g2_basis(), M, seed)
    psi_r = grid.to_real(C)
    npairs = 0
    t0 = time.perf_counter()
    while True:
        ex.apply_vx_real(psi_r, psi_r[:1], khat, w["alpha"])
        npairs += M
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return {"value": npairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{npairs} pair solves ({M} orbitals x 1 target, repeated) of the FP64 oracle on the "
                      f"{'x'.join(map(str, w['n']))} grid, scipy.fft with {cores} workers, {dt:.1f} s"}


# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    res, wall = [], []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = cpu_oracle_pairs_per_s(args.workload, budget_s=args.ref_sample_s, seed=k)
        if k >= args.warmup:
            res.append(r)
            wall.append(time.perf_counter() - t0)
    value = statistics.mean(r["value"] for r in res)
    n_orb = {"si8": 16, "si64": 128, "si216": 432}[args.workload]
    # a reference step is one bounded oracle sample; ms_per_step is its measured wall time
    ms_per_step = 1e3 * sum(wall) / len(wall)
    line = {"impl": "reference", "metric": metric_name(args.workload, args.precision), "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "step_definition": "one bounded sample of the oracle's pair loop (not a PT-CN step)",
            "extrapolated_ms_per_exchange": pairs_per_exchange(n_orb) / value * 1e3,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.workload, args.precision, args.gpus, args.fock_grid),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": res[0]["cores"], "kind": "oracle",
                             "sample": res[0]["sample"]},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
def fp64_leg(args, w_mixed: dict, C0, state, dev) -> dict:
    """The FP64 GPU path on the same state: an FP64 system is created (no relaxation), given
    the mixed run's last state (Psi_n, W_n, n) through pt_set_state, stepped fp64_warmup
    times untimed and fp64_steps times between CUDA events on its stream. Its pair
    pipeline is FP64-ALU bound: the roofline is FLOPs of the pair FFTs against the FP64 peak."""
    import torch
    import paper_1905_01348_gb300 as pkg
    w = dict(w_mixed, precision="fp64", relax_iters=0)
    sysg = pkg.System(w, C0, device=str(dev))
    psi, wv, step = state
    sysg.set_state(psi, wv, step)
    stream = sysg.stream
    pkg.pt_set_timing(sysg.handle, True)
    for _ in range(args.fp64_warmup):
        sysg.step()
    pkg.pt_get_timing(sysg.handle, reset=True)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.fp64_steps + 1)]
    ev[0].record(stream)
    iters = []
    for k in range(args.fp64_steps):
        st, info = sysg.step()
        iters.append(info["scf_iters"])
        ev[k + 1].record(stream)
    torch.cuda.synchronize(dev)
    t_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(args.fp64_steps)]
    pair_ms, pair_count, groups = pkg.pt_get_timing(sysg.handle, reset=True)
    sysg.close()
    del sysg
    torch.cuda.empty_cache()
    pairs = pairs_per_exchange(w["n_orb"])
    flops_pair = pair_fft_flops(w["n"])
    achieved = flops_pair * pair_count / (pair_ms / 1e3) / 1e12 if pair_ms > 0 else None
    return {"pairs_per_s": pairs * args.fp64_steps / (t_ms / 1e3), "ms_per_step": t_ms / args.fp64_steps,
            "wall_s_per_fs": t_ms / args.fp64_steps * STEPS_PER_FS / 1e3, "steps": args.fp64_steps,
            "warmup": args.fp64_warmup, "step_ms": step_ms, "scf_iters": iters,
            "start": "the mixed run's last state through pt_set_state (same Psi_n, W_n)",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": achieved / FP64_PEAK_TFLOPS if achieved else None, "traffic": None,
                         "kernel": "FP64 pair pipeline (fock.cu pair kernels and 3D FFT passes)",
                         "alg_flops_per_pair": flops_pair, "pair_pipeline_ms": pair_ms,
                         "pairs_per_s_in_pipeline": pair_count / (pair_ms / 1e3) if pair_ms > 0 else None,
                         "peak_source": "nominal FP64 rate of GB300 (1.25 TFLOP/s)"}}


# ---------------------------------------------------------------------------
def run_gpu(args):
    import numpy as np
    import torch
    import synthetic as syn
    import paper_1905_01348_gb300 as pkg

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pkg.load()

    w = syn.si_workload(args.workload, precision=args.precision, fock_mode="ace", seed=rank)
    if args.fock_grid:
        w["fock_grid"] = (args.fock_grid,) * 3
    params = pkg.make_params(w)
    n_orb = w["n_orb"]
    g2 = syn.basis_g2(pkg.pt_basis_indices(params), w["n"], w["cell"])
    C0 = syn.initial_coefficients(g2, n_orb, seed=rank)
    pairs = pairs_per_exchange(n_orb)

    sysg = pkg.System(w, C0, device=str(dev))
    stream = sysg.stream
    pkg.pt_set_timing(sysg.handle, True)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    # warm-up
    for _ in range(args.warmup):
        sysg.step()
    pkg.pt_get_timing(sysg.handle, reset=True)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    launches0 = pkg.pt_launch_count()
    torch.cuda.nvtx.range_push("timed_steps")
    e0.record(stream)
    infos = []
    step_ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    step_ev[0].record(stream)
    for k in range(args.steps):
        st, info = sysg.step()
        infos.append(info)
        step_ev[k + 1].record(stream)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    barrier()
    launches = pkg.pt_launch_count() - launches0
    clk = clocks.stop()
    t_ms = e0.elapsed_time(e1)
    step_ms = sorted(step_ev[k].elapsed_time(step_ev[k + 1]) for k in range(args.steps))

    def pct(q):
        import math
        return step_ms[min(len(step_ms) - 1, max(0, math.ceil(q * len(step_ms)) - 1))]
    pair_ms, pair_count, groups = pkg.pt_get_timing(sysg.handle, reset=True)
    if ws > 1:
        t_ms = reduce_max(t_ms, dev)
    value = job_value(pairs * args.steps, ws, t_ms / 1e3)
    ms_per_step = t_ms / args.steps

    # roofline of the pair pipeline (F1 + F2 + F3 of every launch group)
    peaks = measured_peaks()
    mixed = args.precision == "mixed"
    nf = tuple(w.get("fock_grid") or w["n"])          # grid of the pair FFTs
    cubic_fast = mixed and nf[0] == nf[1] == nf[2] and nf[0] in (32, 48, 64, 96)
    live = 1.0
    if cubic_fast:
        # basis flat indices on the main grid -> axis-2 frequencies, then the reach on the Fock grid
        import numpy as np
        i2 = np.asarray(pkg.pt_basis_indices(params)) % w["n"][2]
        f2 = np.where(i2 < (w["n"][2] + 1) // 2, i2, i2 - w["n"][2])
        live = live_fraction(np.mod(f2, nf[2]), nf)
    alg_bytes_pair = pair_pipeline_bytes(nf, mixed, live=live)
    pair_time_s = pair_ms / 1e3
    achieved = alg_bytes_pair * pair_count / pair_time_s / 1e9 if pair_time_s > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": (achieved / peaks["hbm_gbs"]) if achieved else None,
            "traffic": traffic_per_launch(args.workload, args.precision) if not args.fock_grid else None,
            "kernel": "fock pair pipeline (k_fast_f1 + k_fast_f2 + k_fast_f3 at 96^3, FP32), one launch group = "
                      "one round of tiles",
            "launch_groups": groups, "pair_pipeline_ms": pair_ms, "alg_bytes_per_pair": alg_bytes_pair,
            "live_slab_fraction": live,
            "pairs_per_s_in_pipeline": pair_count / pair_time_s if pair_time_s > 0 else None,
            "peak_source": peaks["source"]}

    # end to end through the public API with host buffers: every step loads
    # the state (Psi_n, W_n = V_X Psi_n) from pinned host memory, steps, and
    # stores the new state back to the same host buffers (a trajectory that
    # lives on the host between steps, as in checkpointed or served runs)
    e2e = None
    if not args.no_e2e:
        psi_np, w_np, step = sysg.get_state()
        host_psi = torch.from_numpy(psi_np).pin_memory()
        host_w = torch.from_numpy(w_np).pin_memory()
        hp, hw = host_psi.numpy(), host_w.numpy()
        nbytes = 2 * host_psi.numel() * 16
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pkg.pt_set_state(sysg.handle, hp, hw, step)
            sysg.step()
            step = pkg.pt_get_state(sysg.handle, hp, hw)
        barrier()
        te = time.perf_counter() - t0
        if ws > 1:
            te = reduce_max(te, dev)
        e2e = {"value": job_value(pairs * args.steps, ws, te), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes,
               "note": "per step: pt_set_state from pinned host memory (orbitals and their exchange; rebuilds ACE "
                       "and observables), pt_cn_step, pt_get_state back to the host buffers"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_oracle_pairs_per_s(args.workload)

    fp64 = None
    if args.precision == "mixed" and args.fp64_steps > 0 and not args.fock_grid:
        state = sysg.get_state()
        sysg.close()
        del sysg
        torch.cuda.empty_cache()
        sysg = None
        fp64 = fp64_leg(args, w, C0, state, dev)

    if rank == 0:
        line = {
            "metric": metric_name(args.workload, args.precision), "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.precision == "mixed" else "f64",
            "data": "synthetic (seeded random orbitals, relaxed; Gaussian-well Si supercell)",
            "config": workload_config(args.workload, args.precision, ws, args.fock_grid),
            "wall_s_per_fs": ms_per_step * STEPS_PER_FS / 1e3,
            "step_latency_ms": {"p50": pct(0.50), "p99": pct(0.99), "n": len(step_ms)},
            "scf_iters": [i["scf_iters"] for i in infos],
            "converged": [bool(i["converged"]) for i in infos],
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk,
        }
        if fp64 is not None:
            line["fp64"] = fp64
            line["speedup_mixed_over_fp64"] = value / fp64["pairs_per_s"]
        print(json.dumps(line), flush=True)
    if sysg is not None:
        sysg.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
