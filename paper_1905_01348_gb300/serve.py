"""Serving loop: PT-CN propagations admitted by device-memory footprint and run side by side.

Each request asks for `steps` PT-CN steps (Eq. 5, Alg. 1) of one workload from
seeded start orbitals. Requests are admitted in arrival order: the head of the
queue starts as soon as it has arrived, a slot is free and its workspace
(pt_workspace_size: orbitals, exchange and ACE data, Anderson history, pair
intermediates) fits in what the running requests leave of the memory budget.
An admitted request runs in its own host thread on its slot's CUDA stream, so
its kernels overlap on the device with those of every other running request;
its orbitals and exchange (ACE) state stay resident in its workspace from the
first step to the last, and its memory returns to the budget when it ends.
Requests that arrive while others run are admitted the moment a slot and
memory free up (continuous admission, not a queue drained one at a time).

The library's kernels are deterministic (no atomics; fixed reduction orders)
and distinct systems share no device state, so a request's results are the
same alone and in any mix; `--check-alone` re-runs every request by itself and
reports the largest difference.

    python -m paper_1905_01348_gb300.serve --requests 12 --rate 4 --steps-max 10

prints one JSON object: per-step latency p50 / p99 over all steps of all
requests, queueing delay, aggregate simulated fs per day and pair solves per
second, the peak number of concurrent requests and the peak admitted bytes.

Continuous batching (`BatchedServer`, the default of the command line): admitted
requests of the same workload (grid) step together as one batch (pt_batch_step):
their SCF iterations interleave on their own streams and the pair tiles of all
their exchanges share launch groups replayed from a CUDA graph. Each workload
group has a worker thread that advances its running requests one PT-CN step per
tick; a request admitted while the group runs joins at the next tick, a finished
one leaves at the end of its last tick (the batch is rebuilt when the set
changes). Groups of different workloads run side by side. Workloads whose own
exchange already fills the GPU (Si216) are not batched: each such request is a
group of its own. The pair-tile edge and launch-group size of each workload's
batches come from the autotuner's table (tuning.json), the launch-group size capped
so that a batch's pair intermediate stays within 4 GiB, which the admission budget
reserves while the group runs. `--per-request` runs every request on its own thread and stream
instead, with no shared launches.

The small workloads (those that are batched) run on high-priority streams, so their
kernels are dispatched ahead of a large request's queued step, and the process asks for
32 hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS), so that streams do not share one.
Every workspace is carved from one device arena allocated at start-up (`--no-arena`: one
PyTorch allocation per workspace instead), so nothing is allocated or freed on the device
while requests run.
"""
from __future__ import annotations

import argparse
import collections
import dataclasses
import json
import math
import os
import threading
import time

FS_AU = 41.341374575751   # atomic units of time per femtosecond

# Hardware work queues per process. CUDA multiplexes streams onto this many queues (8
# unless the environment says otherwise); two streams on one queue run in submission
# order, so a small request's kernels would wait behind a large request's queued step.
# The server uses up to 2 x max_active slot streams plus one per running batch.
HW_QUEUES = 32


def use_all_hw_queues() -> None:
    """Ask for HW_QUEUES hardware queues; effective only before CUDA is initialised in this
    process (a value already in the environment is kept)."""
    os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", str(HW_QUEUES))


@dataclasses.dataclass
class Request:
    rid: int
    workload: str                  # "si8", "si64" or "si216"
    steps: int
    arrival_s: float = 0.0         # seconds after the start of the run
    seed: int = 0                  # seed of the start orbitals
    kick: tuple = (0.01, 0.0, 0.0)
    precision: str = "mixed"


@dataclasses.dataclass
class Outcome:
    rid: int
    workload: str
    footprint: int
    arrival_s: float
    admitted_s: float | None = None
    finished_s: float | None = None
    slot: int | None = None
    step_ms: list = dataclasses.field(default_factory=list)
    step_start_s: list = dataclasses.field(default_factory=list)   # seconds after the start of the run
    energy: list = dataclasses.field(default_factory=list)
    dipole: list = dataclasses.field(default_factory=list)
    scf_iters: list = dataclasses.field(default_factory=list)
    orbitals: object = None
    error: str | None = None


class DeviceArena:
    """One device buffer from which the server carves every workspace, so that nothing is
    allocated or freed on the device while requests run. (Through PyTorch's caching
    allocator a finished request's block stays cached for its own stream; a new request on
    another stream then misses it, and near the budget the allocator frees its whole cache,
    whose frees synchronise the device and hold every other thread meanwhile.)

    Offsets are 256-byte aligned. Blocks of at least `large` bytes are placed at the
    highest-addressed free range that fits, smaller ones at the lowest (first fit from
    each end keeps the large, equal-sized workspaces from being split by small ones);
    released ranges coalesce with their neighbours. `nbytes` with device=None keeps the
    bookkeeping only (host tests)."""

    ALIGN = 256

    def __init__(self, nbytes: int, device=None, large: int = 8 << 30):
        self.size = int(nbytes) // self.ALIGN * self.ALIGN
        self.large = int(large)
        self.free_ranges = [(0, self.size)] if self.size > 0 else []   # sorted by offset
        self.used = {}                                                  # offset -> length
        self.lock = threading.Lock()
        self.buf = None
        if device is not None and self.size > 0:
            import torch
            self.buf = torch.empty(self.size, dtype=torch.uint8, device=device)

    def alloc(self, nbytes: int) -> int | None:
        """Offset of a block of at least nbytes, or None when no free range fits."""
        n = max(self.ALIGN, -(-int(nbytes) // self.ALIGN) * self.ALIGN)
        with self.lock:
            order = range(len(self.free_ranges))
            if n >= self.large:
                order = reversed(order)
            for i in order:
                off, length = self.free_ranges[i]
                if length < n:
                    continue
                at = off + length - n if n >= self.large else off
                rest = [(off, at - off)] if at > off else []
                if at + n < off + length:
                    rest.append((at + n, off + length - at - n))
                self.free_ranges[i:i + 1] = rest
                self.used[at] = n
                return at
            return None

    def release(self, offset: int) -> None:
        with self.lock:
            n = self.used.pop(offset)
            r = sorted(self.free_ranges + [(offset, n)])
            merged = []
            for off, length in r:
                if merged and merged[-1][0] + merged[-1][1] == off:
                    merged[-1] = (merged[-1][0], merged[-1][1] + length)
                else:
                    merged.append((off, length))
            self.free_ranges = merged

    def in_use(self) -> int:
        with self.lock:
            return sum(self.used.values())

    def view(self, offset: int, nbytes: int):
        """The device bytes [offset, offset + nbytes) as a uint8 tensor."""
        return self.buf[offset:offset + nbytes]


def percentile(values, q: float) -> float | None:
    """Nearest-rank percentile (q in (0, 1]) of a non-empty sequence; None when empty."""
    v = sorted(values)
    if not v:
        return None
    return v[min(len(v) - 1, max(0, math.ceil(q * len(v)) - 1))]


class Server:
    """Admits requests by footprint and runs each on its own slot (stream + host thread).

    footprint(req) -> bytes a request holds while it runs; open_system(req, slot) -> an
    object with step() -> (status, info dict with energy, dipole, scf_iters), orbitals()
    and close(). The CUDA backend is `cuda_backend`; tests may pass host-only stand-ins.
    """

    def __init__(self, footprint, open_system, budget_bytes: int, max_active: int = 8,
                 keep_orbitals: bool = False, clock=time.perf_counter):
        if max_active < 1:
            raise ValueError("max_active must be >= 1")
        self.footprint = footprint
        self.open_system = open_system
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.keep_orbitals = keep_orbitals
        self.clock = clock
        self.peak_active = 0
        self.peak_bytes = 0
        self.wall_s = 0.0

    def _work(self, req: Request, out: Outcome) -> None:
        system = None
        try:
            system = self.open_system(req, out.slot)
            for _ in range(req.steps):
                t = self.clock()
                _, info = system.step()
                out.step_ms.append((self.clock() - t) * 1e3)
                out.step_start_s.append(t - self._t0)
                out.energy.append(info["energy"])
                out.dipole.append(list(info["dipole"]))
                out.scf_iters.append(info["scf_iters"])
            if self.keep_orbitals:
                out.orbitals = system.orbitals()
        except Exception as e:   # reported per request; the other requests carry on
            out.error = f"{type(e).__name__}: {e}"
        finally:
            if system is not None:
                try:
                    system.close()
                except Exception as e:
                    out.error = out.error or f"close: {type(e).__name__}: {e}"

    def run(self, requests) -> list:
        """Serve `requests` (arrival times relative to the call); returns their outcomes
        in the order given."""
        reqs = list(requests)
        out = {r.rid: Outcome(r.rid, r.workload, int(self.footprint(r)), r.arrival_s) for r in reqs}
        pending = collections.deque(sorted(reqs, key=lambda r: (r.arrival_s, r.rid)))
        cv = threading.Condition()
        free_slots = list(range(self.max_active - 1, -1, -1))
        used = [0]
        active = [0]
        threads = []
        t0 = self._t0 = self.clock()

        def finish(req, o):
            self._work(req, o)
            with cv:
                o.finished_s = self.clock() - t0
                used[0] -= o.footprint
                active[0] -= 1
                free_slots.append(o.slot)
                cv.notify_all()

        with cv:
            while pending or active[0]:
                now = self.clock() - t0
                while pending and pending[0].arrival_s <= now and free_slots:
                    r = pending[0]
                    o = out[r.rid]
                    if o.footprint > self.budget:
                        o.error = f"footprint {o.footprint} B exceeds the budget {self.budget} B"
                        pending.popleft()
                        continue
                    if used[0] + o.footprint > self.budget:
                        break
                    pending.popleft()
                    o.slot = free_slots.pop()
                    o.admitted_s = now
                    used[0] += o.footprint
                    active[0] += 1
                    self.peak_active = max(self.peak_active, active[0])
                    self.peak_bytes = max(self.peak_bytes, used[0])
                    th = threading.Thread(target=finish, args=(r, o), daemon=True)
                    threads.append(th)
                    th.start()
                if not pending and not active[0]:
                    break
                timeout = None
                if pending and pending[0].arrival_s > now:
                    timeout = pending[0].arrival_s - now
                cv.wait(timeout=timeout)
        for th in threads:
            th.join()
        self.wall_s = self.clock() - t0
        return [out[r.rid] for r in reqs]


class BatchedServer:
    """Continuous batching: admitted requests of one group (workload) step together.

    footprint(req) and open_system(req, slot) as for Server; make_batch(systems) -> an
    object with step() -> (status, [info dict per system]) and close(); group_of(req)
    -> the group key (requests of one group must be able to share a batch);
    group_reserve(key) -> device bytes a group's batch holds while the group runs, taken
    from the budget when the group starts and returned when it ends. Systems are opened
    on their own threads (start-state relaxation can take seconds) and join their
    group's running batch at the next tick.
    """

    def __init__(self, footprint, open_system, make_batch, budget_bytes: int, max_active: int = 8,
                 keep_orbitals: bool = False, clock=time.perf_counter, group_of=lambda r: r.workload,
                 group_reserve=lambda key: 0):
        if max_active < 1:
            raise ValueError("max_active must be >= 1")
        self.footprint = footprint
        self.open_system = open_system
        self.make_batch = make_batch
        self.group_reserve = group_reserve    # bytes a group's batch holds while the group runs
        self.budget = int(budget_bytes)
        self.max_active = int(max_active)
        self.keep_orbitals = keep_orbitals
        self.clock = clock
        self.group_of = group_of
        self.peak_active = 0
        self.peak_bytes = 0
        self.peak_batch = 0
        self.ticks = 0
        self.wall_s = 0.0

    def run(self, requests) -> list:
        reqs = list(requests)
        out = {r.rid: Outcome(r.rid, r.workload, int(self.footprint(r)), r.arrival_s) for r in reqs}
        pending = collections.deque(sorted(reqs, key=lambda r: (r.arrival_s, r.rid)))
        cv = threading.Condition()
        free_slots = list(range(self.max_active - 1, -1, -1))
        used = [0]
        active = [0]
        ready = collections.defaultdict(list)       # group -> [(req, outcome, system)] opened, not yet stepping
        groups = {}                                  # group -> worker thread
        reserved = {}                                # group -> bytes held for its batch
        threads = []
        t0 = self._t0 = self.clock()

        def release(o):
            # with cv held
            o.finished_s = self.clock() - t0
            used[0] -= o.footprint
            active[0] -= 1
            free_slots.append(o.slot)
            cv.notify_all()

        def close_quietly(o, system):
            try:
                system.close()
            except Exception as e:
                o.error = o.error or f"close: {type(e).__name__}: {e}"

        def opener(req, o):
            try:
                system = self.open_system(req, o.slot)
            except Exception as e:
                o.error = f"{type(e).__name__}: {e}"
                with cv:
                    release(o)
                return
            with cv:
                ready[self.group_of(req)].append((req, o, system))
                cv.notify_all()

        def worker(key):
            running = []      # [req, outcome, system, steps done]
            batch, members = None, ()
            while True:
                with cv:
                    while not ready[key] and not running:
                        # nothing to step: wait for a request of this group, or finish when none can come
                        more = any(self.group_of(r) == key for r in pending) or any(
                            out[r.rid].admitted_s is not None and out[r.rid].finished_s is None and
                            self.group_of(r) == key for r in reqs)
                        if not more:
                            groups.pop(key, None)
                            used[0] -= reserved.pop(key, 0)
                            cv.notify_all()
                            return
                        cv.wait(timeout=0.05)
                    for req, o, system in ready[key]:
                        running.append([req, o, system, 0])
                    ready[key].clear()
                ids = tuple(id(x[2]) for x in running)
                try:
                    if ids != members:
                        if batch is not None:
                            batch.close()
                        batch = self.make_batch([x[2] for x in running])
                        members = ids
                    t = self.clock()
                    _, infos = batch.step()
                    dt_ms = (self.clock() - t) * 1e3
                except Exception as e:   # the whole group fails this tick; every member is reported
                    msg = f"{type(e).__name__}: {e}"
                    with cv:
                        for req, o, system, _ in running:
                            o.error = msg
                            close_quietly(o, system)
                            release(o)
                    running, batch, members = [], None, ()
                    continue
                keep, done = [], []
                for x, info in zip(running, infos):
                    x[1].step_ms.append(dt_ms)
                    x[1].step_start_s.append(t - t0)
                    x[1].energy.append(info["energy"])
                    x[1].dipole.append(list(info["dipole"]))
                    x[1].scf_iters.append(info["scf_iters"])
                    x[3] += 1
                    (done if x[3] >= x[0].steps else keep).append(x)
                running = keep
                finished = []
                if done:
                    # the batch refers to the finished systems: close it first, so that their
                    # device memory is free before their budget is returned
                    batch.close()
                    batch, members = None, ()
                    for req, o, system, _ in done:
                        if self.keep_orbitals:
                            o.orbitals = system.orbitals()
                        close_quietly(o, system)
                        finished.append(o)
                    done = []
                with cv:
                    self.ticks += 1
                    self.peak_batch = max(self.peak_batch, len(infos))
                    for o in finished:
                        release(o)

        with cv:
            while pending or active[0] or groups:
                now = self.clock() - t0
                while pending and pending[0].arrival_s <= now and free_slots:
                    r = pending[0]
                    o = out[r.rid]
                    key = self.group_of(r)
                    extra = 0 if key in groups else int(self.group_reserve(key))
                    if o.footprint + extra > self.budget:
                        o.error = f"footprint {o.footprint} B (+ {extra} B batch) exceeds the budget {self.budget} B"
                        pending.popleft()
                        continue
                    if used[0] + o.footprint + extra > self.budget:
                        break
                    pending.popleft()
                    o.slot = free_slots.pop()
                    o.admitted_s = now
                    used[0] += o.footprint
                    active[0] += 1
                    if r.steps < 1:
                        release(o)
                        continue
                    th = threading.Thread(target=opener, args=(r, o), daemon=True)
                    threads.append(th)
                    th.start()
                    if key not in groups:
                        reserved[key] = extra
                        used[0] += extra
                        g = threading.Thread(target=worker, args=(key,), daemon=True)
                        groups[key] = g
                        threads.append(g)
                        g.start()
                    self.peak_active = max(self.peak_active, active[0])
                    self.peak_bytes = max(self.peak_bytes, used[0])
                if not pending and not active[0] and not groups:
                    break
                timeout = 0.05
                if pending and pending[0].arrival_s > now:
                    timeout = min(timeout, pending[0].arrival_s - now)
                cv.wait(timeout=timeout)
        for th in threads:
            th.join()
        self.wall_s = self.clock() - t0
        return [out[r.rid] for r in reqs]


def summarize(outcomes, wall_s: float, dt_au: float, pairs_of) -> dict:
    """Latency and throughput of a served run. pairs_of(workload) = pair solves per step."""
    steps = [ms for o in outcomes for ms in o.step_ms]
    waits = [o.admitted_s - o.arrival_s for o in outcomes if o.admitted_s is not None]
    n_steps = len(steps)
    fs = n_steps * dt_au / FS_AU
    pairs = sum(len(o.step_ms) * pairs_of(o.workload) for o in outcomes)
    return {
        "requests": len(outcomes), "completed": sum(1 for o in outcomes if o.error is None and o.finished_s is not None),
        "errors": {o.rid: o.error for o in outcomes if o.error},
        "steps": n_steps, "wall_s": wall_s,
        "step_latency_ms": {"p50": percentile(steps, 0.50), "p99": percentile(steps, 0.99)},
        "step_latency_ms_by_workload": {
            wl: {"p50": percentile([ms for o in outcomes if o.workload == wl for ms in o.step_ms], 0.50),
                 "p99": percentile([ms for o in outcomes if o.workload == wl for ms in o.step_ms], 0.99),
                 "steps": sum(len(o.step_ms) for o in outcomes if o.workload == wl)}
            for wl in sorted({o.workload for o in outcomes})},
        "queue_wait_s": {"p50": percentile(waits, 0.50), "p99": percentile(waits, 0.99)},
        "fs_per_day": fs / wall_s * 86400.0 if wall_s > 0 else None,
        "pair_solves_per_s": pairs / wall_s if wall_s > 0 else None,
        # one line per request: arrival, admission and finish (s after the start), its
        # slowest step (index, ms, start s) and SCF iterations (median, max)
        "per_request": [
            {"rid": o.rid, "workload": o.workload, "steps": len(o.step_ms), "arrival_s": round(o.arrival_s, 3),
             "admitted_s": None if o.admitted_s is None else round(o.admitted_s, 3),
             "finished_s": None if o.finished_s is None else round(o.finished_s, 3),
             "slowest_step": (None if not o.step_ms else
                              [int(max(range(len(o.step_ms)), key=o.step_ms.__getitem__)), round(max(o.step_ms), 1),
                               round(o.step_start_s[max(range(len(o.step_ms)), key=o.step_ms.__getitem__)], 3)
                               if len(o.step_start_s) == len(o.step_ms) else None]),
             "p50_step_ms": None if not o.step_ms else round(percentile(o.step_ms, 0.5), 1),
             "scf_iters": None if not o.scf_iters else [percentile(o.scf_iters, 0.5), max(o.scf_iters)]}
            for o in sorted(outcomes, key=lambda o: o.rid)],
    }


def tuned_batch_shape(workload: str, precision: str, path: str | None = None) -> dict:
    """Pair-tile edge and launch-group size for batches of a workload, from the
    autotuner's table (tuning.json next to this module); automatic when absent."""
    import os
    if path is None:
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")
    try:
        with open(path) as f:
            best = json.load(f)[f"{workload}-{precision}"]["best"]
        return {"pair_tile": int(best["pair_tile"]), "tiles_per_launch": int(best["tiles_per_launch"])}
    except (OSError, KeyError, ValueError, TypeError):
        return {"pair_tile": 0, "tiles_per_launch": 0}


# Batching pays where one system's exchange leaves the GPU idle: workloads with fewer
# unordered pairs per exchange than this share batches, larger ones (Si216: 93,528
# pairs, which fill the GPU alone) run one system per group.
BATCH_MAX_PAIRS = 50000
# cap on a batch's pair intermediate (the launch-group size is reduced to fit)
BATCH_X_BYTES = 4 << 30


def _pair_tile_bytes(workload: str, precision: str) -> int:
    import synthetic as syn
    n = syn.si_workload(workload)["n"]
    return 16 * int(n[0]) * int(n[1]) * int(n[2]) * (8 if precision == "mixed" else 16)


def _small(workload: str) -> bool:
    import synthetic as syn
    n = syn.si_workload(workload)["n_orb"]
    return n * (n + 1) // 2 < BATCH_MAX_PAIRS


def batch_group(req) -> object:
    """Group key of a request: its workload when that workload is batched, else its own."""
    return req.workload if _small(req.workload) else (req.workload, req.rid)


def stream_priority(workload: str) -> int:
    """CUDA stream priority of a workload's systems and batches: -1 (high) for the small
    workloads, 0 for those whose exchange fills the GPU. The device dispatches the
    blocks of queued high-priority kernels before those of queued normal ones (running
    blocks finish), so a small request's dependent kernels do not wait behind the whole
    queued step of a large one (measured without priorities: Si8 steps p50 0.6 s, p99
    65 s beside Si216)."""
    return -1 if _small(workload) else 0


def batch_shape(workload: str, precision: str) -> dict:
    """Tuned shape, with the launch-group size capped so the pair intermediate fits BATCH_X_BYTES."""
    shape = tuned_batch_shape(workload, precision)
    cap = max(1, BATCH_X_BYTES // _pair_tile_bytes(workload, precision))
    tpl = shape["tiles_per_launch"]
    shape["tiles_per_launch"] = cap if tpl == 0 else min(tpl, cap)
    return shape


def batch_reserve(key, precision: str = "mixed") -> int:
    """Bytes a group's batch holds: its capped pair intermediate plus room for the tile table."""
    workload = key if isinstance(key, str) else key[0]
    return batch_shape(workload, precision)["tiles_per_launch"] * _pair_tile_bytes(workload, precision) + (64 << 20)


def _arena_block(arena, nbytes):
    """(offset, uint8 view) of a block of the arena, or (None, None) without an arena or room."""
    off = arena.alloc(nbytes) if arena is not None else None
    return (None, None) if off is None else (off, arena.view(off, nbytes))


def _release_on_close(obj, arena, off, stream):
    """After obj.close(): wait for the work on its stream, then return its block to the arena,
    once. (close() runs again from __del__ when the object is collected, by then perhaps
    after the arena has handed the same offset to another workspace.)"""
    close = obj.close
    lock = threading.Lock()
    released = [False]

    def close_and_release():
        try:
            close()
        finally:
            with lock:
                if not released[0]:
                    released[0] = True
                    stream.synchronize()
                    arena.release(off)

    obj.close = close_and_release


def arena_bytes(budget: int, small_blocks, free_bytes: int) -> int:
    """Size of the serving arena: the admission budget plus room for two of the largest blocks
    placed from the bottom, so that holes left between small blocks (a Si64 workspace of 3.2
    GB freed between batch workspaces of 4 GB) cannot stop a placement that the byte budget
    admitted; at most 97% of the free device memory."""
    slack = 2 * max(small_blocks, default=0)
    return min(int(budget) + slack, int(0.97 * free_bytes))


def cuda_batch_factory(arena: DeviceArena | None = None):
    """make_batch(systems) for BatchedServer: a pt_batch over the systems with the tuned, capped
    shape, its workspace carved from `arena` when one is given and has room."""
    from .system import Batch

    def make_batch(systems):
        shape = batch_shape(systems[0].workload, systems[0].precision)
        kw = dict(pair_tile=shape["pair_tile"], tiles_per_launch=shape["tiles_per_launch"])
        off, ws = _arena_block(arena, Batch.workspace_size(systems, **kw))
        try:
            b = Batch(systems, priority=stream_priority(systems[0].workload), workspace=ws, **kw)
        except Exception:
            if off is not None:
                arena.release(off)
            raise
        if off is not None:
            _release_on_close(b, arena, off, b.stream)
        return b

    return make_batch


def cuda_backend(device: str = "cuda:0", max_active: int = 8, arena: DeviceArena | None = None):
    """(footprint, open_system) for the CUDA library: one torch stream per slot and priority
    (stream_priority of the request's workload), the workspace carved from `arena` (or, with
    no arena or no room in it, allocated on that stream), start orbitals from the seeded
    generator."""
    import torch
    import synthetic as syn
    from . import _native as nat
    from .system import System

    nat.load()
    dev = torch.device(device)
    streams = {pr: [torch.cuda.Stream(dev, priority=pr) for _ in range(max_active)] for pr in (-1, 0)}

    def workload(req):
        return syn.si_workload(req.workload, precision=req.precision, fock_mode="ace", kick=tuple(req.kick))

    def footprint(req):
        return nat.pt_workspace_size(nat.make_params(workload(req)))

    def open_system(req, slot):
        torch.cuda.set_device(dev)
        w = workload(req)
        p = nat.make_params(w)
        g2 = syn.basis_g2(nat.pt_basis_indices(p), w["n"], w["cell"])
        c0 = syn.initial_coefficients(g2, w["n_orb"], seed=req.seed)
        stream = streams[stream_priority(req.workload)][slot]
        off, ws = _arena_block(arena, nat.pt_workspace_size(p))
        try:
            with torch.cuda.stream(stream):
                system = System(w, c0, device=str(dev), stream=stream, workspace=ws)
        except Exception:
            if off is not None:
                stream.synchronize()
                arena.release(off)
            raise
        if off is not None:
            _release_on_close(system, arena, off, stream)
        system.workload, system.precision = req.workload, req.precision
        return system

    return footprint, open_system


def main(argv=None) -> None:
    use_all_hw_queues()
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--requests", type=int, default=12)
    ap.add_argument("--rate", type=float, default=4.0, help="mean arrivals per second (Poisson)")
    ap.add_argument("--seed", type=int, default=2)
    ap.add_argument("--workloads", default="si8,si64,si216")
    ap.add_argument("--steps-min", type=int, default=5)
    ap.add_argument("--steps-max", type=int, default=50)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--max-active", type=int, default=8)
    ap.add_argument("--budget-gb", type=float, default=0.0, help="0: 90%% of the device's free memory")
    ap.add_argument("--no-arena", dest="arena", action="store_false",
                    help="allocate each workspace through PyTorch's caching allocator instead of one arena")
    ap.add_argument("--batched", action="store_true",
                    help="12 Si8 + 12 Si64 trajectories, all at t = 0, 20 steps, kicks from seed 1")
    ap.add_argument("--check-alone", action="store_true",
                    help="re-run every request alone and report the largest difference of its results")
    ap.add_argument("--per-request", action="store_true",
                    help="every request on its own thread and stream (no batching of pair launches)")
    args = ap.parse_args(argv)

    import numpy as np
    import torch
    import synthetic as syn

    if args.batched:
        kicks = syn.batched_kicks(24, seed=1)
        reqs = [Request(k, "si8" if k < 12 else "si64", 20, 0.0, seed=k, kick=tuple(kicks[k]),
                        precision=args.precision) for k in range(24)]
    else:
        stream = syn.request_stream(args.requests, args.rate, seed=args.seed,
                                    workloads=tuple(args.workloads.split(",")), steps=(args.steps_min, args.steps_max))
        reqs = [Request(d["rid"], d["workload"], d["steps"], d["arrival_s"], seed=d["seed"], precision=args.precision)
                for d in stream]
    budget = int(args.budget_gb * 2 ** 30) if args.budget_gb > 0 else int(0.9 * torch.cuda.mem_get_info()[0])
    # the budget (plus placement slack) as one arena: every workspace is carved from it, none is
    # allocated while serving; the largest blocks placed from the bottom are the batch workspaces
    small = [batch_reserve(w, args.precision) for w in sorted({r.workload for r in reqs})]
    arena = (DeviceArena(arena_bytes(budget, small, torch.cuda.mem_get_info()[0]), device="cuda:0")
             if args.arena else None)
    footprint, open_system = cuda_backend(max_active=args.max_active, arena=arena)
    if args.per_request:
        srv = Server(footprint, open_system, budget, args.max_active, keep_orbitals=args.check_alone)
    else:
        srv = BatchedServer(footprint, open_system, cuda_batch_factory(arena), budget, args.max_active,
                            keep_orbitals=args.check_alone, group_of=batch_group,
                            group_reserve=lambda key: batch_reserve(key, args.precision))
    outs = srv.run(reqs)
    n_orb = {k: syn.si_workload(k)["n_orb"] for k in ("si8", "si64", "si216")}
    res = summarize(outs, srv.wall_s, syn.DT_50AS, lambda wl: n_orb[wl] * (n_orb[wl] + 1) // 2)
    res.update({"mode": "batched" if args.batched else "poisson", "rate_per_s": None if args.batched else args.rate,
                "precision": args.precision, "max_active": args.max_active, "budget_bytes": budget,
                "peak_active": srv.peak_active, "peak_bytes": srv.peak_bytes,
                "scheduling": "per-request" if args.per_request else "continuous batching",
                "workspaces": "device arena" if arena is not None else "caching allocator",
                **({} if args.per_request else {"peak_batch": srv.peak_batch, "ticks": srv.ticks,
                                                "batch_shape": {w: batch_shape(w, args.precision)
                                                                for w in sorted({r.workload for r in reqs})},
                                                "batched_workloads": sorted({r.workload for r in reqs
                                                                             if isinstance(batch_group(r), str)})})})
    if args.check_alone:
        alone = Server(footprint, open_system, budget, 1, keep_orbitals=True)
        worst_psi, worst_e = 0.0, 0.0
        for r, o in zip(reqs, outs):
            (a,) = alone.run([dataclasses.replace(r, arrival_s=0.0)])
            if o.error or a.error:
                continue
            worst_psi = max(worst_psi, float(np.max(np.abs(a.orbitals - o.orbitals))))
            worst_e = max(worst_e, float(np.max(np.abs(np.subtract(a.energy, o.energy)))))
        res["alone_vs_mix"] = {"max_orbital_diff": worst_psi, "max_energy_diff_ha": worst_e}
    print(json.dumps(res))


if __name__ == "__main__":
    main()
