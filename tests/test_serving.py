"""The serving loop's host logic on the CPU, with stand-in systems.

Checked: admission in arrival order by footprint and free slots (never over the
budget, never more than max_active at once), requests that arrive while others
run are admitted as soon as memory frees up, oversized and failing requests are
reported without stopping the others, and every request gets its own results
back whatever the mix (a stand-in that steps an oracle model per request). The
continuous-batching server is checked the same way with a stand-in batch that
steps its members in order: requests of one workload share ticks, a request that
arrives while a batch runs joins it at a later tick, groups of different
workloads are batched apart, and a failing batch reports every member.
"""
import os
import threading
import time

import numpy as np
import pytest

import synthetic as syn
from paper_1905_01348_gb300.serve import BatchedServer, Request, Server, percentile, summarize


class SleepSystem:
    """step() sleeps; tracks how many systems are open at once."""
    lock = threading.Lock()
    open_now = 0
    open_peak = 0

    def __init__(self, req, slot, step_s=0.01, fail_at=None):
        self.req, self.k, self.step_s, self.fail_at = req, 0, step_s, fail_at
        with SleepSystem.lock:
            SleepSystem.open_now += 1
            SleepSystem.open_peak = max(SleepSystem.open_peak, SleepSystem.open_now)

    def step(self):
        time.sleep(self.step_s)
        self.k += 1
        if self.fail_at is not None and self.k == self.fail_at:
            raise RuntimeError("planted failure")
        return 0, {"energy": float(self.req.rid * 100 + self.k), "dipole": [0.0, 0.0, float(self.k)], "scf_iters": 3}

    def orbitals(self):
        return np.full(4, self.req.rid, dtype=complex)

    def close(self):
        with SleepSystem.lock:
            SleepSystem.open_now -= 1


def reset_counts():
    SleepSystem.open_now = 0
    SleepSystem.open_peak = 0


def test_admission_by_footprint_and_slots():
    reset_counts()
    sizes = {0: 40, 1: 40, 2: 40, 3: 30, 4: 10}
    steps = {0: 4, 1: 10, 2: 4, 3: 4, 4: 4}
    reqs = [Request(k, "si8", steps[k], 0.0) for k in range(5)]
    srv = Server(lambda r: sizes[r.rid], lambda r, s: SleepSystem(r, s), budget_bytes=100, max_active=3)
    outs = srv.run(reqs)
    assert all(o.error is None and len(o.step_ms) == steps[o.rid] for o in outs)
    assert srv.peak_bytes <= 100 and srv.peak_active <= 3 and SleepSystem.open_peak <= 3
    by = {o.rid: o for o in outs}
    # 0 and 1 start at once; 2 must wait for memory, and 3, 4 queue behind it (arrival order)
    assert by[0].admitted_s < 0.05 and by[1].admitted_s < 0.05
    assert by[2].admitted_s >= min(by[0].finished_s, by[1].finished_s) - 1e-6
    assert by[3].admitted_s >= by[2].admitted_s and by[4].admitted_s >= by[3].admitted_s
    # 2 was admitted when 0 finished, while 1 was still running: continuous admission
    assert by[2].admitted_s >= by[0].finished_s and by[2].admitted_s < by[1].finished_s
    assert [o.slot for o in outs[:2]] == [0, 1]


def test_arrivals_are_respected_and_overlap():
    reset_counts()
    reqs = [Request(0, "si8", 12, 0.0), Request(1, "si8", 2, 0.03), Request(2, "si8", 2, 0.06)]
    srv = Server(lambda r: 1, lambda r, s: SleepSystem(r, s), budget_bytes=10, max_active=4)
    outs = srv.run(reqs)
    for r, o in zip(reqs, outs):
        assert o.admitted_s >= r.arrival_s - 1e-9
    # request 1 arrives while request 0 is running and starts immediately
    assert outs[1].admitted_s < outs[0].finished_s
    assert outs[1].admitted_s - reqs[1].arrival_s < 0.05
    assert SleepSystem.open_peak >= 2


def test_oversized_and_failing_requests_are_reported():
    reset_counts()
    sizes = {0: 500, 1: 10, 2: 10}
    reqs = [Request(k, "si8", 3, 0.0) for k in range(3)]

    def open_system(r, s):
        return SleepSystem(r, s, fail_at=2 if r.rid == 2 else None)

    srv = Server(lambda r: sizes[r.rid], open_system, budget_bytes=100, max_active=2)
    outs = srv.run(reqs)
    assert "exceeds the budget" in outs[0].error and outs[0].admitted_s is None
    assert outs[1].error is None and len(outs[1].step_ms) == 3
    assert "planted failure" in outs[2].error and len(outs[2].step_ms) == 1
    assert SleepSystem.open_now == 0          # every opened system was closed
    s = summarize(outs, srv.wall_s, syn.DT_50AS, lambda wl: 136)
    assert s["completed"] == 1 and set(s["errors"]) == {0, 2} and s["steps"] == 4


def test_percentile_and_summary():
    assert percentile([], 0.5) is None
    assert percentile([3.0, 1.0, 2.0], 0.5) == 2.0
    assert percentile(list(range(1, 101)), 0.99) == 99
    assert percentile(list(range(1, 101)), 1.0) == 100
    reset_counts()
    reqs = [Request(k, "si8", 5, 0.0) for k in range(2)]
    srv = Server(lambda r: 1, lambda r, s: SleepSystem(r, s, step_s=0.002), 10, 2)
    outs = srv.run(reqs)
    s = summarize(outs, srv.wall_s, syn.DT_50AS, lambda wl: 136)
    assert s["steps"] == 10 and s["completed"] == 2
    assert s["pair_solves_per_s"] == pytest.approx(10 * 136 / srv.wall_s)
    assert s["fs_per_day"] == pytest.approx(10 * syn.DT_50AS / 41.341374575751 / srv.wall_s * 86400)


def test_request_stream():
    a = syn.request_stream(4000, 4.0, seed=2)
    assert a == syn.request_stream(4000, 4.0, seed=2)
    t = np.array([d["arrival_s"] for d in a])
    assert t[0] == 0.0 and np.all(np.diff(t) >= 0)
    assert np.mean(np.diff(t)) == pytest.approx(0.25, rel=0.05)
    kinds = [d["workload"] for d in a]
    for k in ("si8", "si64", "si216"):
        assert kinds.count(k) / len(kinds) == pytest.approx(1 / 3, abs=0.03)
    steps = np.array([d["steps"] for d in a])
    assert steps.min() == 5 and steps.max() == 50


class OracleSystem:
    """A stand-in that steps an oracle model (FP64 NumPy) for one request."""

    def __init__(self, req, slot):
        import oracle.ptcn as pc
        cell, frac = syn.diamond_supercell(1)
        p = pc.Params(n=(12, 12, 12), cell=tuple(cell), ecut=1.5, atoms=frac, n_orb=3, relax_iters=0,
                      scf_tol=1e-10, scf_max=100, kick=tuple(req.kick), fock_mode="exact")
        self.m = pc.Model(p)
        self.st = self.m.init_state(syn.initial_coefficients(self.m.grid.g2_basis(), 3, seed=req.seed))

    def step(self):
        self.st, info = self.m.step(self.st)
        return 0, {"energy": self.st.energy, "dipole": list(self.st.dipole), "scf_iters": info.scf_iters}

    def orbitals(self):
        return self.st.Psi.copy()

    def close(self):
        pass


def test_results_are_the_same_alone_and_in_the_mix():
    kicks = syn.batched_kicks(4, seed=1)
    reqs = [Request(k, "si8", 2 + k % 2, 0.01 * k, seed=k, kick=tuple(kicks[k])) for k in range(4)]
    mix = Server(lambda r: 1, OracleSystem, budget_bytes=3, max_active=3, keep_orbitals=True).run(reqs)
    for r, o in zip(reqs, mix):
        (a,) = Server(lambda r: 1, OracleSystem, budget_bytes=3, max_active=1, keep_orbitals=True).run([r])
        assert o.error is None and a.error is None
        assert len(o.energy) == r.steps
        assert np.array_equal(a.orbitals, o.orbitals) and a.energy == o.energy
    # different requests really differ (the comparison above is not vacuous)
    assert not np.allclose(mix[0].orbitals, mix[1].orbitals)


def test_cuda_backend_glue_and_cli_on_host(monkeypatch, capsys):
    """The CUDA backend's glue and the command line, with torch's stream calls and the
    System class replaced by host stand-ins (pt_workspace_size and the basis listing are
    host-only calls of the real library)."""
    import contextlib
    import json
    import torch
    import paper_1905_01348_gb300 as pkg
    import paper_1905_01348_gb300.system as system_mod
    from paper_1905_01348_gb300 import build as b
    from paper_1905_01348_gb300 import serve
    if not os.path.exists(pkg._native.LIB_PATH):
        b.build()

    class FakeStream:
        def __init__(self, device=None, priority=0):
            self.cuda_stream = 0
            self.priority = priority
            self.synced = 0

        def synchronize(self):
            self.synced += 1

    class FakeWorkspace:
        def __init__(self, offset, nbytes):
            self.offset, self.nbytes = offset, nbytes

    arenas = []

    class HostArena(serve.DeviceArena):
        """The arena's bookkeeping with host stand-ins for its device views."""
        def __init__(self, nbytes, device=None, large=1 << 30):
            super().__init__(nbytes, None, large)
            arenas.append(self)

        def view(self, offset, nbytes):
            return FakeWorkspace(offset, nbytes)

    made = []

    class FakeSystem:
        def __init__(self, params, psi0, device="cuda:0", stream=None, workspace=None):
            assert isinstance(stream, FakeStream) and device == "cuda:0"
            assert psi0.shape[0] == params["n_orb"]
            self.params, self.psi0, self.k, self.stream, self.workspace = params, psi0, 0, stream, workspace
            made.append(self)

        def step(self):
            self.k += 1
            return 0, {"energy": -1.0 * self.k, "dipole": np.zeros(3), "scf_iters": 1}

        def orbitals(self):
            return self.psi0

        def close(self):
            pass

    batches = []

    class FakeBatch:
        def __init__(self, systems, pair_tile=0, tiles_per_launch=0, priority=0, workspace=None):
            self.systems, self.priority, self.workspace = systems, priority, workspace
            self.stream = FakeStream()
            batches.append(self)

        @staticmethod
        def workspace_size(systems, pair_tile=0, tiles_per_launch=0):
            return 4096 * len(systems)

        def step(self):
            return 0, [x.step()[1] for x in self.systems]

        def close(self):
            pass

    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "set_device", lambda d: None)
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(system_mod, "System", FakeSystem)
    monkeypatch.setattr(system_mod, "Batch", FakeBatch)
    monkeypatch.setattr(serve, "DeviceArena", HostArena)
    monkeypatch.delenv("CUDA_DEVICE_MAX_CONNECTIONS", raising=False)   # main() sets it; restored afterwards
    monkeypatch.setattr(torch.cuda, "mem_get_info", lambda *a: (2000 << 30, 2000 << 30))

    serve.main(["--batched", "--budget-gb", "1000", "--max-active", "4", "--check-alone"])
    res = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert res["mode"] == "batched" and res["requests"] == 24 and res["completed"] == 24
    assert res["steps"] == 24 * 20 and res["peak_active"] <= 4
    assert res["alone_vs_mix"] == {"max_orbital_diff": 0.0, "max_energy_diff_ha": 0.0}
    kicks = syn.batched_kicks(24, seed=1)
    firsts = made[:24]
    assert sorted(tuple(s.params["kick"]) for s in firsts) == sorted(tuple(k) for k in kicks)
    assert sum(s.params["n_orb"] == 16 for s in firsts) == 12
    assert all(s.params["precision"] == "mixed" and s.params["fock_mode"] == "ace" for s in firsts)
    # the small workloads (batched) run on high-priority streams, their batches too
    assert all(s.stream.priority == -1 for s in firsts)
    assert batches and all(bt.priority == -1 for bt in batches)
    # every workspace came from the run's arena, and all of it was returned (each after its
    # stream was synchronised)
    assert res["workspaces"] == "device arena"
    assert all(isinstance(s.workspace, FakeWorkspace) for s in firsts)
    assert all(isinstance(bt.workspace, FakeWorkspace) for bt in batches)
    assert arenas[0].in_use() == 0 and arenas[0].free_ranges == [(0, arenas[0].size)]
    assert all(s.stream.synced >= 1 for s in firsts) and all(bt.stream.synced >= 1 for bt in batches)

    assert res["scheduling"] == "continuous batching" and res["peak_batch"] >= 2

    made.clear()
    serve.main(["--requests", "5", "--rate", "50", "--steps-max", "6", "--workloads", "si8,si64",
                "--budget-gb", "1000"])
    res = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert res["mode"] == "poisson" and res["completed"] == 5 and res["step_latency_ms"]["p99"] is not None
    serve.main(["--requests", "3", "--rate", "50", "--steps-max", "6", "--budget-gb", "1000", "--per-request"])
    res = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert res["scheduling"] == "per-request" and res["completed"] == 3
    assert all(len(r["slowest_step"]) == 3 for r in res["per_request"])


class SeqBatch:
    """Stand-in for a pt_batch: steps its member systems in order; records its members."""
    made = []

    def __init__(self, systems, fail=False):
        self.systems = list(systems)
        self.fail = fail
        SeqBatch.made.append(tuple(x.req.rid for x in self.systems if hasattr(x, "req")))

    def step(self):
        if self.fail:
            raise RuntimeError("planted batch failure")
        out = [x.step() for x in self.systems]
        return 0, [info for _, info in out]

    def close(self):
        pass


def test_batched_server_joins_and_groups():
    reset_counts()
    SeqBatch.made.clear()
    reqs = [Request(0, "si8", 12, 0.0), Request(1, "si8", 3, 0.0), Request(2, "si64", 4, 0.0),
            Request(3, "si8", 3, 0.05)]
    srv = BatchedServer(lambda r: 1, lambda r, s: SleepSystem(r, s), SeqBatch, budget_bytes=10, max_active=4)
    outs = srv.run(reqs)
    assert all(o.error is None and len(o.step_ms) == r.steps for r, o in zip(reqs, outs))
    assert SleepSystem.open_now == 0 and srv.peak_active <= 4
    groups = {frozenset(m) for m in SeqBatch.made}
    # si8 and si64 requests are never in one batch; 0 and 1 step together; 3 joins 0 later
    assert all(not ({0, 1, 3} & g and 2 in g) for g in groups)
    assert any({0, 1} <= g for g in groups) and any({0, 3} <= g for g in groups)
    assert outs[3].admitted_s < outs[0].finished_s
    assert srv.peak_batch >= 2 and srv.ticks >= 12
    # every member of a tick sees that tick's latency: request 1's ticks all carried request 0
    assert set(outs[1].step_ms) <= set(outs[0].step_ms)


def test_batched_server_budget_and_failure():
    reset_counts()
    sizes = {0: 60, 1: 60, 2: 30}
    reqs = [Request(k, "si8", 3, 0.0) for k in range(3)]
    srv = BatchedServer(lambda r: sizes[r.rid], lambda r, s: SleepSystem(r, s), SeqBatch, budget_bytes=100,
                        max_active=3)
    outs = srv.run(reqs)
    assert srv.peak_bytes <= 100 and all(o.error is None for o in outs)
    assert outs[1].admitted_s >= outs[0].finished_s - 1e-6      # 1 waits for memory
    reset_counts()
    failing = BatchedServer(lambda r: 1, lambda r, s: SleepSystem(r, s), lambda xs: SeqBatch(xs, fail=True),
                            budget_bytes=10, max_active=2)
    outs = failing.run([Request(k, "si8", 2, 0.0) for k in range(2)])
    assert all("planted batch failure" in o.error for o in outs) and SleepSystem.open_now == 0


def test_batched_results_are_the_same_alone_and_in_the_mix():
    kicks = syn.batched_kicks(4, seed=1)
    reqs = [Request(k, "si8", 2 + k % 2, 0.01 * k, seed=k, kick=tuple(kicks[k])) for k in range(4)]
    mix = BatchedServer(lambda r: 1, OracleSystem, SeqBatch, budget_bytes=3, max_active=3,
                        keep_orbitals=True).run(reqs)
    for r, o in zip(reqs, mix):
        (a,) = Server(lambda r: 1, OracleSystem, budget_bytes=3, max_active=1, keep_orbitals=True).run([r])
        assert o.error is None and a.error is None
        assert np.array_equal(a.orbitals, o.orbitals) and a.energy == o.energy


def test_batched_server_reserves_batch_memory():
    reset_counts()
    # two groups; each group's batch holds 30 bytes while it runs: the si64 request must
    # wait for the si8 group to finish (40 + 30 + 40 + 30 > 100)
    reqs = [Request(0, "si8", 4, 0.0), Request(1, "si64", 2, 0.0)]
    srv = BatchedServer(lambda r: 40, lambda r, s: SleepSystem(r, s), SeqBatch, budget_bytes=100, max_active=4,
                        group_reserve=lambda key: 30)
    outs = srv.run(reqs)
    assert all(o.error is None for o in outs)
    assert srv.peak_bytes <= 100
    assert outs[1].admitted_s >= outs[0].finished_s - 1e-6


def test_batch_policy_of_the_cuda_backend():
    import paper_1905_01348_gb300.serve as serve
    assert serve.batch_group(Request(0, "si8", 1)) == "si8"
    assert serve.batch_group(Request(1, "si64", 1)) == "si64"
    assert serve.batch_group(Request(2, "si216", 1)) == ("si216", 2)       # fills the GPU alone
    assert serve.stream_priority("si8") == serve.stream_priority("si64") == -1
    assert serve.stream_priority("si216") == 0
    shape = serve.batch_shape("si216", "mixed")
    assert shape["tiles_per_launch"] * 16 * 96 ** 3 * 8 <= serve.BATCH_X_BYTES
    assert serve.batch_reserve("si8") > 0 and serve.batch_reserve(("si216", 2)) <= serve.BATCH_X_BYTES + (64 << 20)


def test_device_arena_placement_and_coalescing():
    """The serving arena's bookkeeping: 256-byte alignment, large blocks from the top and
    small ones from the bottom, no overlap, None when nothing fits, and released ranges
    coalescing back into one."""
    import random
    from paper_1905_01348_gb300.serve import DeviceArena
    a = DeviceArena(10_000 + 100, large=2000)
    assert a.size == 9984                   # rounded down to 256-byte units
    small = a.alloc(1)                      # rounds up to 256, bottom
    big = a.alloc(3000)                     # 3072, top
    assert small == 0 and big == a.size - 3072 and big % 256 == 0
    assert a.alloc(a.size) is None          # no room for the whole arena any more
    small2 = a.alloc(300)                   # 512, next to the first small block
    assert small2 == 256
    a.release(small)
    assert a.alloc(256) == 0                # the hole is reused first
    for off in (0, small2, big):
        a.release(off)
    assert a.in_use() == 0 and a.free_ranges == [(0, a.size)]
    # random alloc / release: blocks never overlap and everything returns
    rng = random.Random(0)
    b = DeviceArena(1 << 20, large=1 << 16)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off = rng.choice(sorted(live))
            b.release(off)
            del live[off]
        else:
            n = rng.choice([100, 5000, 70_000, 200_000])
            off = b.alloc(n)
            if off is not None:
                assert off % 256 == 0 and off + n <= b.size
                for o, m in live.items():
                    assert off + n <= o or o + m <= off
                live[off] = n
    for off in list(live):
        b.release(off)
    assert b.free_ranges == [(0, b.size)]


def test_arena_block_is_released_once():
    """A workspace wrapper closed twice (explicitly, then again from __del__ after the arena
    has given the same offset to the next workspace) returns its block only once."""
    from paper_1905_01348_gb300 import serve

    class Stream:
        def __init__(self):
            self.synced = 0

        def synchronize(self):
            self.synced += 1

    class Obj:
        def __init__(self):
            self.closed = 0

        def close(self):
            self.closed += 1

    arena = serve.DeviceArena(1 << 20, large=1 << 30)
    a, sa = Obj(), Stream()
    off_a = arena.alloc(4096)
    serve._release_on_close(a, arena, off_a, sa)
    a.close()
    off_b = arena.alloc(4096)              # the freed range is handed out again
    assert off_b == off_a
    a.close()                              # the late second close must not free b's block
    assert arena.in_use() == 4096 and sa.synced == 1 and a.closed == 2
    b = Obj()
    serve._release_on_close(b, arena, off_b, Stream())
    b.close()
    assert arena.in_use() == 0


def test_command_line_asks_for_all_hardware_queues(monkeypatch):
    """The server's streams must not share hardware queues: main() sets
    CUDA_DEVICE_MAX_CONNECTIONS before anything initialises CUDA, keeping a value the
    environment already gives."""
    from paper_1905_01348_gb300 import serve
    monkeypatch.delenv("CUDA_DEVICE_MAX_CONNECTIONS", raising=False)
    serve.use_all_hw_queues()
    import os
    assert os.environ["CUDA_DEVICE_MAX_CONNECTIONS"] == str(serve.HW_QUEUES) == "32"
    assert 2 * 8 + 8 <= serve.HW_QUEUES          # slot streams of both priorities + batches
    monkeypatch.setenv("CUDA_DEVICE_MAX_CONNECTIONS", "4")
    serve.use_all_hw_queues()
    assert os.environ["CUDA_DEVICE_MAX_CONNECTIONS"] == "4"


def test_arena_slack_keeps_admitted_blocks_placeable():
    """Near full use, holes between small blocks can stop a placement the byte budget admits
    (a 3.2 GB workspace freed between 4 GB batch blocks leaves a hole no batch fits); the
    arena's slack of two of the largest small blocks removes that, within the free memory."""
    from paper_1905_01348_gb300 import serve
    G = 1 << 30
    small, sys64 = 4 * G, 3276 << 20              # 256-byte multiples
    budget = 2 * (small + sys64) + sys64          # filled exactly below

    def fill(arena):
        # [Si64][batch][Si64][batch][Si64] up to the budget, then every Si64 block leaves:
        # 8 GB in use, three separate 3.2 GB holes
        s64 = [arena.alloc(sys64)]
        for _ in range(2):
            arena.alloc(small)
            s64.append(arena.alloc(sys64))
        for o in s64:
            arena.release(o)
        return 2 * small

    tight = serve.DeviceArena(budget, large=8 * G)
    used = fill(tight)
    assert used + small <= budget and tight.alloc(small) is None       # admitted, not placeable
    roomy = serve.DeviceArena(serve.arena_bytes(budget, [small, sys64], free_bytes=100 * G), large=8 * G)
    fill(roomy)
    assert roomy.alloc(small) is not None
    assert serve.arena_bytes(budget, [small], free_bytes=21 * G) == int(0.97 * 21 * G)   # capped by free memory
