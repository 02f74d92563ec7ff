"""The serving loop on the GPU: requests run side by side on their own streams give the
same results as each request run alone.

Three Si8 propagations (32^3 grid, 16 orbitals, mixed precision, different kicks and
start orbitals) arrive 20 ms apart and overlap on the device; each is then re-run
alone. The kernels have no atomics and fixed reduction orders and the systems share
no device state, so orbitals and energies must agree bit for bit.
"""
import dataclasses
import os

import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


def test_mix_equals_alone(pkg):
    from paper_1905_01348_gb300.serve import Request, Server, cuda_backend
    kicks = syn.batched_kicks(3, seed=1)
    reqs = [Request(k, "si8", 3, 0.02 * k, seed=k, kick=tuple(kicks[k])) for k in range(3)]
    footprint, open_system = cuda_backend(max_active=3)
    budget = 3 * max(footprint(r) for r in reqs)
    srv = Server(footprint, open_system, budget, max_active=3, keep_orbitals=True)
    mix = srv.run(reqs)
    assert srv.peak_active >= 2 and srv.peak_bytes <= budget
    for r, o in zip(reqs, mix):
        assert o.error is None, o.error
        (a,) = Server(footprint, open_system, budget, 1, keep_orbitals=True).run([dataclasses.replace(r, arrival_s=0.0)])
        assert a.error is None, a.error
        assert len(o.energy) == 3 and np.all(np.isfinite(o.energy))
        assert np.array_equal(a.orbitals, o.orbitals)
        assert a.energy == o.energy and a.dipole == o.dipole
    assert not np.array_equal(mix[0].orbitals, mix[1].orbitals)


def test_continuous_batching_equals_alone(pkg):
    """Continuous batching: Si8 requests arriving 30 ms apart join one batch (shared pair
    launches, interleaved SCF iterations) and leave it as they finish; each must match the
    same request run alone on the per-request path, bit for bit (same pair tile, 4)."""
    from paper_1905_01348_gb300.serve import BatchedServer, Request, Server, cuda_backend
    kicks = syn.batched_kicks(3, seed=1)
    reqs = [Request(k, "si8", 2 + k, 0.03 * k, seed=k, kick=tuple(kicks[k])) for k in range(3)]
    footprint, open_system = cuda_backend(max_active=3)
    budget = 3 * max(footprint(r) for r in reqs)
    srv = BatchedServer(footprint, open_system, lambda systems: pkg.Batch(systems, pair_tile=4), budget,
                        max_active=3, keep_orbitals=True)
    mix = srv.run(reqs)
    assert srv.peak_batch >= 2
    for r, o in zip(reqs, mix):
        assert o.error is None, o.error
        (a,) = Server(footprint, open_system, budget, 1, keep_orbitals=True).run([dataclasses.replace(r, arrival_s=0.0)])
        assert a.error is None, a.error
        assert len(o.energy) == r.steps
        assert np.array_equal(a.orbitals, o.orbitals)
        assert a.energy == o.energy and a.dipole == o.dipole


def test_continuous_batching_from_an_arena_equals_alone(pkg):
    """The same continuous-batching case with every system and batch workspace carved from
    one device arena (as the command line serves): results bitwise equal to the request run
    alone, and every block back in the arena at the end."""
    from paper_1905_01348_gb300.serve import (BatchedServer, DeviceArena, Request, Server, cuda_backend,
                                              cuda_batch_factory)
    kicks = syn.batched_kicks(3, seed=1)
    reqs = [Request(k, "si8", 2 + k, 0.03 * k, seed=k, kick=tuple(kicks[k])) for k in range(3)]
    footprint, _ = cuda_backend(max_active=3)
    budget = 3 * max(footprint(r) for r in reqs) + (1 << 30)
    arena = DeviceArena(budget, device="cuda:0")
    footprint, open_system = cuda_backend(max_active=3, arena=arena)
    srv = BatchedServer(footprint, open_system, cuda_batch_factory(arena), budget, max_active=3, keep_orbitals=True)
    mix = srv.run(reqs)
    assert srv.peak_batch >= 2
    assert arena.in_use() == 0 and arena.free_ranges == [(0, arena.size)]
    for r, o in zip(reqs, mix):
        assert o.error is None, o.error
        (a,) = Server(footprint, open_system, budget, 1, keep_orbitals=True).run([dataclasses.replace(r, arrival_s=0.0)])
        assert a.error is None, a.error
        assert np.array_equal(a.orbitals, o.orbitals)
        assert a.energy == o.energy and a.dipole == o.dipole
