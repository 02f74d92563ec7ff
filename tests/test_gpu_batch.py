"""Batched systems (pt_batch_*) against the same systems run alone, through the C ABI.

The pair tiles of all systems of a batch share launch groups (round r of every
system's tile tournament together), and from the second exchange on the merged
pair-kernel sequence is replayed from a CUDA graph. Each W element still receives
its tile contributions in its own system's order, so with the same pair tile a
batched system must reproduce its solo results bit for bit: the exchange of its
orbitals, and the orbitals, energies and dipoles after PT-CN steps whose SCF
iterations run interleaved with the other systems' on separate streams. The solo
paths are themselves oracle-pinned (test_gpu_parity.py). Cases: the FP32 cubic
pair kernels (Si8 cell, 32^3) with different orbital counts and kicks in one
batch, and the FP64 generic kernels on a small non-cubic grid. Systems that
cannot share launches (other cell) are refused.
"""
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


def si8(pkg, n_orb, seed, kick, precision="mixed"):
    w = syn.si_workload("si8", n_orb=n_orb, relax_iters=4, precision=precision, fock_mode="ace", pair_tile=4,
                        kick=kick)
    g2 = syn.basis_g2(pkg.pt_basis_indices(pkg.make_params(w)), w["n"], w["cell"])
    return w, syn.initial_coefficients(g2, n_orb, seed=seed)


SPECS = [(16, 0, (0.01, 0.0, 0.0)), (12, 1, (0.0, 0.02, 0.0)), (7, 2, (0.0, 0.0, 0.005))]


def make(pkg, specs, own_streams):
    import torch
    out = []
    for n_orb, seed, kick in specs:
        w, C0 = si8(pkg, n_orb, seed, kick)
        out.append(pkg.System(w, C0, stream=torch.cuda.Stream() if own_streams else None))
    return out


def test_batch_exchange_is_bitwise_solo(pkg):
    import torch
    batched = make(pkg, SPECS, own_streams=True)
    solo = make(pkg, SPECS, own_streams=False)
    b = pkg.Batch(batched, pair_tile=4)
    for rep in range(2):               # first run: direct launches; second: the captured graph
        outs = b.exchange()
        for s, o in zip(solo, outs):
            assert torch.equal(s.exchange(), o), rep
    b.close()
    for s in batched + solo:
        s.close()


@pytest.mark.parametrize("tpl", [0, 3])
def test_batch_steps_are_bitwise_solo(pkg, tpl):
    import torch
    batched = make(pkg, SPECS, own_streams=True)
    solo = make(pkg, SPECS, own_streams=False)
    b = pkg.Batch(batched, pair_tile=4, tiles_per_launch=tpl)
    for step in range(3):
        st, infos = b.step()
        for k, s in enumerate(solo):
            st_s, info_s = s.step()
            assert info_s["scf_iters"] == infos[k]["scf_iters"], (step, k)
            assert info_s["energy"] == infos[k]["energy"], (step, k)
            assert np.array_equal(info_s["dipole"], infos[k]["dipole"]), (step, k)
            assert torch.equal(s.orbitals_device(), batched[k].orbitals_device()), (step, k)
    b.close()
    for s in batched + solo:
        s.close()


def test_batch_fp64_generic_kernels(pkg):
    import torch
    base = dict(syn.COMMON, n=(12, 16, 24), cell=(6.1, 7.3, 8.8), ecut=2.5,
                atoms=np.array([[0.1, 0.2, 0.3], [0.6, 0.55, 0.9]]), relax_iters=0, omega=0.3, pair_tile=4,
                precision="fp64", fock_mode="ace")
    from oracle.discretization import Grid
    g = Grid(base["n"], base["cell"], base["ecut"])
    specs = [(6, 0), (5, 1)]
    batched, solo = [], []
    for n_orb, seed in specs:
        C0 = syn.initial_coefficients(g.g2_basis(), n_orb, seed=seed)
        w = dict(base, n_orb=n_orb)
        batched.append(pkg.System(w, C0, stream=torch.cuda.Stream()))
        solo.append(pkg.System(w, C0))
    b = pkg.Batch(batched, pair_tile=4)
    for rep in range(2):
        for s, o in zip(solo, b.exchange()):
            assert torch.equal(s.exchange(), o), rep
    st, infos = b.step()
    for k, s in enumerate(solo):
        s.step()
        assert torch.equal(s.orbitals_device(), batched[k].orbitals_device())
    b.close()
    for s in batched + solo:
        s.close()


def test_batch_refuses_incompatible_systems(pkg):
    w1, C1 = si8(pkg, 8, 0, (0.01, 0.0, 0.0))
    a = pkg.System(w1, C1)
    w2 = dict(w1, cell=(10.5, 10.26, 10.26))
    g2 = syn.basis_g2(pkg.pt_basis_indices(pkg.make_params(w2)), w2["n"], w2["cell"])
    c = pkg.System(w2, syn.initial_coefficients(g2, 8, seed=1))
    with pytest.raises(pkg.PtError) as err:
        pkg.Batch([a, c])
    assert err.value.status == pkg._native.PT_ERR_INVALID
    assert "cells differ" in pkg.pt_last_error(None)
    a.close()
    c.close()
