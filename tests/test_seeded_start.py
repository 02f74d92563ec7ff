"""Seeded start coefficients (pt_seeded_coefficients; pt_init_system with no orbitals).

Both sides implement one published counter-based generator, SplitMix64 (Steele, Lea and
Flood, 2014), with Box-Muller normals: the library in C (its host code), the input
module `synthetic` in NumPy; neither uses the other. Pinned by the generator's published
outputs, by the normal distribution of the draws, and by the two implementations
agreeing; on the GPU, a system created without orbitals equals one given the same
coefficients.
"""
import os

import numpy as np
import pytest
from scipy.special import ndtr

import synthetic as syn


def test_splitmix64_published_outputs():
    # first outputs from the states 0 and 1234567 (the generator's published test values)
    assert [int(v) for v in syn.splitmix64(0, np.arange(3))] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [int(v) for v in syn.splitmix64(1234567, np.arange(5))] == [
        6457827717110365317, 3203168211198807973, 9817491932198370423, 4593380528125082431,
        16408922859458223821]
    # counter-based: output k does not depend on which other outputs were drawn
    k = np.array([7, 3, 100000])
    assert np.array_equal(syn.splitmix64(9, k), syn.splitmix64(9, np.arange(100001))[k])


def test_box_muller_draws_are_standard_normal():
    n = 100000
    z = syn.counter_coefficients(np.zeros(n), 1, seed=11)[0]      # envelope 1: the normals themselves
    for x in (z.real, z.imag):
        assert abs(x.mean()) < 5 / np.sqrt(n) and abs(x.var() - 1.0) < 0.02
        xs = np.sort(x)
        ks = np.max(np.abs(ndtr(xs) - (np.arange(1, n + 1) - 0.5) / n))
        assert ks < 1.63 / np.sqrt(n)                                 # Kolmogorov-Smirnov, 1% level
    assert abs(np.corrcoef(z.real, z.imag)[0, 1]) < 5 / np.sqrt(n)
    # the envelope exp(-|G|^2 / 4) multiplies column m
    g2 = np.array([0.0, 4.0, 8.0])
    c = syn.counter_coefficients(g2, 2, seed=3)
    assert np.allclose(c / syn.counter_coefficients(np.zeros(3), 2, seed=3), np.exp(-g2 / 4)[None, :], rtol=1e-15)


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


@pytest.mark.parametrize("name,seed", [("si8", 0), ("si8", 1234567), ("si64", 5)])
def test_library_generator_equals_restatement(pkg, name, seed):
    w = syn.si_workload(name, seed=seed)
    p = pkg.make_params(w)
    c_lib = pkg.pt_seeded_coefficients(p)
    g2 = syn.basis_g2(pkg.pt_basis_indices(p), w["n"], w["cell"])
    c_py = syn.counter_coefficients(g2, w["n_orb"], seed)
    assert c_lib.shape == c_py.shape == (w["n_orb"], g2.size)
    # the same integers and the same formula; libm and NumPy may differ in the last place
    assert np.max(np.abs(c_lib - c_py)) <= 1e-14 * np.max(np.abs(c_py))
    assert not np.allclose(c_lib, pkg.pt_seeded_coefficients(pkg.make_params(dict(w, seed=seed + 1))))


@pytest.mark.gpu
def test_system_without_orbitals_equals_seeded_coefficients(pkg):
    w = syn.si_workload("si8", relax_iters=0, seed=42)
    p = pkg.make_params(w)
    a = pkg.System(w, None)
    b = pkg.System(w, pkg.pt_seeded_coefficients(p))
    assert np.array_equal(a.orbitals(), b.orbitals())
    a.close()
    b.close()


def test_seeded_coefficients_null_output_is_refused(pkg):
    import ctypes
    lib = pkg.load()
    p = pkg.make_params(syn.si_workload("si8"))
    assert lib.pt_seeded_coefficients(ctypes.byref(p), None) == 1          # PT_ERR_INVALID
    assert pkg.pt_last_error(None).startswith("pt_seeded_coefficients:")
