"""Host-side accounting of bench.py, checked against independent counts.

The roofline's algorithmic bytes per pair are (4 f + 4 / T) N sizeof(complex):
four passes over the live fraction f of the pair intermediate plus orbital and
W traffic amortised over a T x T pair tile. The live fraction is the share of
axis-2 frequency slabs a pair product can reach (|m2| <= 2 max |m2| of the
basis sphere); here it is counted from the cutoff and the cell edge directly,
not from the basis listing bench.py reads.
"""
import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import synthetic as syn  # noqa: E402
from oracle.discretization import Grid  # noqa: E402


@pytest.mark.parametrize("name", ["si8", "si64", "si216"])
def test_live_fraction_from_cutoff(name):
    w = syn.si_workload(name)
    g = Grid(w["n"], w["cell"], w["ecut"])
    n2, a2 = w["n"][2], w["cell"][2]
    m2_max = math.floor(math.sqrt(2.0 * w["ecut"]) * a2 / (2.0 * math.pi))
    slabs = 4 * m2_max + 1
    expect = 1.0 if slabs >= n2 else slabs / n2
    assert bench.live_fraction(g.basis, w["n"]) == pytest.approx(expect, rel=0, abs=1e-15)


def test_si216_live_slabs_and_pair_bytes():
    w = syn.si_workload("si216")
    g = Grid(w["n"], w["cell"], w["ecut"])
    f = bench.live_fraction(g.basis, w["n"])
    assert f * 96 == pytest.approx(85)
    b = bench.pair_pipeline_bytes(w["n"], mixed=True, tile=4, live=f)
    assert b == pytest.approx((4 * 85 / 96 + 1) * 96 ** 3 * 8)
    assert 32.0e6 < b < 32.2e6
    assert bench.pair_pipeline_bytes(w["n"], mixed=False) == pytest.approx(5 * 96 ** 3 * 16)


def test_pairs_per_step_and_config():
    assert bench.pairs_per_exchange(432) == 93528
    cfg = bench.workload_config("si216", "mixed", 1)
    assert cfg["pairs_per_step"] == 93528 and cfg["grid"] == [96, 96, 96] and cfg["n_orb"] == 432
    assert "L2" in cfg["l2"]
    assert bench.workload_config("si216", "mixed", 2, fock_grid=48)["fock_grid"] == [48, 48, 48]
