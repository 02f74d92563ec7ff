"""The accuracy tool's bookkeeping on the host, with a stand-in System (the
library's host-only calls are real; no device work)."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


class FakeSystem:
    """Energy and dipole drift by an amount set by the precision and tolerance."""

    def __init__(self, params, psi0, device="cuda:0", stream=None):
        self.p = params
        self.psi = np.array(psi0, dtype=np.complex128)
        self.k = 0
        self.eps = (1e-7 if params.get("precision") == "mixed" else 0.0) + params["scf_tol"]

    def observables(self):
        return -10.0 - self.eps * self.k, np.array([0.1, 0.2, 0.3]) + self.eps * self.k

    def step(self):
        self.k += 1
        e, d = self.observables()
        return 0, {"energy": e, "dipole": d, "scf_iters": 3}

    def orbitals(self):
        return self.psi

    def close(self):
        pass


def test_accuracy_tool_reports_every_comparison(pkg, monkeypatch, capsys):
    from paper_1905_01348_gb300 import accuracy
    monkeypatch.setattr(pkg, "System", FakeSystem)
    accuracy.main(["--workload", "si8", "--steps", "3", "--mixed-tight-tol", "1e-8"])
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    n_atoms = 8
    assert out["mixed_tight_vs_fp64_tight"]["max_energy_diff_ha_per_atom"] == pytest.approx(
        3 * (1e-7 + 1e-8 - 1e-9) / n_atoms)
    assert out["mixed_vs_fp64"]["max_dipole_diff_au"] == pytest.approx(3 * 1e-7)
    assert set(out["scf_iters"]) == {"fp64", "mixed", "fp64_tight", "mixed_tight"}
