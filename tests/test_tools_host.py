"""The accuracy and trajectory tools' bookkeeping on the host, with stand-in
systems (the library's host-only calls are real; no device work): the accuracy
comparisons, the per-step log, and a checkpoint written mid-run and resumed,
whose log continues the uninterrupted one line for line."""
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


class FakeStateSystem:
    """Deterministic in the step index; state = (psi, w, step) as pt_get_state gives it."""

    def __init__(self, params, psi0, device="cuda:0", stream=None):
        self.psi = np.array(psi0, dtype=np.complex128)
        self.w = -0.5 * self.psi
        self.k = 0

    def step(self):
        self.k += 1
        self.psi = self.psi * np.exp(-0.01j * self.k)
        self.w = -0.5 * self.psi
        return 0, {"energy": -10.0 + 1e-3 * self.k, "dipole": np.array([self.k, 0.0, 0.0]), "scf_iters": 20 + self.k,
                   "converged": True, "resid_norm": 1e-6, "drho": 1e-7}

    def get_state(self):
        return self.psi.copy(), self.w.copy(), self.k

    def set_state(self, psi, w, step):
        self.psi, self.w, self.k = psi.copy(), w.copy(), step

    def close(self):
        pass


def test_trajectory_log_and_checkpoint_resume(pkg, monkeypatch, tmp_path):
    from paper_1905_01348_gb300 import trajectory
    monkeypatch.setattr(pkg, "System", FakeStateSystem)
    full, part, ck = tmp_path / "full.jsonl", tmp_path / "part.jsonl", tmp_path / "state.npz"
    assert trajectory.main(["--workload", "si8", "--steps", "6", "--out", str(full)]) == 0
    assert trajectory.main(["--workload", "si8", "--steps", "4", "--out", str(part), "--checkpoint", str(ck),
                            "--checkpoint-every", "2"]) == 0
    psi, w, step = trajectory.load_checkpoint(str(ck))
    assert step == 4 and np.array_equal(w, -0.5 * psi)
    assert trajectory.main(["--workload", "si8", "--steps", "2", "--out", str(part), "--resume", str(ck)]) == 0
    a = [json.loads(l) for l in full.read_text().splitlines()]
    b = [json.loads(l) for l in part.read_text().splitlines()]
    assert [r["step"] for r in b] == [1, 2, 3, 4, 5, 6]
    for ra, rb in zip(a, b):
        for key in ("step", "time_au", "energy", "dipole", "scf_iters", "converged"):
            assert ra[key] == rb[key], key
    assert a[-1]["time_fs"] == pytest.approx(6 * 2.07 / 41.341374575751)


def test_accuracy_tool_runs_and_compares_on_host(monkeypatch, capsys):
    """The accuracy tool's runs and comparisons, with a host stand-in for System whose
    energies depend on the run's parameters in a known way (the basis listing is a
    host-only call of the real library)."""
    import json
    import numpy as np
    import paper_1905_01348_gb300 as pkg
    from paper_1905_01348_gb300 import accuracy
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(pkg._native.LIB_PATH):
        b.build()
    made = []

    class FakeSystem:
        def __init__(self, params, psi0):
            self.p, self.psi0, self.k = params, psi0, 0
            # energy offset per step: exact 0, ACE 1e-3, each outer rebuild / 10; mixed + 1e-7
            off = 0.0 if params["fock_mode"] == "exact" else 1e-3 / 10 ** params.get("ace_outer", 0)
            self.off = off + (1e-7 if params["precision"] == "mixed" else 0.0)
            made.append(self)

        def observables(self):
            return -10.0, np.zeros(3)

        def step(self):
            self.k += 1
            return 0, {"energy": -10.0 + self.off * self.k, "dipole": np.full(3, self.off),
                       "scf_iters": 3}

        def orbitals(self):
            q, _ = np.linalg.qr(self.psi0.T)      # orthonormal rows, as the library returns them
            return q.T

        def close(self):
            pass

    monkeypatch.setattr(pkg, "System", FakeSystem)
    accuracy.main(["--workload", "si8", "--steps", "4", "--ace-vs-exact", "--tight-tol", "1e-10"])
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    n_atoms = 8
    assert [m.p["fock_mode"] for m in made] == ["exact", "ace", "ace", "ace", "ace"]
    assert [m.p.get("ace_outer") for m in made] == [0, 0, 1, 2, 0]
    assert made[0].p["scf_tol"] == 1e-10 and made[4].p["precision"] == "mixed"
    assert abs(out["ace_vs_exact"]["max_energy_diff_ha_per_atom"] - 4e-3 / n_atoms) < 1e-15
    assert abs(out["ace_outer2_vs_exact"]["max_energy_diff_ha_per_atom"] - 4e-5 / n_atoms) < 1e-15
    assert abs(out["mixed_ace_vs_exact"]["max_dipole_diff_au"] - (1e-3 + 1e-7)) < 1e-15
    assert abs(out["ace_vs_exact"]["subspace_defect"]) < 1e-9            # same orbitals: no defect
    made.clear()
    accuracy.main(["--workload", "si8", "--steps", "3", "--mixed-tight-tol", "1e-9"])
    out = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert [m.p["precision"] for m in made] == ["fp64", "mixed", "fp64", "mixed"]
    assert made[3].p["scf_tol"] == 1e-9 and made[3].p["scf_fp64_below"] == made[1].p["scf_fp64_below"]
    assert abs(out["mixed_vs_fp64"]["max_energy_diff_ha_per_atom"] - 3e-7 / n_atoms) < 1e-15
    assert "mixed_tight_vs_fp64_tight" in out
    assert abs(out["energy_drift_ha_per_atom"]["fp64"] - 3e-3 / n_atoms) < 1e-15   # the stand-in's ACE offset
