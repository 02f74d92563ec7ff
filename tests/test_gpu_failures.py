"""Failure detection through the C ABI, without faulting the GPU.

* The kernels contain no device-side waits (no spin on a flag or barrier), so
  nothing in the library can hang a GPU; errors are detected on the host.
* Host-detected errors: unsupported sizes (PT_ERR_INVALID), a workspace that
  is too small (PT_ERR_OOM), linearly dependent orbitals whose overlap
  matrix has a non-positive Cholesky pivot (PT_ERR_NOT_PD) - after which the
  system keeps its previous state and still steps.
* An SCF iteration cap (PT_ERR_NOT_CONVERGED): the state still advances and
  matches the oracle's capped step.
* Checkpoint / resume: a state taken after a step and loaded into a fresh
  system continues the run bit for bit; an inconsistent state is refused.
"""
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import ptcn as pc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


SMALL = dict(syn.COMMON, n=(16, 16, 16), cell=(10.26,) * 3, ecut=2.0, atoms=syn.DIAMOND_SITES, n_orb=4,
             relax_iters=2, scf_fixed_iters=3)


def test_host_detected_errors(pkg):
    import torch
    bad = pkg.make_params(dict(SMALL, n=(16, 16, 20)))
    with pytest.raises(pkg.PtError) as e:
        pkg.pt_workspace_size(bad)
    assert e.value.status == pkg._native.PT_ERR_INVALID
    p = pkg.make_params(SMALL)
    npw = pkg.pt_basis_size(p)
    need = pkg.pt_workspace_size(p)
    ws = torch.empty(need // 2, dtype=torch.uint8, device="cuda:0")
    C0 = syn.gaussian_vectors((SMALL["n_orb"], npw), seed=2)
    with pytest.raises(pkg.PtError) as e:
        pkg.pt_init_system(p, C0, ws.data_ptr(), need // 2, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pkg._native.PT_ERR_OOM


def test_dependent_orbitals_are_refused_and_state_kept(pkg):
    model = pc.Model(pc.Params.from_dict(SMALL))
    C0 = syn.initial_coefficients(model.grid.g2_basis(), SMALL["n_orb"], seed=4)
    s = pkg.System(SMALL, C0)
    before = s.orbitals()
    dep = C0.copy()
    dep[1] = dep[0]                       # rank-deficient: Psi^H Psi is singular
    with pytest.raises(pkg.PtError) as e:
        s.set_orbitals(dep)
    assert e.value.status == pkg._native.PT_ERR_NOT_PD
    assert np.array_equal(s.orbitals(), before)
    status, info = s.step()
    assert status == 0 and np.isfinite(info["energy"])
    s.close()


def test_scf_cap_reports_not_converged_and_advances(pkg):
    """An SCF cap far below what the tolerance needs: the step returns
    PT_ERR_NOT_CONVERGED, still advances the state, and that state is the
    oracle's after the same capped number of iterations."""
    w = dict(SMALL, scf_fixed_iters=0, scf_max=2, scf_tol=1e-14)
    model = pc.Model(pc.Params.from_dict(w))
    C0 = syn.initial_coefficients(model.grid.g2_basis(), w["n_orb"], seed=5)
    st = model.init_state(C0)
    s = pkg.System(w, C0)
    st, info_o = model.step(st)
    status, info = s.step()
    assert status == pkg._native.PT_ERR_NOT_CONVERGED
    assert info["scf_iters"] == 2 and info_o.scf_iters == 2
    assert not info["converged"]
    Psi = s.orbitals().T
    assert np.max(np.abs(Psi - st.Psi)) / np.max(np.abs(st.Psi)) < 1e-10
    status, info = s.step()               # the system keeps stepping
    assert status == pkg._native.PT_ERR_NOT_CONVERGED and np.isfinite(info["energy"])
    s.close()


@pytest.mark.parametrize("w", [
    dict(SMALL, fock_mode="ace"),
    dict(SMALL, fock_mode="exact", precision="mixed", n=(32, 32, 32), ecut=2.0),
    dict(SMALL, fock_mode="ace", laser_amp=0.3, laser_omega=0.8, laser_duration=20.0, dt=1.0),
])
def test_checkpoint_resume_is_bitwise(pkg, w):
    """pt_get_state after one step, pt_set_state into a fresh system: the next
    step reproduces the uninterrupted run bit for bit."""
    model = pc.Model(pc.Params.from_dict(w))
    C0 = syn.initial_coefficients(model.grid.g2_basis(), w["n_orb"], seed=6)
    a = pkg.System(w, C0)
    a.step()
    a.step()
    psi1, w1, n1 = a.get_state()
    assert n1 == 2
    e1, d1 = a.observables()
    _, info_a = a.step()
    psi2 = a.orbitals()
    b = pkg.System(w, C0[::-1].copy())    # a different start state, overwritten below
    b.set_state(psi1, w1, n1)
    eb, db = b.observables()
    assert eb == e1 and np.array_equal(db, d1)
    _, info_b = b.step()
    assert np.array_equal(b.orbitals(), psi2)
    assert info_b["energy"] == info_a["energy"] and info_b["scf_iters"] == info_a["scf_iters"]
    assert info_b["time"] == info_a["time"] == 3 * w.get("dt", syn.COMMON["dt"])
    a.close()
    b.close()


def test_set_state_refuses_inconsistent_exchange(pkg):
    """W that is not the exchange of Psi (here W = +Psi, so -Psi^H W = -I) is
    refused with PT_ERR_NOT_PD; a consistent state afterwards is accepted."""
    w = dict(SMALL, fock_mode="ace")
    model = pc.Model(pc.Params.from_dict(w))
    C0 = syn.initial_coefficients(model.grid.g2_basis(), w["n_orb"], seed=7)
    s = pkg.System(w, C0)
    psi, wx, n = s.get_state()
    with pytest.raises(pkg.PtError) as e:
        s.set_state(psi, psi.copy(), n)
    assert e.value.status == pkg._native.PT_ERR_NOT_PD
    s.set_state(psi, wx, n)
    status, info = s.step()
    assert status == 0 and np.isfinite(info["energy"])
    s.close()
