"""Failure detection through the C ABI, without faulting the GPU.

* Bounded device waits: the self-test makes a wait on a bulk-copy mbarrier run
  out (the copy is never issued); the call must return PT_ERR_TIMEOUT and the
  context must stay usable (an exchange afterwards still matches the oracle).
* Host-detected errors: unsupported sizes (PT_ERR_INVALID), a workspace that
  is too small (PT_ERR_OOM), linearly dependent orbitals whose overlap
  matrix has a non-positive Cholesky pivot (PT_ERR_NOT_PD) - after which the
  system keeps its previous state and still steps.
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


def test_bounded_wait_times_out_and_context_survives(pkg):
    import torch
    flag = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    st = pkg.pt_selftest_bounded_wait(flag.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == pkg._native.PT_ERR_TIMEOUT
    assert int(flag[0].item()) == 1
    assert "gave up" in pkg.pt_last_error(None)
    model = pc.Model(pc.Params.from_dict(SMALL))
    C0 = syn.initial_coefficients(model.grid.g2_basis(), SMALL["n_orb"], seed=1)
    ref = model.init_state(C0)
    s = pkg.System(SMALL, C0)
    W = s.exchange().cpu().numpy().T
    assert np.max(np.abs(W - ref.W)) < 1e-10 * np.max(np.abs(ref.W))
    s.close()


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
