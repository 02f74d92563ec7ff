"""pt_exchange_static, the exchange entry point that allocates no device memory.

Callers that cannot call cudaMalloc (a plug-in whose host application owns
all device memory, or code that must not allocate after start-up) use
pt_exchange_static: its scratch is a static device array inside the library.
Here it is called through the C ABI twice in a row on the orbitals of a
system built by pt_init_system, and each result is compared with
pt_exchange of that system and with the FP64 oracle's V_X Psi (Eq. 3) for the
same orbitals, to the tolerances of the parity tests; a cap on the pair tiles
per launch (pair_tiles_per_launch) must give the same result. A system too
large for the array must be refused with PT_ERR_OOM. (The test itself
allocates its input and output buffers with torch; only the entry point
under test must not allocate.)
"""
import os

import numpy as np
import pytest

import synthetic as syn
from oracle import discretization as dz
from oracle import exchange as ex

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_1905_01348_gb300 as p
    from paper_1905_01348_gb300 import build as b
    if not os.path.exists(p._native.LIB_PATH):
        b.build()
    p.load()
    return p


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("mixed", 2e-5)])
def test_static_exchange_matches_workspace_exchange(pkg, precision, tol):
    import torch
    w = syn.si_workload("si8", relax_iters=0, precision=precision)
    params = pkg.make_params(w)
    g2 = syn.basis_g2(pkg.pt_basis_indices(params), w["n"], w["cell"])
    C0 = syn.initial_coefficients(g2, w["n_orb"], seed=3)
    s = pkg.System(w, C0)
    ref = s.exchange().cpu().numpy()
    psi = s.orbitals_device()
    grid = dz.Grid(w["n"], w["cell"], w["ecut"])
    Psi = psi.cpu().numpy().T
    oracle_w = ex.apply_vx(grid, ex.screened_kernel(grid, w["omega"]), w["alpha"], Psi, Psi).T
    stream = torch.cuda.current_stream().cuda_stream
    for tpl in (0, 0, 3):
        p_call = pkg.make_params(dict(w, pair_tiles_per_launch=tpl))
        out = torch.full(psi.shape, float("nan"), dtype=torch.complex128, device=psi.device)
        pkg.pt_exchange_static(p_call, psi.data_ptr(), out.data_ptr(), stream)
        got = out.cpu().numpy()
        assert rel(got, ref) < tol
        assert rel(got, oracle_w) < tol
    s.close()


def test_static_exchange_refuses_oversized_system(pkg):
    import torch
    w = syn.si_workload("si64")
    params = pkg.make_params(w)
    npw = pkg.pt_basis_size(params)
    psi = torch.zeros((w["n_orb"], npw), dtype=torch.complex128, device="cuda:0")
    out = torch.zeros_like(psi)
    with pytest.raises(pkg.PtError) as err:
        pkg.pt_exchange_static(params, psi.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert err.value.status == pkg._native.PT_ERR_OOM
    assert "static array" in pkg.pt_last_error(None)
