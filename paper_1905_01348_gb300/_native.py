"""ctypes binding of the C ABI in include/pt.h (argument marshalling only).

Every function here has the name of the C entry point it calls. All compute
happens in libptfock.so; when that library is missing this module raises
instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libptfock.so")

PT_OK, PT_ERR_INVALID, PT_ERR_OOM, PT_ERR_CUDA, PT_ERR_NOT_CONVERGED, PT_ERR_NOT_PD, PT_ERR_TIMEOUT = range(7)
PT_FP64, PT_MIXED = 0, 1
PT_FOCK_EXACT, PT_FOCK_ACE, PT_FOCK_NONE = 0, 1, 2
STATUS_NAMES = {0: "PT_OK", 1: "PT_ERR_INVALID", 2: "PT_ERR_OOM", 3: "PT_ERR_CUDA", 4: "PT_ERR_NOT_CONVERGED",
                5: "PT_ERR_NOT_PD", 6: "PT_ERR_TIMEOUT"}


class PtParams(C.Structure):
    _fields_ = [
        ("n", C.c_int * 3),
        ("cell", C.c_double * 3),
        ("ecut", C.c_double),
        ("n_orb", C.c_int),
        ("n_atoms", C.c_int),
        ("atom_frac", C.POINTER(C.c_double)),
        ("well_depth", C.c_double),
        ("well_sigma", C.c_double),
        ("omega", C.c_double),
        ("alpha", C.c_double),
        ("dt", C.c_double),
        ("kick", C.c_double * 3),
        ("anderson_dim", C.c_int),
        ("anderson_beta", C.c_double),
        ("scf_tol", C.c_double),
        ("scf_max", C.c_int),
        ("scf_fixed_iters", C.c_int),
        ("precision", C.c_int),
        ("fock_mode", C.c_int),
        ("use_hartree", C.c_int),
        ("use_lda", C.c_int),
        ("relax_iters", C.c_int),
        ("relax_tau", C.c_double),
        ("relax_mix", C.c_double),
        ("relax_q0", C.c_double),
        ("pair_tile", C.c_int),
        ("pair_tiles_per_launch", C.c_int),
        ("laser_amp", C.c_double),
        ("laser_omega", C.c_double),
        ("laser_duration", C.c_double),
        ("laser_dir", C.c_double * 3),
        ("n_fock", C.c_int * 3),
        ("scf_fp64_below", C.c_double),
        ("ace_outer", C.c_int),
        ("seed", C.c_uint64),
    ]


class PtStepInfo(C.Structure):
    _fields_ = [
        ("scf_iters", C.c_int),
        ("converged", C.c_int),
        ("resid_norm", C.c_double),
        ("drho", C.c_double),
        ("energy", C.c_double),
        ("dipole", C.c_double * 3),
        ("time", C.c_double),
    ]

    def as_dict(self) -> dict:
        return dict(scf_iters=self.scf_iters, converged=bool(self.converged), resid_norm=self.resid_norm,
                    drho=self.drho, energy=self.energy, dipole=np.array(self.dipole[:]), time=self.time)


class PtError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


_lib = None


def load() -> C.CDLL:
    """Load libptfock.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1905_01348_gb300.build.build()")
    lib = C.CDLL(LIB_PATH)
    P = C.POINTER(PtParams)
    vp = C.c_void_p
    sig = {
        "pt_basis_size": (C.c_int, [P, C.POINTER(C.c_int)]),
        "pt_basis_indices": (C.c_int, [P, C.POINTER(C.c_int64)]),
        "pt_seeded_coefficients": (C.c_int, [P, C.POINTER(C.c_double)]),
        "pt_workspace_size": (C.c_int, [P, C.POINTER(C.c_size_t)]),
        "pt_init_system": (C.c_int, [P, C.POINTER(C.c_double), vp, C.c_size_t, vp, C.POINTER(vp)]),
        "pt_build_ace": (C.c_int, [vp]),
        "pt_apply_h": (C.c_int, [vp, vp, vp, C.c_int, C.c_int]),
        "pt_exchange": (C.c_int, [vp, vp]),
        "pt_cn_step": (C.c_int, [vp, C.POINTER(PtStepInfo)]),
        "pt_rk4_step": (C.c_int, [vp, C.POINTER(PtStepInfo)]),
        "pt_propagate": (C.c_int, [vp, C.c_int, C.POINTER(PtStepInfo)]),
        "pt_get_orbitals": (C.c_int, [vp, C.POINTER(C.c_double)]),
        "pt_set_orbitals": (C.c_int, [vp, C.POINTER(C.c_double)]),
        "pt_get_state": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
        "pt_set_state": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_int64]),
        "pt_observables": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "pt_orbitals_device": (C.c_int, [vp, C.POINTER(vp)]),
        "pt_set_timing": (C.c_int, [vp, C.c_int]),
        "pt_get_timing": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.c_int]),
        "pt_launch_count": (C.c_int, [C.POINTER(C.c_uint64)]),
        "pt_exchange_static": (C.c_int, [P, vp, vp, vp]),
        "pt_complex_product": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), vp,
                                         C.c_int64, vp, C.c_int64, C.POINTER(C.c_double), vp, C.c_int64, C.c_int,
                                         vp, C.c_size_t, vp]),
        "pt_batch_workspace_size": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.c_int, C.POINTER(C.c_size_t)]),
        "pt_batch_create": (C.c_int, [C.POINTER(vp), C.c_int, C.c_int, C.c_int, vp, C.c_size_t, vp, C.POINTER(vp)]),
        "pt_batch_exchange": (C.c_int, [vp, C.POINTER(vp)]),
        "pt_batch_step": (C.c_int, [vp, C.POINTER(PtStepInfo)]),
        "pt_batch_set_timing": (C.c_int, [vp, C.c_int]),
        "pt_batch_get_timing": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                                          C.c_int]),
        "pt_batch_destroy": (C.c_int, [vp]),
        "pt_destroy": (C.c_int, [vp]),
        "pt_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(st: int, handle=None, allow=()):
    if st != PT_OK and st not in allow:
        raise PtError(st, pt_last_error(handle))
    return st


def make_params(d: dict) -> PtParams:
    """pt_params from a workload dictionary (keys as in synthetic.si_workload)."""
    p = PtParams()
    for k in range(3):
        p.n[k] = int(d["n"][k])
        p.cell[k] = float(d["cell"][k])
        p.kick[k] = float(d.get("kick", (0.0, 0.0, 0.0))[k])
    p.ecut = float(d["ecut"])
    p.n_orb = int(d["n_orb"])
    atoms = np.ascontiguousarray(np.asarray(d.get("atoms", np.zeros((0, 3))), dtype=np.float64).reshape(-1, 3))
    p.n_atoms = atoms.shape[0]
    p._atoms_keepalive = atoms
    p.atom_frac = atoms.ctypes.data_as(C.POINTER(C.c_double)) if atoms.size else None
    p.well_depth = float(d.get("well_depth", 2.0))
    p.well_sigma = float(d.get("well_sigma", 1.2))
    p.omega = float(d.get("omega", 0.106))
    p.alpha = float(d.get("alpha", 0.25))
    p.dt = float(d.get("dt", 2.07))
    p.anderson_dim = int(d.get("anderson_dim", 20))
    p.anderson_beta = float(d.get("anderson_beta", 1.0))
    p.scf_tol = float(d.get("scf_tol", 1e-6))
    p.scf_max = int(d.get("scf_max", 50))
    p.scf_fixed_iters = int(d.get("scf_fixed_iters", 0))
    prec = d.get("precision", "fp64")
    p.precision = PT_MIXED if prec in ("mixed", PT_MIXED) else PT_FP64
    fm = d.get("fock_mode", "ace")
    p.fock_mode = {"exact": PT_FOCK_EXACT, "ace": PT_FOCK_ACE}.get(fm, fm)
    p.use_hartree = int(bool(d.get("use_hartree", True)))
    p.use_lda = int(bool(d.get("use_lda", True)))
    p.relax_iters = int(d.get("relax_iters", 40))
    p.relax_tau = float(d.get("relax_tau", 1.0))
    p.relax_mix = float(d.get("relax_mix", 0.5))
    p.relax_q0 = float(d.get("relax_q0", 1.0))
    p.pair_tile = int(d.get("pair_tile", 0))
    p.pair_tiles_per_launch = int(d.get("pair_tiles_per_launch", 0))
    p.laser_amp = float(d.get("laser_amp", 0.0))
    p.laser_omega = float(d.get("laser_omega", 0.1199))
    p.laser_duration = float(d.get("laser_duration", 1240.4))
    ld = d.get("laser_dir", (1.0, 0.0, 0.0))
    for k in range(3):
        p.laser_dir[k] = float(ld[k])
    p.scf_fp64_below = float(d.get("scf_fp64_below", 0.0))
    p.ace_outer = int(d.get("ace_outer", 0))
    p.seed = int(d.get("seed", 0))
    nf = d.get("fock_grid") or (0, 0, 0)
    for k in range(3):
        p.n_fock[k] = int(nf[k])
    return p


def pt_last_error(handle=None) -> str:
    msg = load().pt_last_error(handle)
    return msg.decode() if msg else ""


def pt_basis_size(params: PtParams) -> int:
    n = C.c_int(0)
    _check(load().pt_basis_size(C.byref(params), C.byref(n)))
    return n.value


def pt_basis_indices(params: PtParams) -> np.ndarray:
    out = np.zeros(pt_basis_size(params), dtype=np.int64)
    _check(load().pt_basis_indices(C.byref(params), out.ctypes.data_as(C.POINTER(C.c_int64))))
    return out


def pt_seeded_coefficients(params: PtParams) -> np.ndarray:
    """The start coefficients pt_init_system generates from params.seed, (n_orb, npw) complex128."""
    out = np.zeros((params.n_orb, pt_basis_size(params)), dtype=np.complex128)
    _check(load().pt_seeded_coefficients(C.byref(params), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def pt_workspace_size(params: PtParams) -> int:
    n = C.c_size_t(0)
    _check(load().pt_workspace_size(C.byref(params), C.byref(n)))
    return n.value


def pt_init_system(params: PtParams, psi0, d_workspace: int, workspace_bytes: int, stream: int = 0):
    """psi0: (n_orb, npw) complex128 start coefficients, or None for those of params.seed."""
    if psi0 is None:
        ptr = C.POINTER(C.c_double)()
    else:
        psi0 = np.ascontiguousarray(psi0, dtype=np.complex128)
        ptr = psi0.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    _check(load().pt_init_system(C.byref(params), ptr, C.c_void_p(d_workspace), C.c_size_t(workspace_bytes),
                                 C.c_void_p(stream), C.byref(h)))
    return h


def pt_build_ace(h) -> None:
    _check(load().pt_build_ace(h), h)


def pt_apply_h(h, d_X: int, d_Y: int, ncols: int, fock_mode: int) -> None:
    _check(load().pt_apply_h(h, C.c_void_p(d_X), C.c_void_p(d_Y), int(ncols), int(fock_mode)), h)


def pt_exchange(h, d_W: int) -> None:
    _check(load().pt_exchange(h, C.c_void_p(d_W)), h)


def pt_cn_step(h) -> tuple[int, dict]:
    info = PtStepInfo()
    st = _check(load().pt_cn_step(h, C.byref(info)), h, allow=(PT_ERR_NOT_CONVERGED,))
    return st, info.as_dict()


def pt_rk4_step(h) -> dict:
    info = PtStepInfo()
    _check(load().pt_rk4_step(h, C.byref(info)), h)
    return info.as_dict()


def pt_propagate(h, nsteps: int) -> tuple[int, list]:
    infos = (PtStepInfo * max(1, nsteps))()
    st = _check(load().pt_propagate(h, int(nsteps), infos), h, allow=(PT_ERR_NOT_CONVERGED,))
    return st, [infos[k].as_dict() for k in range(nsteps)]


def pt_get_orbitals(h, n_orb: int, npw: int) -> np.ndarray:
    out = np.zeros((n_orb, npw), dtype=np.complex128)
    _check(load().pt_get_orbitals(h, out.ctypes.data_as(C.POINTER(C.c_double))), h)
    return out


def pt_set_orbitals(h, psi: np.ndarray) -> None:
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    _check(load().pt_set_orbitals(h, psi.ctypes.data_as(C.POINTER(C.c_double))), h)


def _host_c128(a: np.ndarray, shape, name: str) -> np.ndarray:
    if a.dtype != np.complex128 or not a.flags.c_contiguous or a.shape != tuple(shape):
        raise ValueError(f"{name}: expected a C-contiguous complex128 array of shape {tuple(shape)}")
    return a


def pt_get_state(h, psi_out: np.ndarray, w_out: np.ndarray) -> int:
    """Copy the state (Psi, W = V_X Psi) into caller-owned (n_orb, npw) complex128 arrays;
    returns the step index n of the state (time n dt)."""
    _host_c128(psi_out, w_out.shape, "psi_out")
    _host_c128(w_out, psi_out.shape, "w_out")
    step = C.c_int64(0)
    _check(load().pt_get_state(h, psi_out.ctypes.data_as(C.POINTER(C.c_double)),
                               w_out.ctypes.data_as(C.POINTER(C.c_double)), C.byref(step)), h)
    return step.value


def pt_set_state(h, psi: np.ndarray, w: np.ndarray, step: int) -> None:
    """Resume from a state taken by pt_get_state (same parameters) at step index `step`."""
    _host_c128(psi, w.shape, "psi")
    _host_c128(w, psi.shape, "w")
    _check(load().pt_set_state(h, psi.ctypes.data_as(C.POINTER(C.c_double)),
                               w.ctypes.data_as(C.POINTER(C.c_double)), C.c_int64(int(step))), h)


def pt_observables(h) -> tuple[float, np.ndarray]:
    e = C.c_double(0.0)
    d = (C.c_double * 3)()
    _check(load().pt_observables(h, C.byref(e), d), h)
    return e.value, np.array(d[:])


def pt_orbitals_device(h) -> int:
    p = C.c_void_p()
    _check(load().pt_orbitals_device(h, C.byref(p)), h)
    return p.value


def pt_set_timing(h, enable: bool) -> None:
    _check(load().pt_set_timing(h, int(bool(enable))), h)


def pt_get_timing(h, reset: bool = False) -> tuple[float, int, int]:
    ms = C.c_double(0.0)
    pairs = C.c_int64(0)
    groups = C.c_int64(0)
    _check(load().pt_get_timing(h, C.byref(ms), C.byref(pairs), C.byref(groups), int(bool(reset))), h)
    return ms.value, pairs.value, groups.value


def pt_exchange_static(params: PtParams, d_psi: int, d_w: int, stream: int = 0) -> None:
    """V_X Psi with no device allocation (scratch in a static 64 MiB device array)."""
    _check(load().pt_exchange_static(C.byref(params), C.c_void_p(d_psi), C.c_void_p(d_w), C.c_void_p(stream)))


def pt_complex_product(op_a: int, op_b: int, M: int, N: int, K: int, alpha: complex, d_A: int, lda: int, d_B: int,
                       ldb: int, beta: complex, d_C: int, ldc: int, upper_b: bool, d_ws: int, ws_bytes: int,
                       stream: int = 0) -> None:
    """C = alpha op(A) op(B) + beta C (complex64 A, B; complex128 C) on the tensor cores."""
    a = (C.c_double * 2)(complex(alpha).real, complex(alpha).imag)
    b = (C.c_double * 2)(complex(beta).real, complex(beta).imag)
    _check(load().pt_complex_product(int(op_a), int(op_b), int(M), int(N), int(K), a, C.c_void_p(d_A), int(lda),
                                     C.c_void_p(d_B), int(ldb), b, C.c_void_p(d_C), int(ldc), int(bool(upper_b)),
                                     C.c_void_p(d_ws), int(ws_bytes), C.c_void_p(stream)))


def _handles(handles):
    arr = (C.c_void_p * len(handles))()
    for k, h in enumerate(handles):
        arr[k] = h.value if isinstance(h, C.c_void_p) else h
    return arr


def pt_batch_workspace_size(handles, pair_tile: int = 0, tiles_per_launch: int = 0) -> int:
    n = C.c_size_t(0)
    _check(load().pt_batch_workspace_size(_handles(handles), len(handles), int(pair_tile), int(tiles_per_launch),
                                          C.byref(n)))
    return n.value


def pt_batch_create(handles, pair_tile: int, tiles_per_launch: int, d_ws: int, ws_bytes: int, stream: int):
    b = C.c_void_p()
    _check(load().pt_batch_create(_handles(handles), len(handles), int(pair_tile), int(tiles_per_launch),
                                  C.c_void_p(d_ws), int(ws_bytes), C.c_void_p(stream), C.byref(b)))
    return b


def pt_batch_exchange(b, d_w_ptrs) -> None:
    _check(load().pt_batch_exchange(b, _handles(d_w_ptrs)))


def pt_batch_step(b, nsys: int):
    """One PT-CN step of every system; returns (status, [info dict per system])."""
    infos = (PtStepInfo * nsys)()
    st = _check(load().pt_batch_step(b, infos), allow=(PT_ERR_NOT_CONVERGED,))
    return st, [infos[k].as_dict() for k in range(nsys)]


def pt_batch_set_timing(b, enable: bool) -> None:
    _check(load().pt_batch_set_timing(b, int(bool(enable))))


def pt_batch_get_timing(b, reset: bool = False):
    ms, pairs, groups = C.c_double(0), C.c_int64(0), C.c_int64(0)
    _check(load().pt_batch_get_timing(b, C.byref(ms), C.byref(pairs), C.byref(groups), int(bool(reset))))
    return ms.value, pairs.value, groups.value


def pt_batch_destroy(b) -> None:
    load().pt_batch_destroy(b)


def pt_launch_count() -> int:
    n = C.c_uint64(0)
    _check(load().pt_launch_count(C.byref(n)))
    return n.value


def pt_destroy(h) -> None:
    load().pt_destroy(h)
