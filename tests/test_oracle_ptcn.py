"""Pins of the oracle's PT-CN step (Eq. 4, Eq. 5, Alg. 1) and its helpers.

* Eigenstates of a fixed linear H (alpha = 0, no Hartree, no LDA): the PT
  residual vanishes, so one step returns the same orbitals.
* Brute force: for a fixed linear H the density matrix P(T) = Psi Psi^H after
  T/dt steps is compared with exp(-iHT) P(0) exp(iHT) from a dense matrix
  exponential; the error falls by ~4x when dt halves (second order).
* Anderson mixing converges to the same fixed point as plain (undamped)
  iteration where the latter converges (small dt, full nonlinear H).
* The step output is orthonormal; the Cholesky helper agrees with LAPACK and
  refuses an indefinite matrix.
* Laser (velocity gauge): the vector potential's closed form; free electrons
  (single planewaves, no potential) stay fixed and their energy follows
  2 sum |G + kappa + A(t_n)|^2 / 2 exactly; with wells and the field the
  density matrix converges at second order to a fine midpoint-exponential
  reference of the time-dependent linear H.
* RK4 (Sec. 5's comparison integrator): fourth order against the matrix
  exponential for a fixed linear H; on the full nonlinear H with exact
  exchange and the laser it agrees with PT-CN up to PT-CN's O(dt^2) error.
* Energy: with the full time-independent H after the kick, the energy change
  over a fixed time falls at second order in dt.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic as syn
from oracle import ptcn as pc


def tiny_params(**kw):
    cell, frac = syn.diamond_supercell(1)
    base = dict(n=(12, 12, 12), cell=tuple(cell), ecut=1.5, atoms=frac, n_orb=3, relax_iters=0,
                scf_tol=1e-14, scf_max=300, kick=(0.01, 0.0, 0.0))
    base.update(kw)
    return pc.Params(**base)


def linear_h_matrix(m):
    g = m.grid
    eye = np.eye(g.npw, dtype=complex)
    return m.local.apply_local(m.local.v_ion, eye)


def test_eigenstates_are_stationary():
    p = tiny_params(alpha=0.0, use_hartree=False, use_lda=False)
    m = pc.Model(p)
    H = linear_h_matrix(m)
    assert np.max(np.abs(H - H.conj().T)) < 1e-12
    w, V = np.linalg.eigh(0.5 * (H + H.conj().T))
    st = m.init_state(V[:, :3].T)
    st2, info = m.step(st)
    assert info.converged
    assert np.max(np.abs(st2.Psi - st.Psi)) < 1e-11
    assert np.max(np.abs(m.density(st2.Psi) - m.density(st.Psi))) < 1e-11


def test_second_order_against_matrix_exponential():
    T = 0.8
    errs = []
    for nsteps in (2, 4, 8):
        p = tiny_params(alpha=0.0, use_hartree=False, use_lda=False, dt=T / nsteps)
        m = pc.Model(p)
        C0 = syn.initial_coefficients(m.grid.g2_basis(), 3, seed=4)
        st = m.init_state(C0)
        P0 = st.Psi @ st.Psi.conj().T
        H = linear_h_matrix(m)
        U = sla.expm(-1j * T * 0.5 * (H + H.conj().T))
        P_exact = U @ P0 @ U.conj().T
        st, infos = m.propagate(st, nsteps)
        assert all(i.converged for i in infos)
        P = st.Psi @ st.Psi.conj().T
        errs.append(np.linalg.norm(P - P_exact))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


def test_anderson_reaches_plain_fixed_point():
    outs = []
    for dim in (20, 0):        # dim 0: no history, plain x <- x - R_f(x)
        p = tiny_params(dt=0.05, anderson_dim=dim, fock_mode="exact", omega=0.3)
        m = pc.Model(p)
        C0 = syn.initial_coefficients(m.grid.g2_basis(), 3, seed=6)
        st = m.init_state(C0)
        st2, info = m.step(st)
        assert info.converged
        outs.append((st2.Psi, info.scf_iters))
    assert outs[0][1] < outs[1][1]
    assert np.max(np.abs(outs[0][0] - outs[1][0])) < 1e-10


def ace_vs_exact_one_step(dt, outer):
    """Projector and energy differences after one step: ACE (with `outer` rebuilds) vs exact."""
    out = {}
    for mode, k in (("exact", 0), ("ace", outer)):
        m = pc.Model(tiny_params(fock_mode=mode, omega=0.3, scf_tol=1e-13, scf_max=400, dt=dt, ace_outer=k))
        st = m.init_state(syn.initial_coefficients(m.grid.g2_basis(), 3, seed=7))
        st2, info = m.step(st)
        assert info.converged
        S = st2.Psi.conj().T @ st2.Psi
        assert np.max(np.abs(S - np.eye(3))) < 1e-13
        out[mode] = st2
    e, a = out["exact"], out["ace"]
    dP = np.linalg.norm(e.Psi @ e.Psi.conj().T - a.Psi @ a.Psi.conj().T)
    return dP, abs(e.energy - a.energy)


def test_ace_once_per_step_is_second_order_per_step():
    # Both modes share W = V_X Psi_n for R_n; inside the SCF, ACE built from Psi_n differs
    # from V_X[Psi_f] by O(dt), which enters the step through dt/2: O(dt^2) per step.
    d = [ace_vs_exact_one_step(dt, 0) for dt in (0.5, 0.25, 0.125)]
    for (p1, e1), (p2, e2) in zip(d, d[1:]):
        assert 3.5 < p1 / p2 < 4.5 and 3.5 < e1 / e2 < 4.5, d
    assert d[0][0] < 2.5e-3 and d[0][1] < 5e-3, d


def test_outer_ace_rebuilds_raise_the_order():
    # a rebuild from the converged Psi_f (= Psi_{n+1} + O(dt^2)) leaves an O(dt^2) operator
    # error: O(dt^3) per step; a second rebuild O(dt^4)
    d1 = [ace_vs_exact_one_step(dt, 1)[0] for dt in (0.5, 0.25, 0.125)]
    assert all(6.5 < a / b < 9.5 for a, b in zip(d1, d1[1:])), d1
    d2 = [ace_vs_exact_one_step(dt, 2)[0] for dt in (0.5, 0.25)]
    assert 12.0 < d2[0] / d2[1] < 20.0 and d2[0] < 1e-7, d2


def test_cholesky_helper():
    A = syn.gaussian_vectors((5, 5), seed=8)
    S = A.conj().T @ A + 0.1 * np.eye(5)
    L = pc.cholesky_or_none(S)
    assert np.max(np.abs(L - np.linalg.cholesky(S))) < 1e-13
    assert pc.cholesky_or_none(S - 100 * np.eye(5)) is None


# ---- laser field (velocity gauge, time-dependent kinetic term) ------------------------

def test_laser_vector_potential_values():
    p = tiny_params(laser_amp=0.3, laser_omega=0.5, laser_duration=10.0, laser_dir=(0.0, 0.6, 0.8))
    m = pc.Model(p)
    assert np.all(m.laser(0.0) == 0.0) and np.all(m.laser(10.5) == 0.0) and np.all(m.laser(-1.0) == 0.0)
    t = 2.5   # sin^2(pi / 4) = 1/2
    expect = 0.3 * 0.5 * np.sin(0.5 * t) * np.array([0.0, 0.6, 0.8])
    assert np.allclose(m.laser(t), expect, rtol=0, atol=1e-15)
    assert np.all(pc.Model(tiny_params()).laser(3.0) == 0.0)      # amplitude 0: no field


def test_free_electrons_follow_the_field():
    """No potential, no exchange: single planewaves stay eigenstates at all times, so
    PT-CN keeps them fixed and the energy is 2 sum_i |G_i + kappa + A(t_n)|^2 / 2 exactly."""
    p = tiny_params(alpha=0.0, use_hartree=False, use_lda=False, well_depth=0.0, laser_amp=0.4,
                    laser_omega=0.9, laser_duration=6.0, laser_dir=(0.6, 0.0, 0.8), dt=0.5)
    m = pc.Model(p)
    npw = m.grid.npw
    pick = [0, 5, 17]
    C0 = np.zeros((3, npw), complex)
    for r, k in enumerate(pick):
        C0[r, k] = 1.0
    st = m.init_state(C0)
    G = m.grid.gvec_basis()[pick]
    kick = np.asarray(p.kick)
    for n in range(1, 9):
        st, info = m.step(st)
        gk = G + kick[None, :] + m.laser(n * p.dt)[None, :]
        assert abs(info.energy - float(np.sum(gk * gk))) < 1e-12
        assert np.max(np.abs(np.abs(st.Psi[pick, range(3)]) - 1.0)) < 1e-12
    assert np.any(m.laser(2.0) != 0.0)


def test_laser_second_order_against_fine_exponential_integrator():
    """Linear H(t) (wells + kinetic with the field): the density matrix after T converges
    at second order in dt to a fine midpoint-exponential reference."""
    T = 1.2
    kw = dict(alpha=0.0, use_hartree=False, use_lda=False, laser_amp=0.6, laser_omega=2.0, laser_duration=1.5)

    m = pc.Model(tiny_params(**kw))
    H0 = linear_h_matrix(m)                       # kinetic with the kick alone
    H0 = 0.5 * (H0 + H0.conj().T)

    def h_at(t):                                  # the field only changes the kinetic diagonal
        return H0 + np.diag(m.local.kin_at(m.laser(t)) - m.local.kin)

    C0 = syn.initial_coefficients(m.grid.g2_basis(), 3, seed=4)
    st0 = m.init_state(C0)
    P0 = st0.Psi @ st0.Psi.conj().T
    nref = 600
    h = T / nref
    U = np.eye(m.grid.npw, dtype=complex)
    for k in range(nref):
        w, V = np.linalg.eigh(h_at((k + 0.5) * h))
        U = (V * np.exp(-1j * h * w)[None, :]) @ V.conj().T @ U
    P_ref = U @ P0 @ U.conj().T
    errs = []
    for nsteps in (3, 6, 12):
        mm = pc.Model(tiny_params(dt=T / nsteps, **kw))
        st = mm.init_state(C0)
        st, infos = mm.propagate(st, nsteps)
        assert all(i.converged for i in infos)
        errs.append(np.linalg.norm(st.Psi @ st.Psi.conj().T - P_ref))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.3 < r1 < 4.7 and 3.3 < r2 < 4.7, errs


# ---- RK4 (the explicit integrator the paper compares with) ---------------------------

def test_rk4_fourth_order_against_matrix_exponential():
    """Fixed linear H: the error of P(T) falls ~16x per halving of dt."""
    T = 0.8
    errs = []
    for nsteps in (4, 8, 16):
        m = pc.Model(tiny_params(alpha=0.0, use_hartree=False, use_lda=False, dt=T / nsteps))
        C0 = syn.initial_coefficients(m.grid.g2_basis(), 3, seed=4)
        st = m.init_state(C0)
        P0 = st.Psi @ st.Psi.conj().T
        H = linear_h_matrix(m)
        w, V = np.linalg.eigh(0.5 * (H + H.conj().T))
        U = (V * np.exp(-1j * T * w)[None, :]) @ V.conj().T
        for _ in range(nsteps):
            st, _ = m.rk4_step(st)
        errs.append(np.linalg.norm(st.Psi @ st.Psi.conj().T - U @ P0 @ U.conj().T))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 13.0 < r1 < 19.0 and 13.0 < r2 < 19.0, errs


def test_rk4_and_ptcn_agree_on_the_full_hamiltonian():
    """Nonlinear H (Hartree, LDA, exact exchange, laser): RK4 at a small step and PT-CN at
    steps of 4 of those give the same density matrix up to PT-CN's O(dt^2) error, which
    shrinks 4x when both steps halve."""
    kw = dict(fock_mode="exact", laser_amp=0.2, laser_omega=1.0, laser_duration=2.0, n_orb=3)
    T = 0.4
    diffs = []
    for n_pt in (2, 4):
        m_rk = pc.Model(tiny_params(dt=T / (4 * n_pt), **kw))
        m_pt = pc.Model(tiny_params(dt=T / n_pt, **kw))
        C0 = syn.initial_coefficients(m_rk.grid.g2_basis(), 3, seed=6)
        a = m_rk.init_state(C0)
        b = m_pt.init_state(C0)
        for _ in range(4 * n_pt):
            a, _ = m_rk.rk4_step(a)
        b, infos = m_pt.propagate(b, n_pt)
        assert all(i.converged for i in infos)
        diffs.append(np.linalg.norm(a.Psi @ a.Psi.conj().T - b.Psi @ b.Psi.conj().T))
    assert diffs[1] < diffs[0] / 3.0, diffs
    assert diffs[1] < 1e-3, diffs


# ---- energy conservation --------------------------------------------------------------

def test_nonlinear_energy_drift_is_second_order():
    """Full H (Hartree, LDA, exact exchange) after the kick, time-independent: the energy
    change over a fixed time falls about 4x when dt halves."""
    T = 0.8
    drifts = []
    for nsteps in (2, 4, 8):
        m = pc.Model(tiny_params(fock_mode="exact", dt=T / nsteps, kick=(0.3, 0.0, 0.0)))
        C0 = syn.initial_coefficients(m.grid.g2_basis(), 3, seed=10)
        st = m.init_state(C0)
        e0 = st.energy
        st, infos = m.propagate(st, nsteps)
        assert all(i.converged for i in infos)
        drifts.append(abs(st.energy - e0))
    r1, r2 = drifts[0] / drifts[1], drifts[1] / drifts[2]
    assert 2.8 < r1 < 5.5 and 2.8 < r2 < 5.5, drifts


def test_anderson_fixed_point_equals_newton_solution():
    """The PT-CN fixed point R_f(Psi_f) = 0 (Eq. 5 with exact exchange) solved by Newton's
    method with a dense finite-difference Jacobian (real and imaginary parts as unknowns)
    equals the oracle's Anderson iterate."""
    p = tiny_params(dt=0.3, fock_mode="exact", omega=0.3, ecut=1.0, n_orb=2)
    m = pc.Model(p)
    C0 = syn.initial_coefficients(m.grid.g2_basis(), 2, seed=15)
    st = m.init_state(C0)
    st2, info = m.step(st)
    assert info.converged

    dt = p.dt
    Psi_n = st.Psi
    HP = m.apply_h(Psi_n, Psi_n, "exact")
    Psi_half = Psi_n - 0.5j * dt * (HP - Psi_n @ (Psi_n.conj().T @ HP))
    shape = Psi_n.shape

    def resid(z):
        Psi = (z[: z.size // 2] + 1j * z[z.size // 2:]).reshape(shape)
        H = m.apply_h(Psi, Psi, "exact")
        R = Psi + 0.5j * dt * (H - Psi @ (Psi.conj().T @ H)) - Psi_half
        return np.concatenate([R.real.ravel(), R.imag.ravel()])

    z = np.concatenate([Psi_half.real.ravel(), Psi_half.imag.ravel()])
    h = 1e-6
    for _ in range(8):
        F = resid(z)
        if np.linalg.norm(F) < 1e-12:
            break
        J = np.empty((z.size, z.size))
        for k in range(z.size):
            e = np.zeros(z.size)
            e[k] = h
            J[:, k] = (resid(z + e) - resid(z - e)) / (2 * h)
        z = z - np.linalg.solve(J, F)
    assert np.linalg.norm(resid(z)) < 1e-10
    Psi_newton = pc.orthonormalize((z[: z.size // 2] + 1j * z[z.size // 2:]).reshape(shape))
    assert np.max(np.abs(Psi_newton - st2.Psi)) < 1e-9


def test_si8_trajectory_is_stable_under_perturbation():
    """The Si8 configuration the GPU trajectory test compares step by step (40 relaxation
    steps, 20 SCF iterations per step) is a stable iteration: a 1e-13 relative change of
    the start orbitals stays at that size over five PT-CN steps (with 6 iterations from a
    10-step relaxation, by contrast, the fixed-point iteration of Alg. 1 diverges and
    rounding decides the trajectory)."""
    w = syn.si_workload("si8", scf_fixed_iters=20)
    m = pc.Model(pc.Params.from_dict(w))
    C0 = syn.initial_coefficients(m.grid.g2_basis(), w["n_orb"], seed=0)
    C1 = C0 * (1 + 1e-13 * np.random.default_rng(1).standard_normal(C0.shape))
    a, b = m.init_state(C0), m.init_state(C1)
    for _ in range(5):
        a, ia = m.step(a)
        b, _ = m.step(b)
        assert np.abs(a.Psi - b.Psi).max() / np.abs(a.Psi).max() < 1e-11
        assert ia.resid_norm < 1e-2
