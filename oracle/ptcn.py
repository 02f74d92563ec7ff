"""ORACLE (test infrastructure only): one PT-CN step (Alg. 1) with Anderson mixing.

The parallel-transport gauge (Eq. 4) evolves i dPsi/dt = H Psi - Psi (Psi^H H Psi);
its Crank-Nicolson form (Eq. 5) is the implicit equation

    Psi_{n+1} + i dt/2 {H_{n+1} Psi_{n+1} - Psi_{n+1}(Psi_{n+1}^H H_{n+1} Psi_{n+1})}
        = Psi_n - i dt/2 {H_n Psi_n - Psi_n (Psi_n^H H_n Psi_n)},

solved per step as in Alg. 1:
  1. R_n = H_n Psi_n - Psi_n (Psi_n^H H_n Psi_n)
  2. Psi_half = Psi_n - i dt/2 R_n ; Psi_f = Psi_half
  3. rho_f from Psi_f
  4. loop: update H_f from rho_f and Psi_f; R_f = Psi_f + i dt/2 (H_f Psi_f - Psi_f S_f)
     - Psi_half with S_f = Psi_f^H H_f Psi_f (Alg. 3 computes it this way);
     Anderson update of Psi_f; new rho_f; stop when rho changes little
  5. orthonormalise Psi_f by Cholesky of Psi_f^H Psi_f (Sec. 3.4) -> Psi_{n+1}

Readings (the paper is silent on these details):

* Alg. 1 writes "Psi_f H_f Psi_f" inside R_f; the conjugate transpose of Eq. 5 is meant.
* Anderson mixing (Sec. 3.4: one least-squares problem per wavefunction, mixing
  dimension up to 20) is read as type-II Anderson for each band b on its own,
  with x = Psi_f[:, b] and r = -R_f[:, b]:
      x <- x + beta r - (dX + beta dR) gamma,  (dR^H dR + 1e-14 tr(dR^H dR) I) gamma = dR^H r,
  dX, dR the differences of consecutive iterates and residuals (newest last,
  oldest dropped past the mixing dimension), the small system solved by
  Cholesky; when that factorisation meets a non-positive pivot (or the Gram
  matrix is zero) gamma = 0 for that band. The history restarts every step.
* Density change: dV sum_r |rho_new - rho_old| / N_el with N_el = 2 N_e; the
  loop stops when it drops below scf_tol (Sec. 4: 1e-6), or after exactly
  scf_fixed_iters iterations when that is positive.
* Fock modes: "exact" re-evaluates V_X[Psi_f] Psi_f every iteration (the paper's
  GPU path, 24 exchange evaluations per step, Sec. 6); "ace" builds the ACE
  operator once from Psi_n and keeps it through the loop. Rebuilding ACE from
  Psi_f every iteration equals "exact" for H_f Psi_f. With ``ace_outer`` = k > 0
  the "ace" step, once its SCF has converged, rebuilds ACE from the converged
  Psi_f and runs the SCF again (restarted Anderson history), k times: the
  operator then tracks Psi_{n+1} instead of Psi_n. Building ACE once per step
  perturbs H_f by O(dt), so one step differs from "exact" by O(dt^2) (pinned:
  tests/test_oracle_ptcn.py).
* The exchange data of Psi_{n+1} (W = V_X Psi_{n+1}, and the ACE operator) are
  produced at the end of a step, where they also give the energy E_{n+1}, and
  the next step reuses them for R_n.
* Laser (Sec. 4 drives the system with a 380 nm pulse over 30 fs; the pulse
  shape is shown only in a figure): velocity gauge with the uniform vector
  potential A(t) = A0 sin^2(pi t / T) sin(omega t) e for 0 <= t <= T and 0
  after, omega = 2 pi c / 380 nm = 0.1199 a.u., T = 30 fs = 1240.4 a.u.; the
  kinetic term is |G + kappa + A(t)|^2 / 2. Step n runs from t_n = n dt to
  t_{n+1}: H_n uses A(t_n), H_f and the observables of Psi_{n+1} use A(t_{n+1}).
  A0 = 0 (the default) leaves the kick alone.
* Fock grid (Sec. 4: the paper evaluates the exchange on the wavefunction grid,
  half the density grid per axis): with ``fock_grid`` set, Eq. 3 is evaluated
  on that grid -- orbitals placed there from their basis coefficients (the
  basis sphere must fit), pair products, kernel and W formed there, W read back
  on the basis sphere. Pair products then alias (their frequencies reach twice
  the sphere's), which is the discretisation the paper uses; None keeps the
  alias-free grid n.
* Start state: the paper propagates from a ground state (Sec. 4: the laser
  drives a converged system). The synthetic orbitals are random, and from a
  random start the fixed point of Alg. 1 does not converge at dt = 50 as. So
  the initial orbitals are first orthonormalised and then relaxed by
  ``relax_iters`` steps of preconditioned steepest descent on the local
  Hamiltonian (no Fock term):
      Psi <- orth(Psi - tau P (H_loc Psi - Psi (Psi^H H_loc Psi))),
      P = diag 1 / (1 + |G + kappa|^2 / 2),
  with H_loc built from a Kerker-mixed density
      rho_mix <- rho_mix + F^{-1}[ b |G|^2 / (|G|^2 + q0^2) F[rho(Psi) - rho_mix] ],
  rho_mix starting at rho(Psi_0) (b = relax_mix, q0 = relax_q0). Without
  the mixing the long-wavelength Hartree response (4 pi / |G|^2, growing with
  the cell) makes the descent unstable in the 3x3x3 supercell. Pinned by its
  fixed point (tests/test_oracle_relax.py): the lowest eigen-subspace of the
  dense H for a linear H, the self-consistent aufbau state with Hartree + LDA.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.linalg as sla

from .discretization import Grid
from . import exchange as ex
from . import hamiltonian as hm


@dataclasses.dataclass
class Params:
    n: tuple
    cell: tuple
    ecut: float
    atoms: np.ndarray
    n_orb: int
    well_depth: float = 2.0
    well_sigma: float = 1.2
    omega: float = 0.106
    alpha: float = 0.25
    dt: float = 2.07
    kick: tuple = (0.01, 0.0, 0.0)
    anderson_dim: int = 20
    anderson_beta: float = 1.0
    scf_tol: float = 1e-6
    scf_max: int = 50
    scf_fixed_iters: int = 0
    fock_mode: str = "ace"          # "exact" or "ace"
    use_hartree: bool = True
    use_lda: bool = True
    relax_iters: int = 40
    relax_tau: float = 1.0
    relax_mix: float = 0.5
    relax_q0: float = 1.0
    laser_amp: float = 0.0            # A0 (a.u.); 0 switches the laser off
    laser_omega: float = 0.1199       # carrier frequency (a.u.): 380 nm
    laser_duration: float = 1240.4    # pulse length T (a.u.): 30 fs
    laser_dir: tuple = (1.0, 0.0, 0.0)
    fock_grid: tuple = None           # grid of the pair FFTs; None: the grid n (alias-free)
    ace_outer: int = 0                # "ace" mode: ACE rebuilds from the converged Psi_f per step

    @classmethod
    def from_dict(cls, d: dict) -> "Params":
        names = {f.name for f in dataclasses.fields(cls)}
        return cls(**{k: v for k, v in d.items() if k in names})


@dataclasses.dataclass
class State:
    Psi: np.ndarray          # (npw, N_e) orthonormal orbitals
    W: np.ndarray            # V_X[Psi] Psi, (npw, N_e)
    M: np.ndarray            # Psi^H W
    xi: np.ndarray           # ACE projector (npw, N_e) or None
    energy: float
    dipole: np.ndarray
    step: int = 0


@dataclasses.dataclass
class StepInfo:
    scf_iters: int
    converged: bool
    resid_norm: float
    drho: float
    energy: float
    dipole: np.ndarray


class Model:
    def __init__(self, p: Params):
        self.p = p
        self.grid = Grid(p.n, p.cell, p.ecut)
        self.local = hm.LocalModel(self.grid, p.atoms, p.well_depth, p.well_sigma, p.kick, p.alpha,
                                   p.use_hartree, p.use_lda)
        self.fgrid = self.grid
        if p.fock_grid is not None and tuple(p.fock_grid) != tuple(p.n):
            self.fgrid = Grid(p.fock_grid, p.cell, p.ecut)
            if not np.array_equal(self.fgrid.gvec_basis(), self.grid.gvec_basis()):
                raise ValueError("the basis sphere does not fit on the Fock grid")
        self.khat = ex.screened_kernel(self.fgrid, p.omega)

    # -- external field ---------------------------------------------------------
    def laser(self, t: float) -> np.ndarray:
        """Laser vector potential A(t) (laser reading in the module header)."""
        p = self.p
        if p.laser_amp == 0.0 or t < 0.0 or t > p.laser_duration:
            return np.zeros(3)
        env = np.sin(np.pi * t / p.laser_duration) ** 2
        e = np.asarray(p.laser_dir, dtype=np.float64)
        return p.laser_amp * env * np.sin(p.laser_omega * t) * e

    def kin_at_step(self, n: int) -> np.ndarray:
        return self.local.kin_at(self.laser(n * self.p.dt))

    # -- pieces of H --------------------------------------------------------
    def density(self, C: np.ndarray) -> np.ndarray:
        return hm.density(self.grid, self.grid.to_real(C.T))

    def vx(self, C: np.ndarray, X: np.ndarray) -> np.ndarray:
        if self.p.alpha == 0.0:
            return np.zeros_like(X)
        return ex.apply_vx(self.fgrid, self.khat, self.p.alpha, C, X)

    def exchange_data(self, C: np.ndarray):
        """W = V_X C, M = C^H W and the ACE projector (None when alpha = 0 or mode is exact)."""
        if self.p.alpha == 0.0:
            W = np.zeros_like(C)
            return W, np.zeros((C.shape[1], C.shape[1]), complex), None
        if self.p.fock_mode == "ace":
            W, M, _, xi = ex.build_ace(self.fgrid, self.khat, self.p.alpha, C)
            return W, M, xi
        W = self.vx(C, C)
        return W, C.conj().T @ W, None

    def apply_h(self, C: np.ndarray, X: np.ndarray, fock: str, xi=None, kin=None) -> np.ndarray:
        """H[P] X with P from the columns of C; fock = "exact" | "ace" | "none"."""
        rho = self.density(C)
        out = self.local.apply_local(self.local.local_potential(rho), X, kin)
        if fock == "exact":
            out = out + self.vx(C, X)
        elif fock == "ace" and xi is not None:
            out = out + ex.apply_ace(xi, X)
        return out

    def observables(self, C: np.ndarray, M: np.ndarray, kin=None):
        rho = self.density(C)
        e = self.local.energy_terms(C, rho, float(np.real(np.trace(M))), kin)
        return e["total"], hm.dipole(self.grid, rho)

    # -- state ----------------------------------------------------------------
    def relax(self, Psi: np.ndarray, iters: int, tau: float) -> np.ndarray:
        """Preconditioned steepest descent on the local Hamiltonian (start-state reading above)."""
        from .discretization import fftn, ifftn
        prec = (1.0 / (1.0 + self.local.kin))[:, None]
        g2 = self.grid.g2
        q2 = self.p.relax_q0 ** 2
        kerker = self.p.relax_mix * g2 / (g2 + q2)
        rho_mix = self.density(Psi)
        for _ in range(int(iters)):
            rho = self.density(Psi)
            rho_mix = rho_mix + np.real(ifftn(kerker * fftn((rho - rho_mix).astype(complex))))
            HP = self.local.apply_local(self.local.local_potential(rho_mix), Psi)
            R = HP - Psi @ (Psi.conj().T @ HP)
            Psi = orthonormalize(Psi - tau * prec * R)
        return Psi

    def init_state(self, C0_rows: np.ndarray) -> State:
        """Orthonormalise the given coefficients (rows = orbitals), relax, build the exchange data."""
        Psi = orthonormalize(np.asarray(C0_rows, dtype=np.complex128).T)
        Psi = self.relax(Psi, self.p.relax_iters, self.p.relax_tau)
        W, M, xi = self.exchange_data(Psi)
        E, d = self.observables(Psi, M)
        return State(Psi=Psi, W=W, M=M, xi=xi, energy=E, dipole=d, step=0)

    def step(self, st: State) -> tuple[State, StepInfo]:
        p = self.p
        g = self.grid
        dt = p.dt
        ne = st.Psi.shape[1]
        n_el = 2.0 * ne

        # kinetic diagonals of H_n (t_n) and H_{n+1} (t_{n+1})
        kin_n = self.kin_at_step(st.step)
        kin_f = self.kin_at_step(st.step + 1)

        # Alg. 1: initial residual and half step (H_n Psi_n uses the stored W = V_X[Psi_n] Psi_n)
        Psi_n = st.Psi
        rho_n = self.density(Psi_n)
        HPsi_n = self.local.apply_local(self.local.local_potential(rho_n), Psi_n, kin_n) + st.W
        S_n = Psi_n.conj().T @ HPsi_n
        R_n = HPsi_n - Psi_n @ S_n
        Psi_half = Psi_n - 0.5j * dt * R_n

        # Alg. 1: Psi_f starts at Psi_half, with its density
        Psi_f = Psi_half.copy()
        rho_f = self.density(Psi_f)

        fixed = int(p.scf_fixed_iters)
        n_iter = fixed if fixed > 0 else int(p.scf_max)
        resid = np.inf
        drho = np.inf
        total = 0
        xi = st.xi
        outer_left = int(p.ace_outer) if (p.fock_mode == "ace" and p.alpha != 0.0) else 0
        while True:
            mix = Anderson(p.anderson_dim, p.anderson_beta)
            converged = False
            for _ in range(n_iter):
                total += 1
                # update the potential and H_f
                vloc = self.local.local_potential(rho_f)
                HPf = self.local.apply_local(vloc, Psi_f, kin_f)
                if p.alpha != 0.0:
                    if p.fock_mode == "exact":
                        HPf = HPf + self.vx(Psi_f, Psi_f)
                    else:
                        HPf = HPf + ex.apply_ace(xi, Psi_f)
                # fixed-point residual R_f (computed as in Alg. 3)
                S_f = Psi_f.conj().T @ HPf
                R_f = Psi_f + 0.5j * dt * (HPf - Psi_f @ S_f) - Psi_half
                resid = float(np.linalg.norm(R_f))
                # Anderson mixing
                Psi_f = mix.update(Psi_f, -R_f)
                # new density, convergence test
                rho_new = self.density(Psi_f)
                drho = float(g.dV * np.sum(np.abs(rho_new - rho_f)) / n_el)
                rho_f = rho_new
                if fixed == 0 and drho < p.scf_tol:
                    converged = True
                    break
            if fixed > 0:
                converged = True
            if outer_left == 0:
                break
            # outer ACE rebuild: the operator of the converged Psi_f, then the SCF again
            outer_left -= 1
            _, _, _, xi = ex.build_ace(self.fgrid, self.khat, p.alpha, Psi_f)
        it = total

        # orthonormalise, then the exchange data and observables of Psi_{n+1}
        Psi_next = orthonormalize(Psi_f)
        W, M, xi = self.exchange_data(Psi_next)
        E, d = self.observables(Psi_next, M, kin_f)
        new = State(Psi=Psi_next, W=W, M=M, xi=xi, energy=E, dipole=d, step=st.step + 1)
        return new, StepInfo(scf_iters=it, converged=converged, resid_norm=resid, drho=drho, energy=E, dipole=d)

    # -- explicit comparison integrator ----------------------------------------
    def h_of(self, X: np.ndarray, t: float) -> np.ndarray:
        """H[X X^H](t) X: density, local potential and exact exchange of the columns of X
        themselves, kinetic term at time t."""
        kin = self.local.kin_at(self.laser(t))
        out = self.local.apply_local(self.local.local_potential(self.density(X)), X, kin)
        if self.p.alpha != 0.0:
            out = out + self.vx(X, X)
        return out

    def rk4_step(self, st: State) -> tuple[State, StepInfo]:
        """One classical 4th-order Runge-Kutta step of i dPsi/dt = H[P] Psi (Eq. 1, the explicit
        integrator the paper compares PT-CN with in Sec. 5). The Hamiltonian of each stage is
        built from that stage's orbitals (exact exchange); no orthonormalisation."""
        dt = self.p.dt
        t = st.step * dt
        P0 = st.Psi
        k1 = -1j * self.h_of(P0, t)
        k2 = -1j * self.h_of(P0 + 0.5 * dt * k1, t + 0.5 * dt)
        k3 = -1j * self.h_of(P0 + 0.5 * dt * k2, t + 0.5 * dt)
        k4 = -1j * self.h_of(P0 + dt * k3, t + dt)
        Psi = P0 + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        W, M, xi = self.exchange_data(Psi)
        E, d = self.observables(Psi, M, self.kin_at_step(st.step + 1))
        new = State(Psi=Psi, W=W, M=M, xi=xi, energy=E, dipole=d, step=st.step + 1)
        return new, StepInfo(scf_iters=0, converged=True, resid_norm=0.0, drho=0.0, energy=E, dipole=d)

    def propagate(self, st: State, nsteps: int):
        infos = []
        for _ in range(int(nsteps)):
            st, info = self.step(st)
            infos.append(info)
        return st, infos


class Anderson:
    """Per-band type-II Anderson mixing with a bounded history (reading in the module header)."""

    def __init__(self, dim: int, beta: float):
        self.dim = int(dim)
        self.beta = float(beta)
        self.dX: list[np.ndarray] = []
        self.dR: list[np.ndarray] = []
        self.x_prev = None
        self.r_prev = None

    def update(self, x: np.ndarray, r: np.ndarray) -> np.ndarray:
        if self.x_prev is not None and self.dim > 0:
            self.dX.append(x - self.x_prev)
            self.dR.append(r - self.r_prev)
            if len(self.dX) > self.dim:
                self.dX.pop(0)
                self.dR.pop(0)
        self.x_prev = x.copy()
        self.r_prev = r.copy()
        out = x + self.beta * r
        if not self.dX:
            return out
        DX = np.stack(self.dX, axis=-1)                  # (npw, nb, k)
        DR = np.stack(self.dR, axis=-1)
        k = DX.shape[-1]
        for b in range(x.shape[1]):
            A = DR[:, b, :]
            G = A.conj().T @ A
            rhs = A.conj().T @ r[:, b]
            tr = float(np.real(np.trace(G)))
            gamma = np.zeros(k, dtype=np.complex128)
            if tr > 0.0:
                Gs = G + (1e-14 * tr) * np.eye(k)
                L = cholesky_or_none(Gs)
                if L is not None:
                    y = sla.solve_triangular(L, rhs, lower=True)
                    gamma = sla.solve_triangular(L.conj().T, y, lower=False)
            out[:, b] -= (DX[:, b, :] + self.beta * A) @ gamma
        return out


def cholesky_or_none(A: np.ndarray):
    """Lower Cholesky factor, or None at a non-positive pivot (textbook column algorithm)."""
    n = A.shape[0]
    L = np.zeros_like(A, dtype=np.complex128)
    for j in range(n):
        d = np.real(A[j, j] - np.vdot(L[j, :j], L[j, :j]))
        if not d > 0.0:
            return None
        L[j, j] = np.sqrt(d)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], np.conj(L[j, :j]))) / L[j, j]
    return L


def orthonormalize(Psi: np.ndarray) -> np.ndarray:
    """Psi L^{-H} with L L^H = Psi^H Psi (Cholesky orthogonalisation, Sec. 3.4)."""
    S = Psi.conj().T @ Psi
    L = np.linalg.cholesky(S)
    # X L^H = Psi  <=>  conj(L) X^T = Psi^T
    return sla.solve_triangular(L.conj(), Psi.T, lower=True).T
