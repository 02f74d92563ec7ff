/*
 * pt.h -- C ABI of the GB300 library for parallel-transport Crank-Nicolson
 * real-time TDDFT with a screened hybrid functional (arXiv:1905.01348).
 *
 * The library applies the Fock exchange operator of Eq. 3 by a fused
 * pair-product / 3D FFT / kernel multiply / inverse FFT / accumulate CUDA
 * pipeline, builds and applies its adaptively compressed (ACE) form, and runs
 * the PT-CN step of Eq. 5 / Alg. 1 (residual of Alg. 3, per-band Anderson
 * mixing and Cholesky orthonormalisation of Sec. 3.4) on one GPU.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Cell: orthorhombic, edge lengths cell[3] (bohr); grid n[3] points, row-major
 *   with axis 2 fastest; each n[k] must be one of 8, 12, 16, 24, 32, 48, 64, 96.
 * Basis: the grid frequencies G = 2 pi m / a with |G|^2 / 2 <= ecut, listed
 *   by increasing flat grid index (m in FFT index order). npw = basis size.
 * Orbitals: complex128, interleaved (re, im), band-major: orbital b occupies
 *   elements [b * npw, (b + 1) * npw). psi(r) = Omega^{-1/2} sum_G c(G) e^{iG.r}.
 * Occupation: every orbital doubly occupied, rho = 2 sum_b |psi_b|^2 (spin
 *   omitted as in Sec. 2).
 * Memory: the caller owns all device memory. pt_init_system receives one
 *   device workspace of at least pt_workspace_size() bytes (256-byte aligned)
 *   and a cudaStream_t (as void*, NULL = default stream); the library never
 *   allocates device memory and enqueues all device work on that stream.
 *   Host pointers are borrowed for the duration of the call. The workspace
 *   must stay valid until pt_destroy.
 * Errors: every call returns pt_status. On failure nothing is aborted;
 *   pt_last_error() gives a message. A failed step leaves the orbitals at the
 *   last consistent state. Calls that return host data synchronise the stream.
 * Threads: a pt_system is not thread safe; distinct systems are independent.
 */
#ifndef PT_H
#define PT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum pt_status {
  PT_OK = 0,
  PT_ERR_INVALID = 1,        /* bad argument or unsupported size */
  PT_ERR_OOM = 2,            /* workspace smaller than pt_workspace_size() */
  PT_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  PT_ERR_NOT_CONVERGED = 4,  /* SCF loop reached scf_max (state still advanced) */
  PT_ERR_NOT_PD = 5,         /* Cholesky met a non-positive pivot */
  PT_ERR_TIMEOUT = 6         /* reserved: the kernels have no device-side waits */
} pt_status;

enum { PT_FP64 = 0, PT_MIXED = 1 };                       /* precision */
enum { PT_FOCK_EXACT = 0, PT_FOCK_ACE = 1, PT_FOCK_NONE = 2 }; /* exchange mode */

typedef struct pt_params {
  int n[3];              /* grid points per axis */
  double cell[3];        /* cell edge lengths, bohr */
  double ecut;           /* planewave cutoff, Ha (Sec. 4: 10 Ha) */
  int n_orb;             /* number of orbitals N_e */
  int n_atoms;           /* Gaussian wells */
  const double* atom_frac; /* host, 3 * n_atoms fractional positions (read during init only) */
  double well_depth;     /* D: V_ion(r) = -D sum_a exp(-|r - R_a|^2 / (2 sigma^2)) */
  double well_sigma;     /* sigma, bohr */
  double omega;          /* screening w of K(r) = erfc(w r)/r, bohr^-1 */
  double alpha;          /* Fock mixing fraction (Sec. 2); (1 - alpha) Slater exchange */
  double dt;             /* time step, a.u. (Sec. 4: 50 as) */
  double kick[3];        /* velocity-gauge kick kappa, bohr^-1: kinetic |G + kappa|^2 / 2 */
  int anderson_dim;      /* Anderson history depth (Sec. 4: 20) */
  double anderson_beta;  /* Anderson mixing parameter */
  double scf_tol;        /* density-change tolerance (Sec. 4: 1e-6) */
  int scf_max;           /* iteration cap when scf_fixed_iters == 0 */
  int scf_fixed_iters;   /* > 0: run exactly this many SCF iterations */
  int precision;         /* PT_FP64, or PT_MIXED: FP32 pair FFTs and ACE products */
  int fock_mode;         /* PT_FOCK_EXACT (V_X every SCF iteration) or PT_FOCK_ACE (once per step) */
  int use_hartree;       /* 1: include the Hartree potential */
  int use_lda;           /* 1: include (1 - alpha) Slater exchange */
  int relax_iters;       /* start-state relaxation steps (steepest descent on H_loc) */
  double relax_tau;      /* relaxation step length */
  double relax_mix;      /* Kerker mixing weight b of the relaxation density */
  double relax_q0;       /* Kerker wavevector q0 (bohr^-1): weight b |G|^2 / (|G|^2 + q0^2) */
  int pair_tile;         /* orbitals per pair-tile edge (0 = automatic) */
  int pair_tiles_per_launch; /* cap on pair tiles per launch group, which sizes the pair
                              * intermediate in the workspace (0 = automatic: up to 16 GB) */
  /* Laser pulse (Sec. 4: 380 nm, 30 fs; its shape is given only as a figure), velocity
   * gauge: A(t) = laser_amp sin^2(pi t / laser_duration) sin(laser_omega t) laser_dir for
   * 0 <= t <= laser_duration, 0 after; kinetic |G + kick + A(t)|^2 / 2. Step n runs from
   * t_n = n dt to t_{n+1}: H_n uses A(t_n), the SCF and the new observables A(t_{n+1}).
   * laser_amp = 0 switches it off. */
  double laser_amp;      /* A0, a.u. */
  double laser_omega;    /* carrier frequency, a.u. (380 nm: 0.1199) */
  double laser_duration; /* pulse length T, a.u. (30 fs: 1240.4) */
  double laser_dir[3];   /* polarisation (used as given) */
  /* Grid of the pair FFTs of the exchange (Eq. 3). All 0: the grid n (alias-free for the
   * workloads). Otherwise a grid that must hold the basis sphere but may alias the pair
   * products, as the paper's exchange on its wavefunction grid (Sec. 4); the orbitals are
   * transformed onto it for every exchange. pt_exchange_static does not support it. */
  int n_fock[3];
} pt_params;

typedef struct pt_system pt_system;

typedef struct pt_step_info {
  int scf_iters;         /* SCF iterations taken */
  int converged;         /* 1 if the density change fell below scf_tol (or fixed iterations) */
  double resid_norm;     /* Frobenius norm of R_f at the last iteration (FP64) */
  double drho;           /* last density change dV sum |rho_new - rho_old| / (2 N_e) */
  double energy;         /* total energy of the new orbitals, Ha */
  double dipole[3];      /* -dV sum_r r rho(r), r in [0, a) */
  double time;           /* t_{n+1} = (n + 1) dt, a.u., the time of the new orbitals */
} pt_step_info;

/* Basis size for these parameters. Planewave basis of Sec. 3.1 / Sec. 4. */
pt_status pt_basis_size(const pt_params* p, int* npw);

/* Basis listing: flat grid index (int64) of each basis vector, in basis order.
 * out_host must hold npw entries. */
pt_status pt_basis_indices(const pt_params* p, int64_t* out_host);

/* Device workspace bytes pt_init_system needs for these parameters. */
pt_status pt_workspace_size(const pt_params* p, size_t* bytes);

/* Create a system (Eq. 5 state). psi0_host: n_orb x npw complex128 initial
 * coefficients (need not be orthonormal). They are orthonormalised by
 * Cholesky (Sec. 3.4), relaxed by relax_iters preconditioned steepest-descent
 * steps on the local Hamiltonian of a Kerker-mixed density (a stand-in for
 * the ground state the paper starts from), and the exchange data of the
 * start state (W = V_X Psi, and ACE when fock_mode is PT_FOCK_ACE) are
 * built. Synchronises the stream. */
pt_status pt_init_system(const pt_params* p, const double* psi0_host, void* d_workspace,
                         size_t workspace_bytes, void* stream, pt_system** out);

/* Build ACE from the current orbitals (ACE cited in Sec. 1): W = V_X Psi by
 * the symmetric pair pipeline (Eq. 3, Alg. 2), M = Psi^H W, -M = L L^H,
 * xi = W L^{-H}. Returns PT_ERR_NOT_PD if -M is not positive definite. */
pt_status pt_build_ace(pt_system* s);

/* Y = H[P] X for ncols device columns X (complex128, band-major, npw each),
 * P the current density matrix; H as in Eq. 2. fock_mode PT_FOCK_EXACT
 * applies V_X by the pair pipeline (Eq. 3), PT_FOCK_ACE applies
 * -xi (xi^H X), PT_FOCK_NONE omits exchange. X and Y may not overlap. */
pt_status pt_apply_h(pt_system* s, const void* d_X, void* d_Y, int ncols, int fock_mode);

/* W = V_X[P] Psi for the current orbitals, device output (npw x n_orb
 * complex128, band-major). The hot path: symmetric pair tiles, Eq. 3. */
pt_status pt_exchange(pt_system* s, void* d_W);

/* One PT-CN step (Eq. 5, Alg. 1). out (host, may be NULL) receives the step
 * information. Returns PT_ERR_NOT_CONVERGED if scf_max was reached (the step
 * is still taken). */
pt_status pt_cn_step(pt_system* s, pt_step_info* out);

/* One explicit 4th-order Runge-Kutta step of i dPsi/dt = H[P] Psi (Eq. 1), the
 * integrator the paper compares PT-CN with (Sec. 5: RK4 needs about 0.5 as
 * where PT-CN takes 50 as). No counterpart in the PT-CN path: each stage's
 * Hamiltonian is built from that stage's orbitals (density, local potential,
 * exact exchange whatever fock_mode says; the laser field at the stage time),
 * and the orbitals are not re-orthonormalised. Advances the step index; out
 * (may be NULL) gets energy, dipole and time (scf_iters = 0). Errors as
 * pt_cn_step. */
pt_status pt_rk4_step(pt_system* s, pt_step_info* out);

/* nsteps PT-CN steps; out_host (may be NULL) receives nsteps entries. Stops
 * early only on an error other than PT_ERR_NOT_CONVERGED. */
pt_status pt_propagate(pt_system* s, int nsteps, pt_step_info* out_host);

/* Copy the current orbitals (n_orb x npw complex128) to host memory. */
pt_status pt_get_orbitals(pt_system* s, double* psi_host);

/* Replace the current orbitals (n_orb x npw complex128, host), orthonormalise
 * them and rebuild the exchange data (no relaxation). Checkpoint resume. */
pt_status pt_set_orbitals(pt_system* s, const double* psi_host);

/* Energy and dipole of the current orbitals (host outputs, dipole[3]). */
pt_status pt_observables(pt_system* s, double* energy, double* dipole);

/* Device pointer of the current orbitals (npw x n_orb complex128). */
pt_status pt_orbitals_device(pt_system* s, void** d_psi);

/* Timing of the exchange pair pipeline (the three pair kernels of every
 * exchange application, Eq. 3): when enabled, CUDA events are recorded on the
 * system's stream around each application's pair kernels (one extra
 * synchronisation per application). pt_get_timing returns the accumulated
 * milliseconds, unordered pairs solved and pair-kernel launch groups since
 * the last reset; reset clears them. */
pt_status pt_set_timing(pt_system* s, int enable);
pt_status pt_get_timing(pt_system* s, double* pair_ms, int64_t* pairs, int64_t* launch_groups, int reset);

/* Checkpoint and resume (no counterpart in the paper). Between steps a
 * system's state is its step index n (time t_n = n dt, which fixes the laser
 * field of H_n), its orbitals Psi_n and W = V_X Psi_n (the exchange of Eq. 3
 * applied to them), both npw x n_orb complex128 (interleaved re, im),
 * band-major.
 * pt_get_state copies Psi and W to host buffers psi_host and w_host
 * (caller-owned, npw * n_orb complex128 each; pinned memory copies fastest),
 * stores n in *step (may be NULL) and synchronises the system's stream.
 * pt_set_state uploads a state taken by pt_get_state from a system with the
 * same parameters, then rebuilds from it, without an exchange, what the next
 * step needs: the kinetic term at t_n, the real-space orbitals, the ACE
 * operator (-Psi^H W = L L^H, xi = W L^{-H}) and the observables. The next
 * pt_cn_step then reproduces the original run bit for bit. Host buffers are
 * read during the call only.
 * Errors: PT_ERR_INVALID for NULL arguments or step < 0; PT_ERR_NOT_PD when
 * -Psi^H W is not positive definite (W is not the exchange of Psi), after
 * which the system must be given a state again (pt_set_state or
 * pt_set_orbitals) before it steps; PT_ERR_CUDA for a failed copy or launch. */
pt_status pt_get_state(pt_system* sys, double* psi_host, double* w_host, int64_t* step);
pt_status pt_set_state(pt_system* sys, const double* psi_host, const double* w_host, int64_t step);

/* Number of CUDA kernels this library has launched in this process (all
 * systems); differences of two readings count the launches in between. */
pt_status pt_launch_count(uint64_t* count);

/* V_X Psi without any device allocation. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc (a plug-in whose
 * host application owns all device memory through its own allocator, or code
 * that must not allocate after start-up, since an allocation can synchronise
 * the device or fail under memory pressure). It computes what pt_exchange
 * computes, for the orbitals d_psi given by the caller (n_orb x npw
 * complex128, band-major, device; they define P and are the vectors V_X is
 * applied to) into d_w (same shape, device), enqueued on `stream`, and
 * synchronises that stream before returning. Only the p fields that define
 * the grid, basis, kernel and precision are used.
 * Scratch: a file-scope device array of 64 MiB that every GPU loading this
 * library holds until the process exits. It must fit the real-space
 * orbitals, the exchange accumulators and at least one pair tile;
 * larger systems get PT_ERR_OOM with the sizes in pt_last_error(NULL).
 * The first call on a device looks up the array's device address (set-up);
 * make that first call before any stream capture. Every call reuses the same
 * array and overwrites its contents (the accumulators are cleared by each
 * call): calls that overlap on the GPU, from any stream or thread, race. */
pt_status pt_exchange_static(const pt_params* p, const void* d_psi, void* d_w, void* stream);

/* Release the handle (the workspace stays owned by the caller). */
pt_status pt_destroy(pt_system* s);

/* Message of the last error on this handle, or, when s is NULL, of the last
 * failed call without a handle (pt_init_system, pt_workspace_size,
 * pt_exchange_static, pt_launch_count, or any call given a NULL handle) on
 * the calling thread. Never NULL; valid until the next call on the same
 * handle or thread. */
const char* pt_last_error(const pt_system* s);

#ifdef __cplusplus
}
#endif

#endif /* PT_H */
