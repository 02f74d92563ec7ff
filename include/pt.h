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
 *   Each system takes one 256-byte page-locked host block from a process-wide
 *   pool (allocated in chunks of 64, kept until exit) for its step readbacks;
 *   pt_exchange_static takes none. Host pointers are borrowed for the duration
 *   of the call. The workspace must stay valid until pt_destroy.
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
  PT_ERR_TIMEOUT = 6         /* a bounded wait inside a tensor-core kernel expired */
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
  /* Mixed precision only (iterative refinement of Alg. 1's fixed point): when scf_tol is
   * below this value (> 0), the residual R_n of the half step and every SCF iteration
   * after the density change has fallen below it evaluate H Psi (local potential,
   * ACE, PT projection) and R_f in FP64, so the iteration converges past the FP32
   * rounding floor (about 1e-8 in the density change). 0 = FP32 throughout. The
   * exchange of exact mode (PT_FOCK_EXACT) keeps its FP32 pair FFTs. */
  double scf_fp64_below;
  /* PT_FOCK_ACE only: after the SCF of a step has converged with ACE built from Psi_n,
   * rebuild ACE from the converged Psi_f (its exchange W = V_X Psi_f, M = Psi_f^H W,
   * -M = L L^H, xi = W L^{-H}) and run the SCF again (Anderson history restarted), this
   * many times per step. Each rebuild raises the order in dt of the difference to exact
   * exchange every iteration by one, at the cost of one exchange per rebuild. 0: ACE once
   * per step. */
  int ace_outer;
  /* Seed of the start coefficients pt_init_system generates when psi0_host is NULL
   * (pt_seeded_coefficients). */
  uint64_t seed;
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

/* Seeded start coefficients (host only, no device): out_host receives n_orb x npw
 * complex128 values (band-major, interleaved re/im), not orthonormal. Coefficient m
 * of band b is (g1 + i g2) exp(-|G_m|^2 / 4) with (g1, g2) standard normals by the
 * Box-Muller transform of the uniforms u1 = U(2j), u2 = U(2j + 1), j = b npw + m:
 * g1 = sqrt(-2 ln u1) cos(2 pi u2), g2 = sqrt(-2 ln u1) sin(2 pi u2). U(k) =
 * ((x_k >> 11) + 0.5) 2^-53, x_k the (k + 1)-th output of SplitMix64 (Steele, Lea and
 * Flood, 2014) started from the state p->seed: state += 0x9E3779B97F4A7C15; z = state;
 * z = (z ^ (z >> 30)) 0xBF58476D1CE4E5B9; z = (z ^ (z >> 27)) 0x94D049BB133111EB;
 * x = z ^ (z >> 31). A stand-in for the paper's ground state (Sec. 4), as any start. */
pt_status pt_seeded_coefficients(const pt_params* p, double* out_host);

/* Device workspace bytes pt_init_system needs for these parameters. */
pt_status pt_workspace_size(const pt_params* p, size_t* bytes);

/* Create a system (Eq. 5 state). psi0_host: n_orb x npw complex128 initial
 * coefficients (need not be orthonormal), or NULL for pt_seeded_coefficients of
 * p->seed. They are orthonormalised by
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

/* The complex products of ACE and of the PT residual as the mixed-precision path
 * computes them on the tensor cores: C = alpha op(A) op(B) + beta C, the
 * contractions M = Psi^H W, xi = W L^{-H}, xi^H X and -xi (xi^H X) of ACE (cited
 * in Sec. 1) and S = Psi^H (H Psi), H Psi - Psi S of Alg. 3. A and B are
 * complex64 (interleaved re, im), C is complex128, all column-major on the device:
 * element (i, k) of op(A) is A[i + k lda] for op_a = 0 and conj(A[k + i lda]) for
 * op_a = 1; likewise op(B) with ldb. op(A) is M x K, op(B) K x N, C M x N (ldc).
 * upper_b = 1 promises that op(B) is upper triangular (op(B)(k, j) = 0 for k > j),
 * which lets each output tile stop its reduction at its last column. Arithmetic: 3xTF32 (each operand split into two TF32 parts,
 * three products) with FP32 accumulation. d_ws: device scratch of ws_bytes >= 256
 * (256-byte aligned): its first 256 bytes hold a status word, the rest takes the
 * split-K partials of long reductions (M N complex128 per split; with no room the
 * reduction is not split). Enqueued on `stream`, which is synchronised before the
 * call returns (A and B may be NULL when K = 0: then C = beta C). Errors:
 * PT_ERR_INVALID for bad sizes or pointers, PT_ERR_TIMEOUT if
 * a bounded wait inside the kernel expired, PT_ERR_CUDA for a failed launch. */
pt_status pt_complex_product(int op_a, int op_b, int M, int N, int K, const double* alpha2, const void* d_A,
                             int64_t lda, const void* d_B, int64_t ldb, const double* beta2, void* d_C, int64_t ldc,
                             int upper_b, void* d_ws, size_t ws_bytes, void* stream);

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

/* Batches: several systems stepped together (no counterpart in the paper, which batches
 * the pair FFTs of one system into library calls, Sec. 3.2). The systems must share the
 * grid, Fock grid, precision, cell, cutoff and screened kernel (omega, alpha != 0); their
 * orbital counts, kicks, lasers and start states may differ. The pair tiles of all
 * systems go into shared launch groups: round r of every system's tile tournament
 * (Eq. 3, the pair loop of Alg. 2) forms one merged round, split into launch groups of
 * at most tiles_per_launch tiles (0: whole rounds, up to a 16 GB pair intermediate), with
 * pair_tile orbitals per tile edge (0: min(4, largest n_orb)). The merged pair-kernel
 * sequence is captured into a CUDA graph after its first run and replayed. With the same
 * pair_tile as a system's own (pt_params.pair_tile), batched results are bitwise those
 * of the system stepped alone.
 * pt_batch_workspace_size: device bytes pt_batch_create needs for these systems.
 * pt_batch_create: systems (nsys >= 1, distinct, created by pt_init_system and kept alive
 *   until pt_batch_destroy), a device workspace (256-byte aligned, caller-owned, not
 *   shared with the systems' workspaces) and a created stream (not the NULL stream: the
 *   graph is captured on it) for the merged pair kernels; the systems keep their own
 *   streams, ordered against the batch stream by events. Errors: PT_ERR_INVALID
 *   (incompatible systems, bad arguments), PT_ERR_OOM (workspace too small).
 * pt_batch_exchange: W = V_X Psi of every system's current orbitals into d_w[i]
 *   (npw x n_orb complex128, device), synchronising the systems' streams.
 * pt_batch_step: one PT-CN step (Eq. 5, Alg. 1) of every system, out_host[i] (may be
 *   NULL) receiving system i's step information. The SCF iterations of all systems are
 *   interleaved on their streams; the exchange of the new orbitals is the merged launch
 *   sequence. Returns PT_ERR_NOT_CONVERGED if any system reached scf_max (all steps are
 *   still taken), another error naming the system otherwise.
 * pt_batch_set_timing / pt_batch_get_timing: CUDA-event time of the merged pair kernels
 *   on the batch stream, as pt_set_timing / pt_get_timing.
 * Errors of batch calls are reported through pt_last_error(NULL) on the calling thread. */
typedef struct pt_batch pt_batch;
pt_status pt_batch_workspace_size(pt_system* const* systems, int nsys, int pair_tile, int tiles_per_launch,
                                  size_t* bytes);
pt_status pt_batch_create(pt_system* const* systems, int nsys, int pair_tile, int tiles_per_launch, void* d_ws,
                          size_t ws_bytes, void* stream, pt_batch** out);
pt_status pt_batch_exchange(pt_batch* b, void* const* d_w);
pt_status pt_batch_step(pt_batch* b, pt_step_info* out_host);
pt_status pt_batch_set_timing(pt_batch* b, int enable);
pt_status pt_batch_get_timing(pt_batch* b, double* pair_ms, int64_t* pairs, int64_t* launch_groups, int reset);
pt_status pt_batch_destroy(pt_batch* b);

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
