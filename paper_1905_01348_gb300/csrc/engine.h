// Engine internals shared by the library's translation units (not part of the C ABI):
// the record of one PT-CN system, the error macros, and the operations that
// setup.cu (parameters, tables, workspace layout, start state), engine.cu (the
// exchange, ACE, H Psi and the PT-CN step), batch.cu (several systems stepped
// together) and api.cu (the C ABI of include/pt.h) call across files.
#pragma once

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include "pt.h"
#include "common.cuh"
#include "internal.h"
#include "kernels.h"

#include <nvtx3/nvToolsExt.h>

using pt::Grid3;

// Named range around one phase of a step for profilers (NVTX; header-only, a no-op
// unless a tool is attached). Phases follow the timing rows of the paper's Table 1:
// H Psi, exchange / ACE, residual, Anderson mixing, density, orthonormalisation.
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};

// Carves 256-byte aligned pieces out of a caller-owned workspace (base 0: sizing only).
struct Carver {
  uintptr_t base;
  size_t off = 0;
  template <typename T> T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

constexpr double kSlater = 0.75;   // times (3/pi)^{1/3}

struct pt_system {
  // page-locked host block for the small readbacks of a step (read_small); nullptr on the
  // static path, which allocates nothing and reads back through plain copies
  void* pinned = nullptr;
  pt_params p{};
  std::vector<double> atoms;
  std::string err;
  cudaStream_t s = nullptr;
  Grid3 g{};
  long N = 0;
  int npw = 0, ne = 0, mdim = 0, hb = 1;
  double vol = 0.0, dV = 0.0;
  bool mixed = false;
  // device data
  int* basis = nullptr;
  double* kin = nullptr;            // |G + kick + A(t)|^2 / 2 of the current time
  double* gk3 = nullptr;            // G + kick per basis vector (three arrays of npw)
  int64_t n_step = 0;               // time index of the current orbitals: t = n_step dt
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  double* khat64 = nullptr;
  float* khat32 = nullptr;
  double *hfac = nullptr, *kfac = nullptr, *rho_mix = nullptr, *vion = nullptr, *vloc = nullptr, *vh = nullptr, *rho = nullptr, *rho2 = nullptr;
  double* d_atoms = nullptr;
  float* vloc32 = nullptr;
  double2 *psi = nullptr, *psi_half = nullptr, *psi_f = nullptr, *hpsi = nullptr, *tmp = nullptr, *rbuf = nullptr;
  double2 *wg = nullptr, *xi = nullptr, *xprev = nullptr, *rprev = nullptr;
  // Anderson history: complex128, or complex64 in mixed precision
  unsigned char *dX = nullptr, *dR = nullptr;
  double2* hbuf = nullptr;
  double2* psi_r = nullptr;
  float2* psi_r32 = nullptr;
  // complex64 copies for the FP32 products of mixed precision: xi (per step) and two
  // operand staging buffers (n_orb x npw) plus one n_orb x n_orb buffer
  float2 *xi32 = nullptr, *ga32 = nullptr, *gb32 = nullptr, *gs32 = nullptr;
  // basis-sphere tables of the pruned FP32 transforms (cubic 32/64/96 grids)
  bool use_sphere = false;
  pt::SphereTables sph{};
  int *sph_row_idx = nullptr, *sph_row_kbeg = nullptr, *sph_krow = nullptr, *sph_planes = nullptr;
  unsigned char *sph_rowlive = nullptr, *sph_planelive = nullptr;
  void *w_r = nullptr, *x_r = nullptr, *scratch = nullptr;   // on the Fock grid
  // Fock grid of the pair FFTs (the main grid unless n_fock is set)
  bool fock_own = false;
  Grid3 gf{};
  long Nf = 0;
  int* basis_f = nullptr;           // flat index of each basis vector on the Fock grid
  void* psi_rf = nullptr;           // real-space orbitals on the Fock grid (exchange precision)
  bool use_sphere_f = false;
  pt::SphereTables sphf{};
  int *sphf_row_idx = nullptr, *sphf_row_kbeg = nullptr, *sphf_krow = nullptr, *sphf_planes = nullptr;
  unsigned char *sphf_rowlive = nullptr, *sphf_planelive = nullptr;
  double2 *S = nullptr, *Mneg = nullptr, *Linv = nullptr, *Z = nullptr, *gemm_ws = nullptr;
  size_t gemm_ws_elems = 0;
  double2 *gram = nullptr, *rhs = nullptr, *gamma = nullptr;
  double *part = nullptr, *red = nullptr;
  int* status = nullptr;
  pt::PairTile *d_tiles_sym = nullptr, *d_tiles_x = nullptr;
  size_t max_tiles_x = 0;
  pt::FockPlan plan_sym{}, plan_x{};
  int plan_x_ncols = -1;
  pt::DevTwiddles tw{};
  // host state
  bool have_ace = false;
  bool psi_r_current = false;   // psi_r holds the real-space form of psi
  double energy = 0.0, dipole[3] = {0, 0, 0};
  int and_count = 0;
  std::vector<int> and_order;
  // pair-pipeline timing
  bool timing = false;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  double t_pair_ms = 0.0;
  long long t_pairs = 0, t_groups = 0;
};

// last error of calls that have no system handle (per calling thread)
// last error of calls that have no system handle (per calling thread)
extern thread_local std::string g_last_error;

// Argument errors of the handle entry points: the message goes to the handle, or to the
// calling thread's handle-less message when the handle itself is NULL.
pt_status invalid_arg(pt_system* sys, const char* fn, const char* what);

#define PT_CK(call)                                                               \
  do {                                                                            \
    cudaError_t _e = (call);                                                      \
    if (_e != cudaSuccess) {                                                      \
      sys->err = std::string(#call) + " -> " + pt::cuda_msg(_e);                  \
      return PT_ERR_CUDA;                                                         \
    }                                                                             \
  } while (0)
#define PT_TRY(call)                        \
  do {                                      \
    pt_status _st = (call);                 \
    if (_st != PT_OK) return _st;           \
  } while (0)

// ---- setup.cu: parameters, basis, tables, workspace layout, start state ----------
pt_status check_params(const pt_params* p, std::string* why);
int freq(int i, int n);   // FFT index -> signed frequency
void basis_list(const pt_params* p, std::vector<int>* idx, std::vector<double>* g2out);
pt_params fock_params(const pt_params* p);   // the parameters with the Fock grid as the grid
bool fock_is_own(const pt_params* p);
void set_pair_reach(pt::FockPlan* plan, const pt_params* p);
// pt_seeded_coefficients: n_orb x npw complex128 (interleaved) from p->seed
void seeded_coefficients(const pt_params* p, double* out);
int choose_tile(const pt_params* p);
int tiles_per_launch(const pt_params* p, long N, bool mixed);
int h_batch(const pt_params* p);
size_t carve(pt_system* sys, const pt_params* p, uintptr_t base);
pt_status init_body(pt_system* sys, const double* psi0_host);
// the static-scratch exchange (pt_exchange_static)
extern const size_t kStaticScratchBytes;
pt_status static_scratch_address(void** out);
size_t static_layout(pt_system* t, const pt_params* p, int npw, uintptr_t base, int tpl);
pt_status exchange_static_body(pt_system* t, const pt_params* p, const std::vector<int>& idx, const double2* d_psi,
                               double2* d_w);

// ---- engine.cu: exchange, ACE, H Psi, PT-CN step --------------------------------
pt_status real_orbitals(pt_system* sys, const double2* c);
pt_status real_orbitals_scf(pt_system* sys, const double2* c);
pt_status density_scf(pt_system* sys, double* rho);
pt_status local_potential(pt_system* sys);
pt_status apply_local(pt_system* sys, const double2* X, double2* out, int ncols);
pt_status apply_local_from_real(pt_system* sys, const double2* c, double2* out);
pt_status apply_local_scf(pt_system* sys, const double2* c, double2* out);
const void* fock_orbitals_addr(const pt_system* sys);
size_t exchange_cs(const pt_system* sys);
pt_status exchange_sym(pt_system* sys, const double2* coef, double2* out, int accumulate);
// the two ends of exchange_sym around the pair kernels (a batch runs those shared)
pt_status exchange_prepare(pt_system* sys, const double2* coef);
pt_status exchange_finish(pt_system* sys, double2* out, int accumulate);
pt_status exchange_x(pt_system* sys, const double2* X, int ncols, double2* out);
pt_status tc_status(pt_system* sys);
pt_status read_status(pt_system* sys, int* h);
// bytes (at most kPinnedBytes) from the device into dst after the system's stream has
// reached this point, through the system's page-locked block
constexpr size_t kPinnedBytes = 256;
pt_status read_small(pt_system* sys, void* dst, const void* d_src, size_t bytes);
// page-locked blocks of kPinnedBytes from a process-wide pool (allocated in chunks and
// kept until exit: freeing page-locked memory can synchronise the device)
void* pinned_block_get();
void pinned_block_put(void* block);
pt_status projection(pt_system* sys, const double2* A, double2* HB, bool fp64 = false);
pt_status orthonormalize(pt_system* sys, const double2* src, double2* dst);
pt_status ace_from_w(pt_system* sys, const double2* psi_src = nullptr);
pt_status exchange_data(pt_system* sys);
pt_status ace_apply(pt_system* sys, const double2* X, int ncols, double2* out, bool fp64 = false);
pt_status observables(pt_system* sys);
pt_status relax(pt_system* sys);
pt_status state_from_psi(pt_system* sys);
pt_status set_kinetic_t(pt_system* sys, double t);
pt_status set_kinetic(pt_system* sys, int64_t n);
// The phases of a PT-CN step (engine.cu): cn_step = cn_begin, then cn_iterate + cn_check
// until done, cn_orthonormalize, the exchange of Psi_{n+1} into wg, cn_complete.
struct StepCtx {
  bool refine = false;      // mixed precision: FP64 refinement below scf_fp64_below
  bool hi = false;          // the next iteration runs in FP64
  bool hi_prev = false;     // the last one did
  bool have_prev = false;   // Anderson has a previous iterate
  bool converged = false;
  bool done = false;
  int it = 0, niter = 0, fixed = 0;
  int outer = 0;            // outer ACE rebuilds done this step
  double drho = 0.0;
  double hres[2] = {0.0, 0.0};   // |R_f|^2 and the density change of the last iteration (device sums)
};
pt_status cn_begin(pt_system* sys, StepCtx* c);
pt_status cn_iterate(pt_system* sys, StepCtx* c);
pt_status cn_check(pt_system* sys, StepCtx* c);
// outer ACE rebuild (ace_outer): when the SCF is done and rebuilds remain, rebuild ACE
// from Psi_f and restart the SCF (*again = true)
pt_status cn_outer(pt_system* sys, StepCtx* c, bool* again);
pt_status cn_orthonormalize(pt_system* sys, StepCtx* c);
pt_status cn_complete(pt_system* sys, StepCtx* c, pt_step_info* info);
pt_status cn_step(pt_system* sys, pt_step_info* info);
pt_status rk4_step(pt_system* sys, pt_step_info* info);
