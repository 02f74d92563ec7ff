// Engine and C ABI (include/pt.h): one PT-CN system on one GPU.
//
// The engine lays the caller's workspace out once (orbitals and their
// Anderson history in the planewave basis, real-space orbitals and exchange
// accumulators, the pair intermediate, tables), then drives the kernels for
//   * the exchange operator V_X Psi (Eq. 3, pair pipeline of fock.cu),
//   * ACE: M = Psi^H W, -M = L L^H, xi = W L^{-H}, K_ACE X = -xi (xi^H X),
//   * H Psi (Eq. 2): kinetic diagonal, local potential by FFT, exchange,
//   * the PT-CN step of Eq. 5 / Alg. 1 with the residual of Alg. 3,
//     per-band Anderson mixing and Cholesky orthonormalisation (Sec. 3.4).
// All device work is enqueued on the caller's stream; host synchronisation
// happens only where a scalar decides control flow (SCF exit, pivots).
#include <cmath>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>
#include <mutex>

#include "pt.h"
#include "common.cuh"
#include "internal.h"
#include "kernels.h"
#include "fft.cuh"

#include <nvtx3/nvToolsExt.h>

using pt::Grid3;

namespace {
// Named range around one phase of a step for profilers (NVTX; header-only, a no-op
// unless a tool is attached). Phases follow the timing rows of the paper's Table 1:
// H Psi, exchange / ACE, residual, Anderson mixing, density, orthonormalisation.
struct Phase {
  explicit Phase(const char* name) { nvtxRangePushA(name); }
  ~Phase() { nvtxRangePop(); }
  Phase(const Phase&) = delete;
  Phase& operator=(const Phase&) = delete;
};
}  // namespace

namespace {

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

}  // namespace

struct pt_system {
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
static thread_local std::string g_last_error = "no error";

// Argument errors of the handle entry points: the message goes to the handle, or to the
// calling thread's handle-less message when the handle itself is NULL.
static pt_status invalid_arg(pt_system* sys, const char* fn, const char* what);

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

// ---------------------------------------------------------------------------
// parameter checks and host tables

static bool supported_n(int n) { return pt::fft_length_supported(n); }

static pt_status check_params(const pt_params* p, std::string* why) {
  if (p == nullptr) { *why = "params is NULL"; return PT_ERR_INVALID; }
  for (int k = 0; k < 3; ++k) {
    if (!supported_n(p->n[k])) { *why = "grid size must be one of 8,12,16,24,32,48,64,96"; return PT_ERR_INVALID; }
    if (!(p->cell[k] > 0.0)) { *why = "cell lengths must be positive"; return PT_ERR_INVALID; }
  }
  if (!(p->ecut > 0.0)) { *why = "ecut must be positive"; return PT_ERR_INVALID; }
  if (p->n_orb < 1) { *why = "n_orb must be >= 1"; return PT_ERR_INVALID; }
  if (p->n_atoms < 0 || (p->n_atoms > 0 && p->atom_frac == nullptr)) { *why = "atoms"; return PT_ERR_INVALID; }
  if (p->anderson_dim < 0 || p->anderson_dim > 20) { *why = "anderson_dim must be in [0, 20]"; return PT_ERR_INVALID; }
  if (p->precision != PT_FP64 && p->precision != PT_MIXED) { *why = "precision"; return PT_ERR_INVALID; }
  if (p->fock_mode != PT_FOCK_EXACT && p->fock_mode != PT_FOCK_ACE) { *why = "fock_mode"; return PT_ERR_INVALID; }
  if (!(p->omega > 0.0)) { *why = "omega must be positive"; return PT_ERR_INVALID; }
  if (p->pair_tile < 0 || p->pair_tile > pt::kTileMax) { *why = "pair_tile must be in [0, 4]"; return PT_ERR_INVALID; }
  if (p->pair_tiles_per_launch < 0) { *why = "pair_tiles_per_launch must be >= 0"; return PT_ERR_INVALID; }
  if (p->scf_max < 1 && p->scf_fixed_iters < 1) { *why = "scf_max or scf_fixed_iters must be >= 1"; return PT_ERR_INVALID; }
  if (p->laser_amp != 0.0 && !(p->laser_duration > 0.0)) { *why = "laser_duration must be positive"; return PT_ERR_INVALID; }
  {
    const bool any = p->n_fock[0] || p->n_fock[1] || p->n_fock[2];
    for (int k = 0; k < 3 && any; ++k)
      if (!supported_n(p->n_fock[k])) { *why = "n_fock must be all 0 or supported grid sizes"; return PT_ERR_INVALID; }
  }
  return PT_OK;
}

static inline int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

static void basis_list(const pt_params* p, std::vector<int>* idx, std::vector<double>* g2out) {
  const int n0 = p->n[0], n1 = p->n[1], n2 = p->n[2];
  idx->clear();
  if (g2out) g2out->clear();
  for (int i0 = 0; i0 < n0; ++i0)
    for (int i1 = 0; i1 < n1; ++i1)
      for (int i2 = 0; i2 < n2; ++i2) {
        const double g0 = 2.0 * M_PI * freq(i0, n0) / p->cell[0];
        const double g1 = 2.0 * M_PI * freq(i1, n1) / p->cell[1];
        const double g2 = 2.0 * M_PI * freq(i2, n2) / p->cell[2];
        const double gg = g0 * g0 + g1 * g1 + g2 * g2;
        if (0.5 * gg <= p->ecut) {
          idx->push_back((i0 * n1 + i1) * n2 + i2);
          if (g2out) g2out->push_back(gg);
        }
      }
}

// The parameters with the Fock grid as the grid (for its basis listing and sizes).
static pt_params fock_params(const pt_params* p) {
  pt_params q = *p;
  if (p->n_fock[0] || p->n_fock[1] || p->n_fock[2])
    for (int k = 0; k < 3; ++k) q.n[k] = p->n_fock[k];
  return q;
}

static bool fock_is_own(const pt_params* p) {
  const pt_params q = fock_params(p);
  return q.n[0] != p->n[0] || q.n[1] != p->n[1] || q.n[2] != p->n[2];
}

static long fock_points(const pt_params* p) {
  const pt_params q = fock_params(p);
  return (long)q.n[0] * q.n[1] * q.n[2];
}

// Twice the largest |g2| over the basis: the reach of pair products along axis 2.
static int pair_g2_reach(const pt_params* p) {
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  int m = 0;
  for (int v : idx) m = std::max(m, std::abs(freq(v % p->n[2], p->n[2])));
  return 2 * m;
}

// Screened kernel K(G) = 4 pi (1 - exp(-G^2 / (4 w^2))) / G^2, K(0) = pi / w^2 (its limit),
// on the grid g in the pair-intermediate layout [i2][i0][i1], scaled by -alpha / N (the
// inverse-FFT factor) so that the pair kernels multiply by it directly (Eq. 3).
static std::vector<double> khat_table(const pt_params* p, Grid3 g) {
  const int n0 = g.n0, n1 = g.n1, n2 = g.n2;
  const double w2 = p->omega * p->omega;
  const double scale = -p->alpha / (double)g.N();
  std::vector<double> kt((size_t)g.N());
  for (int i2 = 0; i2 < n2; ++i2)
    for (int i0 = 0; i0 < n0; ++i0)
      for (int i1 = 0; i1 < n1; ++i1) {
        const double g0 = 2.0 * M_PI * freq(i0, n0) / p->cell[0];
        const double g1 = 2.0 * M_PI * freq(i1, n1) / p->cell[1];
        const double gz = 2.0 * M_PI * freq(i2, n2) / p->cell[2];
        const double gg = g0 * g0 + g1 * g1 + gz * gz;
        const double k = gg > 0.0 ? 4.0 * M_PI * (-std::expm1(-gg / (4.0 * w2))) / gg : M_PI / w2;
        kt[((size_t)i2 * n0 + i0) * n1 + i1] = scale * k;
      }
  return kt;
}

// Uploads the twiddle tables (FP64 and FP32) and the kernel table of grid g in the
// exchange precision; synchronises the stream before the host vectors go away.
static cudaError_t upload_fft_tables(const pt_params* p, Grid3 g, bool mixed, double2* tw64, float2* tw32,
                                     double* khat64, float* khat32, cudaStream_t s) {
  std::vector<double2> tw(pt::kTwiddleTotal);
  pt::twiddle_host(tw.data());
  std::vector<float2> twf(pt::kTwiddleTotal);
  for (int k = 0; k < pt::kTwiddleTotal; ++k) twf[k] = make_float2((float)tw[k].x, (float)tw[k].y);
  const std::vector<double> kt = khat_table(p, g);
  std::vector<float> kf;
  cudaError_t e = cudaMemcpyAsync(tw64, tw.data(), sizeof(double2) * tw.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tw32, twf.data(), sizeof(float2) * twf.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    if (mixed) {
      kf.resize(kt.size());
      for (size_t k = 0; k < kt.size(); ++k) kf[k] = (float)kt[k];
      e = cudaMemcpyAsync(khat32, kf.data(), sizeof(float) * kf.size(), cudaMemcpyHostToDevice, s);
    } else {
      e = cudaMemcpyAsync(khat64, kt.data(), sizeof(double) * kt.size(), cudaMemcpyHostToDevice, s);
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  return e != cudaSuccess ? e : e2;
}

static int choose_tile(const pt_params* p) {
  if (p->pair_tile > 0) return p->pair_tile;
  return std::min(pt::kTileMax, p->n_orb);
}

static int tiles_per_launch(const pt_params* p, long N, bool mixed) {
  const int tile = choose_tile(p);
  const int nb = (p->n_orb + tile - 1) / tile;
  const double per_tile = (double)pt::kTileMax * pt::kTileMax * N * (mixed ? 8.0 : 16.0);
  const double budget = 16.0e9;
  int cap = (int)std::max(1.0, std::floor(budget / per_tile));
  if (p->pair_tiles_per_launch > 0) cap = std::min(cap, p->pair_tiles_per_launch);
  return std::max(1, std::min(nb, cap));
}

static int h_batch(const pt_params* p) { return std::min(p->n_orb, 32); }

// Carve (or size, when base == 0) the workspace.
static size_t carve(pt_system* sys, const pt_params* p, uintptr_t base) {
  Carver c{base};
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  const long npw = (long)idx.size();
  const long N = (long)p->n[0] * p->n[1] * p->n[2];
  const long ne = p->n_orb;
  const int m = p->anderson_dim;
  const bool mixed = p->precision == PT_MIXED;
  const size_t cs = mixed ? sizeof(float2) : sizeof(double2);
  const int tile = choose_tile(p);
  const long nb = (ne + tile - 1) / tile;
  const long Nf = fock_points(p);
  const bool own = fock_is_own(p);
  const int tpl = tiles_per_launch(p, Nf, mixed);
  const int hb = h_batch(p);
  pt_system dummy;
  pt_system* t = sys ? sys : &dummy;
  t->basis = c.take<int>(npw);
  t->kin = c.take<double>(npw);
  t->gk3 = c.take<double>(3 * (size_t)npw);
  t->tw64 = c.take<double2>(pt::kTwiddleTotal);
  t->tw32 = c.take<float2>(pt::kTwiddleTotal);
  if (mixed) t->khat32 = c.take<float>(Nf); else t->khat64 = c.take<double>(Nf);
  t->hfac = c.take<double>(N);
  t->kfac = c.take<double>(N);
  t->rho_mix = c.take<double>(N);
  t->vion = c.take<double>(N);
  t->vloc = c.take<double>(N);
  if (mixed) t->vloc32 = c.take<float>(N);
  t->vh = c.take<double>(N);
  t->rho = c.take<double>(N);
  t->rho2 = c.take<double>(N);
  t->d_atoms = c.take<double>(3 * std::max(1, p->n_atoms));
  const size_t pe = (size_t)npw * ne;
  t->psi = c.take<double2>(pe);
  t->psi_half = c.take<double2>(pe);
  t->psi_f = c.take<double2>(pe);
  t->hpsi = c.take<double2>(pe);
  t->tmp = c.take<double2>(pe);
  t->rbuf = c.take<double2>(pe);
  t->wg = c.take<double2>(pe);
  t->xi = c.take<double2>(pe);
  t->xprev = c.take<double2>(pe);
  t->rprev = c.take<double2>(pe);
  const size_t hs = mixed ? sizeof(float2) : sizeof(double2);
  t->dX = c.take<unsigned char>(pe * std::max(1, m) * hs);
  t->dR = c.take<unsigned char>(pe * std::max(1, m) * hs);
  t->hbuf = c.take<double2>((size_t)N * hb);
  t->psi_r = c.take<double2>((size_t)N * ne);
  if (mixed) t->psi_r32 = c.take<float2>((size_t)N * ne);
  {
    const long L0 = p->n[0], L1 = p->n[1];
    t->sph_row_idx = c.take<int>(L0 * L1);
    t->sph_row_kbeg = c.take<int>(L0 * L1 + 1);
    t->sph_krow = c.take<int>(npw);
    t->sph_planes = c.take<int>(L0);
    t->sph_rowlive = c.take<unsigned char>(L0 * L1);
    t->sph_planelive = c.take<unsigned char>(L0);
  }
  if (mixed) {
    t->xi32 = c.take<float2>(pe);
    t->ga32 = c.take<float2>(pe);
    t->gb32 = c.take<float2>(pe);
    t->gs32 = c.take<float2>(ne * ne);
  }
  t->w_r = c.take<unsigned char>((size_t)Nf * ne * cs);
  t->x_r = c.take<unsigned char>((size_t)Nf * ne * cs);
  t->scratch = c.take<unsigned char>((size_t)tpl * pt::kTileMax * pt::kTileMax * Nf * cs);
  if (own) {
    const pt_params q = fock_params(p);
    const long L0 = q.n[0], L1 = q.n[1];
    t->basis_f = c.take<int>(npw);
    t->psi_rf = c.take<unsigned char>((size_t)Nf * ne * cs);
    t->sphf_row_idx = c.take<int>(L0 * L1);
    t->sphf_row_kbeg = c.take<int>(L0 * L1 + 1);
    t->sphf_krow = c.take<int>(npw);
    t->sphf_planes = c.take<int>(L0);
    t->sphf_rowlive = c.take<unsigned char>(L0 * L1);
    t->sphf_planelive = c.take<unsigned char>(L0);
  }
  t->S = c.take<double2>(ne * ne);
  t->Mneg = c.take<double2>(ne * ne);
  t->Linv = c.take<double2>(ne * ne);
  t->Z = c.take<double2>(ne * ne);
  t->gemm_ws_elems = (size_t)16 * ne * ne + 4096;
  t->gemm_ws = c.take<double2>(t->gemm_ws_elems);
  t->gram = c.take<double2>((size_t)ne * std::max(1, m) * std::max(1, m));
  t->rhs = c.take<double2>((size_t)ne * std::max(1, m));
  t->gamma = c.take<double2>((size_t)ne * std::max(1, m));
  t->part = c.take<double>(8192);
  t->red = c.take<double>(64);
  t->status = c.take<int>(16);
  t->d_tiles_sym = c.take<pt::PairTile>((size_t)(nb * (nb - 1) / 2 + nb));
  t->max_tiles_x = (size_t)nb * nb;
  t->d_tiles_x = c.take<pt::PairTile>(t->max_tiles_x);
  return c.off + 256;
}

// ---------------------------------------------------------------------------
// building blocks

static const float2* tw_for(pt_system* sys, int L, float*) { return sys->tw32 + pt::twiddle_offset(L); }
static const double2* tw_for(pt_system* sys, int L, double*) { return sys->tw64 + pt::twiddle_offset(L); }

// A grid the orbital transforms run on: the main grid (density, local potential) or
// the Fock grid of the pair FFTs.
struct GridView {
  Grid3 g;
  long N;
  const int* basis;
  bool use_sphere;
  const pt::SphereTables* sph;
};
static GridView main_grid(pt_system* sys) { return GridView{sys->g, sys->N, sys->basis, sys->use_sphere, &sys->sph}; }
static GridView fock_grid(pt_system* sys) {
  if (!sys->fock_own) return main_grid(sys);
  return GridView{sys->gf, sys->Nf, sys->basis_f, sys->use_sphere_f, &sys->sphf};
}

// real-space form (scale Omega^{-1/2}) of ncols basis-coefficient columns c on grid v
template <typename T>
static pt_status to_real(pt_system* sys, const GridView& v, const double2* c, long ncols, void* dst) {
  if (v.use_sphere) {
    PT_CK(pt::sphere_to_real(c, sys->npw, (pt::cplx<T>*)dst, ncols, v.g, *v.sph, v.basis, 1.0 / std::sqrt(sys->vol),
                             tw_for(sys, v.g.n0, (T*)nullptr), sys->s));
    return PT_OK;
  }
  PT_CK(pt::scatter_basis<T>(c, sys->npw, dst, ncols, v.g, v.basis, sys->npw, 1.0 / std::sqrt(sys->vol), sys->s));
  PT_CK(pt::fft_rows<T>(dst, dst, ncols, v.g, 1, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<T>(dst, ncols, v.g, 1, 1, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<T>(dst, ncols, v.g, 0, 1, 0, 1.0, nullptr, sys->tw, sys->s));
  return PT_OK;
}

template <typename T>
static pt_status to_real(pt_system* sys, const double2* c, long ncols, void* dst) {
  return to_real<T>(sys, main_grid(sys), c, ncols, dst);
}

// forward transform of src on grid v (destroyed) and gather into out (scale sqrt(Omega)/N_v)
template <typename T>
static pt_status to_basis(pt_system* sys, const GridView& v, void* src, long ncols, double2* out, int accumulate,
                          const double* kin, const double2* x) {
  if (v.use_sphere) {
    PT_CK(pt::sphere_from_real((const pt::cplx<T>*)src, (const T*)nullptr, (pt::cplx<T>*)src, ncols, v.g, *v.sph,
                               v.basis, std::sqrt(sys->vol) / v.N, kin, x, sys->npw, out, sys->npw, accumulate,
                               tw_for(sys, v.g.n0, (T*)nullptr), sys->s));
    return PT_OK;
  }
  PT_CK(pt::fft_rows<T>(src, src, ncols, v.g, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<T>(src, ncols, v.g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<T>(src, ncols, v.g, 0, 0, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::gather_basis<T>(src, out, sys->npw, ncols, v.g, v.basis, sys->npw, std::sqrt(sys->vol) / v.N, kin, x,
                            sys->npw, accumulate, sys->s));
  return PT_OK;
}

// psi_r (and its FP32 copy) <- real-space form of the columns c (n_orb of them)
static pt_status real_orbitals(pt_system* sys, const double2* c) {
  PT_TRY(to_real<double>(sys, c, sys->ne, sys->psi_r));
  if (sys->mixed) PT_CK(pt::convert_c128_to_c64(sys->psi_r, sys->psi_r32, sys->N * sys->ne, sys->s));
  return PT_OK;
}

static pt_status local_potential(pt_system* sys, const double* rho) {
  const int use_h = sys->p.use_hartree ? 1 : 0;
  if (use_h) {
    PT_CK(pt::rho_to_complex(rho, sys->hbuf, sys->N, sys->s));
    PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, 1, sys->g, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 0, 0, 2, 1.0, sys->hfac, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 1, 1, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, 1, sys->g, 1, 1.0, nullptr, sys->tw, sys->s));
  }
  const double w_lda = sys->p.use_lda ? (1.0 - sys->p.alpha) : 0.0;
  PT_CK(pt::assemble_vloc(sys->vion, sys->hbuf, rho, sys->N, use_h, w_lda, sys->vh, sys->vloc, sys->s));
  return PT_OK;
}

static pt_status local_potential(pt_system* sys) { return local_potential(sys, sys->rho); }

// rho_mix += F^-1[ b |G|^2/(|G|^2 + q0^2) F[rho - rho_mix] ]
static pt_status kerker_mix(pt_system* sys) {
  PT_CK(pt::diff_to_complex(sys->rho, sys->rho_mix, sys->hbuf, sys->N, sys->s));
  PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, 1, sys->g, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 0, 0, 2, 1.0, sys->kfac, sys->tw, sys->s));
  PT_CK(pt::fft_cols<double>(sys->hbuf, 1, sys->g, 1, 1, 0, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, 1, sys->g, 1, 1.0, nullptr, sys->tw, sys->s));
  PT_CK(pt::add_real(sys->hbuf, sys->rho_mix, sys->N, sys->s));
  return PT_OK;
}

// out = kin * c + local(vloc) c, using the real-space form psi_r of the n_orb columns c
static pt_status apply_local_from_real(pt_system* sys, const double2* c, double2* out) {
  for (int c0 = 0; c0 < sys->ne; c0 += sys->hb) {
    const int cnt = std::min(sys->hb, sys->ne - c0);
    if (sys->use_sphere) {
      PT_CK(pt::sphere_from_real(sys->psi_r + (long)c0 * sys->N, sys->vloc, sys->hbuf, cnt, sys->g, sys->sph,
                                 sys->basis, std::sqrt(sys->vol) / sys->N, sys->kin, c + (long)c0 * sys->npw, sys->npw,
                                 out + (long)c0 * sys->npw, sys->npw, 0, tw_for(sys, sys->g.n0, (double*)nullptr),
                                 sys->s));
      continue;
    }
    PT_CK(pt::fft_rows<double>(sys->psi_r + (long)c0 * sys->N, sys->hbuf, cnt, sys->g, 0, 1.0, sys->vloc, sys->tw,
                               sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, cnt, sys->g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, cnt, sys->g, 0, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::gather_basis<double>(sys->hbuf, out + (long)c0 * sys->npw, sys->npw, cnt, sys->g, sys->basis, sys->npw,
                                   std::sqrt(sys->vol) / sys->N, sys->kin, c + (long)c0 * sys->npw, sys->npw, 0,
                                   sys->s));
  }
  return PT_OK;
}

// out = kin * X + local(vloc) X for arbitrary columns X
static pt_status apply_local(pt_system* sys, const double2* X, double2* out, int ncols) {
  for (int c0 = 0; c0 < ncols; c0 += sys->hb) {
    const int cnt = std::min(sys->hb, ncols - c0);
    PT_CK(pt::scatter_basis<double>(X + (long)c0 * sys->npw, sys->npw, sys->hbuf, cnt, sys->g, sys->basis, sys->npw,
                                    1.0 / std::sqrt(sys->vol), sys->s));
    PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, cnt, sys->g, 1, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, cnt, sys->g, 1, 1, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, cnt, sys->g, 0, 1, 1, 1.0, sys->vloc, sys->tw, sys->s));
    PT_CK(pt::fft_cols<double>(sys->hbuf, cnt, sys->g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_rows<double>(sys->hbuf, sys->hbuf, cnt, sys->g, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::gather_basis<double>(sys->hbuf, out + (long)c0 * sys->npw, sys->npw, cnt, sys->g, sys->basis, sys->npw,
                                   std::sqrt(sys->vol) / sys->N, sys->kin, X + (long)c0 * sys->npw, sys->npw, 0,
                                   sys->s));
  }
  return PT_OK;
}

// Real-space orbitals of the coefficients `coef` (n_orb columns) on the Fock grid in the
// exchange precision: when the Fock grid is the main grid these are psi_r32 / psi_r, which
// the caller keeps current for `coef`; otherwise they are transformed here.
template <typename T>
static pt_status fock_orbitals(pt_system* sys, const double2* coef, const void** out) {
  if (!sys->fock_own) {
    *out = sys->mixed ? (const void*)sys->psi_r32 : (const void*)sys->psi_r;
    return PT_OK;
  }
  PT_TRY(to_real<T>(sys, fock_grid(sys), coef, sys->ne, sys->psi_rf));
  *out = sys->psi_rf;
  return PT_OK;
}

// V_X Psi for the orbitals Psi = coef (Eq. 3 on the Fock grid); out = (or +=) result
template <typename T>
static pt_status exchange_sym_t(pt_system* sys, const double2* coef, double2* out, int accumulate) {
  const size_t cs = sizeof(pt::cplx<T>);
  const GridView fv = fock_grid(sys);
  const void* pr = nullptr;
  PT_TRY(fock_orbitals<T>(sys, coef, &pr));
  PT_CK(cudaMemsetAsync(sys->w_r, 0, cs * fv.N * sys->ne, sys->s));
  const T* kt = sys->mixed ? (const T*)(const void*)sys->khat32 : (const T*)(const void*)sys->khat64;
  if (sys->timing) PT_CK(cudaEventRecord(sys->ev0, sys->s));
  PT_CK(pt::fock_pairs<T>(pr, nullptr, sys->w_r, nullptr, sys->plan_sym, 1, fv.g, kt, sys->scratch, sys->tw, sys->s));
  if (sys->timing) {
    PT_CK(cudaEventRecord(sys->ev1, sys->s));
    PT_CK(cudaEventSynchronize(sys->ev1));
    float ms = 0.f;
    PT_CK(cudaEventElapsedTime(&ms, sys->ev0, sys->ev1));
    sys->t_pair_ms += ms;
    sys->t_pairs += (long long)sys->ne * (sys->ne + 1) / 2;
    sys->t_groups += sys->plan_sym.n_launch;
  }
  return to_basis<T>(sys, fv, sys->w_r, sys->ne, out, accumulate, nullptr, nullptr);
}

static pt_status exchange_sym(pt_system* sys, const double2* coef, double2* out, int accumulate) {
  if (sys->p.alpha == 0.0) {
    if (!accumulate) PT_CK(cudaMemsetAsync(out, 0, sizeof(double2) * sys->npw * sys->ne, sys->s));
    return PT_OK;
  }
  return sys->mixed ? exchange_sym_t<float>(sys, coef, out, accumulate)
                    : exchange_sym_t<double>(sys, coef, out, accumulate);
}

static pt_status ensure_plan_x(pt_system* sys, int ncols) {
  if (sys->plan_x_ncols == ncols) return PT_OK;
  pt::PairTile* tiles = nullptr;
  int *lf = nullptr, *lc = nullptr, nl = 0;
  const int tile = choose_tile(&sys->p);
  const int nt = pt::fock_build_tiles(sys->ne, ncols, tile, 0, tiles_per_launch(&sys->p, sys->Nf, sys->mixed), &tiles,
                                      &lf, &lc, &nl);
  if (nt < 0 || (size_t)nt > sys->max_tiles_x) {
    std::free(tiles); std::free(lf); std::free(lc);
    sys->err = "exchange tile schedule does not fit";
    return PT_ERR_INVALID;
  }
  PT_CK(cudaMemcpyAsync(sys->d_tiles_x, tiles, sizeof(pt::PairTile) * nt, cudaMemcpyHostToDevice, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  std::free(tiles);
  std::free(sys->plan_x.launch_first);
  std::free(sys->plan_x.launch_count);
  sys->plan_x.tile = tile;
  sys->plan_x.tiles_per_launch = tiles_per_launch(&sys->p, sys->Nf, sys->mixed);
  sys->plan_x.n_launch = nl;
  sys->plan_x.launch_first = lf;
  sys->plan_x.launch_count = lc;
  sys->plan_x.d_tiles = sys->d_tiles_x;
  sys->plan_x.n_tiles = nt;
  sys->plan_x.g2_reach = pair_g2_reach(&sys->p);
  sys->plan_x_ncols = ncols;
  return PT_OK;
}

template <typename T>
static pt_status exchange_x_t(pt_system* sys, const double2* X, int ncols, double2* out) {
  const size_t cs = sizeof(pt::cplx<T>);
  const GridView fv = fock_grid(sys);
  PT_TRY(ensure_plan_x(sys, ncols));
  PT_TRY(to_real<T>(sys, fv, X, ncols, sys->x_r));
  PT_CK(cudaMemsetAsync(sys->w_r, 0, cs * fv.N * ncols, sys->s));
  const void* pr = nullptr;
  PT_TRY(fock_orbitals<T>(sys, sys->psi, &pr));
  const T* kt = sys->mixed ? (const T*)(const void*)sys->khat32 : (const T*)(const void*)sys->khat64;
  PT_CK(pt::fock_pairs<T>(pr, sys->x_r, nullptr, sys->w_r, sys->plan_x, 0, fv.g, kt, sys->scratch, sys->tw, sys->s));
  return to_basis<T>(sys, fv, sys->w_r, ncols, out, 1, nullptr, nullptr);
}

template <typename Tc>
static pt_status gemm(pt_system* sys, int opA, int opB, int M, int N, int K, double2 alpha, const double2* A, long lda,
                      const double2* B, long ldb, double2 beta, double2* C, long ldc,
                      int structure = pt::GEMM_GENERAL) {
  PT_CK(pt::gemm<Tc>(opA, opB, M, N, K, alpha, A, lda, 0, B, ldb, 0, beta, C, ldc, 0, 1, sys->gemm_ws,
                     sys->gemm_ws_elems, sys->s, structure));
  return PT_OK;
}

static const double2 kOne = {1.0, 0.0}, kZero = {0.0, 0.0}, kMinusOne = {-1.0, 0.0};

// FP32 product of complex64 copies (mixed precision); C stays complex128.
static pt_status gemm32(pt_system* sys, int opA, int opB, int M, int N, int K, double2 alpha, const float2* A, long lda,
                        const float2* B, long ldb, double2 beta, double2* C, long ldc,
                        int structure = pt::GEMM_GENERAL) {
  PT_CK(pt::gemm_c64(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sys->gemm_ws, sys->gemm_ws_elems, sys->s,
                     structure));
  return PT_OK;
}

static pt_status to32(pt_system* sys, const double2* src, float2* dst, long n) {
  PT_CK(pt::convert_c128_to_c64(src, dst, n, sys->s));
  return PT_OK;
}

// SCF-iteration forms. In mixed precision the real-space orbitals, the
// density they give and the local-potential product run in FP32; in FP64
// mode these are the FP64 routines above.
static pt_status real_orbitals_scf(pt_system* sys, const double2* c) {
  if (!sys->mixed) return real_orbitals(sys, c);
  return to_real<float>(sys, c, sys->ne, sys->psi_r32);
}

static pt_status density_scf(pt_system* sys, double* rho) {
  if (sys->mixed) PT_CK(pt::density32(sys->psi_r32, sys->N, sys->ne, rho, sys->s));
  else PT_CK(pt::density(sys->psi_r, sys->N, sys->ne, rho, sys->s));
  return PT_OK;
}

static pt_status apply_local_scf(pt_system* sys, const double2* c, double2* out) {
  if (!sys->mixed) return apply_local_from_real(sys, c, out);
  PT_CK(pt::to_float(sys->vloc, sys->vloc32, sys->N, sys->s));
  float2* hb = reinterpret_cast<float2*>(sys->hbuf);
  for (int c0 = 0; c0 < sys->ne; c0 += sys->hb) {
    const int cnt = std::min(sys->hb, sys->ne - c0);
    if (sys->use_sphere) {
      PT_CK(pt::sphere_from_real(sys->psi_r32 + (long)c0 * sys->N, sys->vloc32, hb, cnt, sys->g, sys->sph, sys->basis,
                                 std::sqrt(sys->vol) / sys->N, sys->kin, c + (long)c0 * sys->npw, sys->npw,
                                 out + (long)c0 * sys->npw, sys->npw, 0, tw_for(sys, sys->g.n0, (float*)nullptr),
                                 sys->s));
      continue;
    }
    PT_CK(pt::fft_rows<float>(sys->psi_r32 + (long)c0 * sys->N, hb, cnt, sys->g, 0, 1.0, sys->vloc32, sys->tw, sys->s));
    PT_CK(pt::fft_cols<float>(hb, cnt, sys->g, 1, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::fft_cols<float>(hb, cnt, sys->g, 0, 0, 0, 1.0, nullptr, sys->tw, sys->s));
    PT_CK(pt::gather_basis<float>(hb, out + (long)c0 * sys->npw, sys->npw, cnt, sys->g, sys->basis, sys->npw,
                                  std::sqrt(sys->vol) / sys->N, sys->kin, c + (long)c0 * sys->npw, sys->npw, 0,
                                  sys->s));
  }
  return PT_OK;
}

// S = A^H B and C -= A S (the PT projection, Alg. 3): FP32 in mixed precision
static pt_status projection(pt_system* sys, const double2* A, double2* HB) {
  const int ne = sys->ne, npw = sys->npw;
  if (sys->mixed) {
    PT_TRY(to32(sys, A, sys->ga32, (long)npw * ne));
    PT_TRY(to32(sys, HB, sys->gb32, (long)npw * ne));
    PT_TRY(gemm32(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kOne, sys->ga32, npw, sys->gb32, npw, kZero, sys->S, ne));
    PT_TRY(to32(sys, sys->S, sys->gs32, (long)ne * ne));
    PT_TRY(gemm32(sys, pt::OP_N, pt::OP_N, npw, ne, ne, kMinusOne, sys->ga32, npw, sys->gs32, ne, kOne, HB, npw));
  } else {
    PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kOne, A, npw, HB, npw, kZero, sys->S, ne));
    PT_TRY(gemm<double>(sys, pt::OP_N, pt::OP_N, npw, ne, ne, kMinusOne, A, npw, sys->S, ne, kOne, HB, npw));
  }
  return PT_OK;
}

static pt_status read_status(pt_system* sys, int* h) {
  PT_CK(cudaMemcpyAsync(h, sys->status, sizeof(int), cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

// dst = src L^{-H}, L L^H = src^H src  (Sec. 3.4)
static pt_status orthonormalize(pt_system* sys, const double2* src, double2* dst) {
  Phase phase_("orthonormalize");
  const int ne = sys->ne, npw = sys->npw;
  PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kOne, src, npw, src, npw, kZero, sys->S, ne,
                      pt::GEMM_HERM));
  PT_CK(pt::cholesky(sys->S, ne, sys->status, sys->s));
  int h = 0;
  PT_TRY(read_status(sys, &h));
  if (h != 0) { sys->err = "orthonormalisation: overlap matrix is not positive definite"; return PT_ERR_NOT_PD; }
  PT_CK(pt::tri_inverse(sys->S, sys->Linv, ne, sys->s));
  PT_TRY(gemm<double>(sys, pt::OP_N, pt::OP_H, npw, ne, ne, kOne, src, npw, sys->Linv, ne, kZero, dst, npw,
                      pt::GEMM_TRI_B));
  return PT_OK;
}

// ACE data of the current (psi, wg): Mneg = -Psi^H W; Cholesky -M = L L^H;
// xi = W L^{-H} (ACE construction following Eq. 3 and the ACE definition).
static pt_status ace_from_w(pt_system* sys) {
  const int ne = sys->ne, npw = sys->npw;
  const bool ace = sys->p.fock_mode == PT_FOCK_ACE && sys->p.alpha != 0.0;
  if (sys->mixed && ace) {
    PT_TRY(to32(sys, sys->psi, sys->ga32, (long)npw * ne));
    PT_TRY(to32(sys, sys->wg, sys->gb32, (long)npw * ne));
    PT_TRY(gemm32(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kMinusOne, sys->ga32, npw, sys->gb32, npw, kZero, sys->Mneg, ne));
  } else
    PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kMinusOne, sys->psi, npw, sys->wg, npw, kZero, sys->Mneg, ne));
  sys->have_ace = false;
  if (!ace) return PT_OK;
  PT_CK(cudaMemcpyAsync(sys->S, sys->Mneg, sizeof(double2) * ne * ne, cudaMemcpyDeviceToDevice, sys->s));
  PT_CK(pt::cholesky(sys->S, ne, sys->status, sys->s));
  int h = 0;
  PT_TRY(read_status(sys, &h));
  if (h != 0) { sys->err = "ACE: -M is not positive definite"; return PT_ERR_NOT_PD; }
  PT_CK(pt::tri_inverse(sys->S, sys->Linv, ne, sys->s));
  if (sys->mixed) {
    // W is still in gb32; xi and its complex64 copy for the FP32 ACE products
    PT_TRY(to32(sys, sys->Linv, sys->gs32, (long)ne * ne));
    PT_TRY(gemm32(sys, pt::OP_N, pt::OP_H, npw, ne, ne, kOne, sys->gb32, npw, sys->gs32, ne, kZero, sys->xi, npw,
                  pt::GEMM_TRI_B));
    PT_TRY(to32(sys, sys->xi, sys->xi32, (long)npw * ne));
  } else
    PT_TRY(gemm<double>(sys, pt::OP_N, pt::OP_H, npw, ne, ne, kOne, sys->wg, npw, sys->Linv, ne, kZero, sys->xi, npw,
                        pt::GEMM_TRI_B));
  sys->have_ace = true;
  return PT_OK;
}

// exchange data of psi (psi_r current): wg = V_X psi, then its ACE data
static pt_status exchange_data(pt_system* sys) {
  Phase phase_("exchange + ACE build");
  PT_TRY(exchange_sym(sys, sys->psi, sys->wg, 0));
  return ace_from_w(sys);
}

// out += -xi (xi^H X)
static pt_status ace_apply(pt_system* sys, const double2* X, int ncols, double2* out) {
  const int ne = sys->ne, npw = sys->npw;
  if (sys->mixed) {
    PT_TRY(to32(sys, X, sys->ga32, (long)npw * ncols));
    PT_TRY(gemm32(sys, pt::OP_H, pt::OP_N, ne, ncols, npw, kOne, sys->xi32, npw, sys->ga32, npw, kZero, sys->Z, ne));
    PT_TRY(to32(sys, sys->Z, sys->gs32, (long)ne * ncols));
    PT_TRY(gemm32(sys, pt::OP_N, pt::OP_N, npw, ncols, ne, kMinusOne, sys->xi32, npw, sys->gs32, ne, kOne, out, npw));
  } else {
    PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ncols, npw, kOne, sys->xi, npw, X, npw, kZero, sys->Z, ne));
    PT_TRY(gemm<double>(sys, pt::OP_N, pt::OP_N, npw, ncols, ne, kMinusOne, sys->xi, npw, sys->Z, ne, kOne, out, npw));
  }
  return PT_OK;
}

// energy and dipole of psi (psi_r current, Mneg current)
static pt_status observables(pt_system* sys) {
  PT_CK(pt::density(sys->psi_r, sys->N, sys->ne, sys->rho, sys->s));
  PT_TRY(local_potential(sys));
  PT_CK(pt::energy_sums(sys->rho, sys->vion, sys->vh, sys->p.use_hartree ? 1 : 0, sys->g, sys->p.cell, sys->psi,
                        sys->kin, sys->npw, sys->ne, sys->Mneg, sys->part, sys->red + 8, sys->s));
  double h[8];
  PT_CK(cudaMemcpyAsync(h, sys->red + 8, sizeof(h), cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  const double dV = sys->dV;
  double e = 2.0 * h[6] + dV * h[0];
  if (sys->p.use_hartree) e += 0.5 * dV * h[1];
  if (sys->p.use_lda) e += (1.0 - sys->p.alpha) * (-kSlater * std::cbrt(3.0 / M_PI)) * dV * h[2];
  e += -h[7];
  sys->energy = e;
  for (int k = 0; k < 3; ++k) sys->dipole[k] = -dV * h[3 + k];
  return PT_OK;
}

// relaxation of the start state: psi <- orth(psi - tau P (H_loc psi - psi S))
static pt_status relax(pt_system* sys) {
  Phase phase_("relax start state");
  const int ne = sys->ne, npw = sys->npw;
  const long n = (long)npw * ne;
  if (sys->p.relax_iters > 0) {
    PT_TRY(real_orbitals(sys, sys->psi));
    PT_CK(pt::density(sys->psi_r, sys->N, ne, sys->rho_mix, sys->s));
  }
  for (int k = 0; k < sys->p.relax_iters; ++k) {
    PT_TRY(real_orbitals(sys, sys->psi));
    PT_CK(pt::density(sys->psi_r, sys->N, ne, sys->rho, sys->s));
    PT_TRY(kerker_mix(sys));
    PT_TRY(local_potential(sys, sys->rho_mix));
    PT_TRY(apply_local_from_real(sys, sys->psi, sys->hpsi));
    PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kOne, sys->psi, npw, sys->hpsi, npw, kZero, sys->S, ne));
    PT_TRY(gemm<double>(sys, pt::OP_N, pt::OP_N, npw, ne, ne, kMinusOne, sys->psi, npw, sys->S, ne, kOne, sys->hpsi, npw));
    PT_CK(pt::precond_step(sys->psi, sys->hpsi, sys->kin, npw, n, sys->p.relax_tau, sys->s));
    PT_TRY(orthonormalize(sys, sys->psi, sys->psi_f));
    std::swap(sys->psi, sys->psi_f);
  }
  return PT_OK;
}

static pt_status state_from_psi(pt_system* sys) {
  Phase phase_("new state");
  PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  PT_TRY(exchange_data(sys));
  PT_TRY(observables(sys));
  return PT_OK;
}

// Laser vector potential A(t) (velocity gauge; pulse shape as stated in pt.h).
static void laser_field(const pt_params* p, double t, double a[3]) {
  a[0] = a[1] = a[2] = 0.0;
  if (p->laser_amp == 0.0 || t < 0.0 || t > p->laser_duration) return;
  const double s = std::sin(M_PI * t / p->laser_duration);
  const double f = p->laser_amp * s * s * std::sin(p->laser_omega * t);
  for (int k = 0; k < 3; ++k) a[k] = f * p->laser_dir[k];
}

// kinetic diagonal |G + kick + A(t)|^2 / 2 at time t (only with the laser on; otherwise
// the kick-only table of the start stays)
static pt_status set_kinetic_t(pt_system* sys, double t) {
  if (sys->p.laser_amp == 0.0) return PT_OK;
  double a[3];
  laser_field(&sys->p, t, a);
  PT_CK(pt::kinetic_shifted(sys->gk3, sys->npw, a[0], a[1], a[2], sys->kin, sys->s));
  return PT_OK;
}

static pt_status set_kinetic(pt_system* sys, int64_t n) { return set_kinetic_t(sys, (double)n * sys->p.dt); }

// one PT-CN step (Eq. 5, Alg. 1)
static pt_status cn_step(pt_system* sys, pt_step_info* info) {
  Phase phase_("PT-CN step");
  const int ne = sys->ne, npw = sys->npw;
  const long n = (long)npw * ne;
  const double hdt = 0.5 * sys->p.dt;
  const int m = sys->p.anderson_dim;
  const long stride = n;
  if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
  // initial residual R_n = H_n Psi_n - Psi_n (Psi_n^H H_n Psi_n) and the half step (H_n at t_n)
  PT_TRY(set_kinetic(sys, sys->n_step));
  PT_TRY(density_scf(sys, sys->rho));
  PT_TRY(local_potential(sys));
  PT_TRY(apply_local_scf(sys, sys->psi, sys->hpsi));
  PT_CK(pt::axpy(kOne, sys->wg, sys->hpsi, n, sys->s));
  PT_TRY(projection(sys, sys->psi, sys->hpsi));
  PT_CK(pt::half_step(sys->psi, sys->hpsi, hdt, sys->psi_half, n, sys->s));
  // the SCF loop and the observables of Psi_{n+1} use H at t_{n+1}
  PT_TRY(set_kinetic(sys, sys->n_step + 1));
  PT_CK(cudaMemcpyAsync(sys->psi_f, sys->psi_half, sizeof(double2) * n, cudaMemcpyDeviceToDevice, sys->s));
  PT_TRY(real_orbitals_scf(sys, sys->psi_f));
  sys->psi_r_current = false;
  PT_TRY(density_scf(sys, sys->rho));
  // SCF loop
  const int fixed = sys->p.scf_fixed_iters;
  const int niter = fixed > 0 ? fixed : sys->p.scf_max;
  sys->and_count = 0;
  sys->and_order.clear();
  bool have_prev = false;
  bool converged = false;
  int it = 0;
  double drho = 0.0;
  for (it = 1; it <= niter; ++it) {
    Phase iter_("SCF iteration");
    {
      Phase p_("H Psi");
      PT_TRY(local_potential(sys));
      PT_TRY(apply_local_scf(sys, sys->psi_f, sys->hpsi));
      if (sys->p.alpha != 0.0) {
        Phase x_(sys->p.fock_mode == PT_FOCK_EXACT ? "exchange" : "ACE apply");
        if (sys->p.fock_mode == PT_FOCK_EXACT) PT_TRY(exchange_sym(sys, sys->psi_f, sys->hpsi, 1));
        else PT_TRY(ace_apply(sys, sys->psi_f, ne, sys->hpsi));
      }
    }
    {
      Phase p_("PT residual");
      PT_TRY(projection(sys, sys->psi_f, sys->hpsi));
      PT_CK(pt::pt_residual(sys->psi_f, sys->hpsi, sys->psi_half, hdt, sys->rbuf, n, sys->part, sys->red + 0, sys->s));
    }
    // Anderson (per band)
    {
      Phase and_("Anderson");
      int newslot = -1;
      if (have_prev && m > 0) {
        if (sys->and_count < m) {
          newslot = sys->and_count;
          sys->and_count++;
        } else {
          newslot = sys->and_order.front();
          sys->and_order.erase(sys->and_order.begin());
        }
        sys->and_order.push_back(newslot);
      }
      const size_t hs = sys->mixed ? sizeof(float2) : sizeof(double2);
      PT_CK(pt::anderson_push(sys->psi_f, sys->rbuf, sys->xprev, sys->rprev,
                              sys->dX + (newslot >= 0 ? newslot : 0) * stride * hs,
                              sys->dR + (newslot >= 0 ? newslot : 0) * stride * hs, n, newslot >= 0 ? 1 : 0,
                              sys->mixed ? 1 : 0, sys->s));
      have_prev = true;
      pt::SlotList sl{};
      sl.k = (int)sys->and_order.size();
      for (int q = 0; q < sl.k; ++q) sl.s[q] = sys->and_order[q];
      if (sl.k > 0) {
        PT_CK(pt::anderson_dots(sys->dR, stride, sl, newslot, sys->rbuf, npw, ne, m, sys->gram, sys->rhs,
                                sys->mixed ? 1 : 0, sys->s));
        PT_CK(pt::anderson_solve(sys->gram, sys->rhs, sl, m, ne, sys->gamma, sys->s));
      }
      PT_CK(pt::anderson_update(sys->psi_f, sys->rbuf, sys->dX, sys->dR, stride, sl, sys->gamma, std::max(m, 1), npw, n,
                                sys->p.anderson_beta, sys->mixed ? 1 : 0, sys->s));
    }
    // new density and its change
    Phase rho_("density");
    PT_TRY(real_orbitals_scf(sys, sys->psi_f));
    PT_TRY(density_scf(sys, sys->rho2));
    PT_CK(pt::rho_change(sys->rho2, sys->rho, sys->N, sys->part, sys->red + 1, sys->s));
    std::swap(sys->rho, sys->rho2);
    if (fixed == 0) {
      double h = 0.0;
      PT_CK(cudaMemcpyAsync(&h, sys->red + 1, sizeof(double), cudaMemcpyDeviceToHost, sys->s));
      PT_CK(cudaStreamSynchronize(sys->s));
      drho = h * sys->dV / (2.0 * ne);
      if (drho < sys->p.scf_tol) { converged = true; break; }
    }
  }
  if (it > niter) it = niter;
  if (fixed > 0) converged = true;
  double hres[2];
  PT_CK(cudaMemcpyAsync(hres, sys->red, sizeof(hres), cudaMemcpyDeviceToHost, sys->s));
  // orthonormalise and rebuild the exchange data / observables of Psi_{n+1}
  PT_TRY(orthonormalize(sys, sys->psi_f, sys->psi));
  PT_TRY(state_from_psi(sys));
  if (fixed > 0) drho = hres[1] * sys->dV / (2.0 * ne);
  sys->n_step += 1;
  if (info) {
    info->time = (double)sys->n_step * sys->p.dt;
    info->scf_iters = it;
    info->converged = converged ? 1 : 0;
    info->resid_norm = std::sqrt(hres[0]);
    info->drho = drho;
    info->energy = sys->energy;
    for (int k = 0; k < 3; ++k) info->dipole[k] = sys->dipole[k];
  }
  return converged ? PT_OK : PT_ERR_NOT_CONVERGED;
}

// H[X X^H](t) X for n_orb columns X: the density, local potential and exact exchange
// of X itself, the kinetic term at time t (the stage Hamiltonian of the RK4 step).
static pt_status h_of_self(pt_system* sys, const double2* X, double2* out, double t) {
  PT_TRY(set_kinetic_t(sys, t));
  PT_TRY(real_orbitals_scf(sys, X));
  sys->psi_r_current = false;
  PT_TRY(density_scf(sys, sys->rho));
  PT_TRY(local_potential(sys));
  PT_TRY(apply_local_scf(sys, X, out));
  if (sys->p.alpha != 0.0) PT_TRY(exchange_sym(sys, X, out, 1));
  return PT_OK;
}

// One classical RK4 step of i dPsi/dt = H[P] Psi (Eq. 1; the explicit integrator of the
// paper's Sec. 5 comparison): k_s = -i H_s Psi_s with stage orbitals Psi_1 = Psi_n,
// Psi_2,3 = Psi_n + dt/2 k_1,2, Psi_4 = Psi_n + dt k_3 at t_n, t_n + dt/2 (twice),
// t_n + dt; Psi_{n+1} = Psi_n + dt/6 (k_1 + 2 k_2 + 2 k_3 + k_4). k_1 uses the stored
// exchange of Psi_n; the other stages evaluate V_X of their own orbitals.
static pt_status rk4_step(pt_system* sys, pt_step_info* info) {
  Phase phase_("RK4 step");
  const long n = (long)sys->npw * sys->ne;
  const double dt = sys->p.dt;
  const double t = (double)sys->n_step * dt;
  const double w[4] = {dt / 6.0, dt / 3.0, dt / 3.0, dt / 6.0};
  const double c[3] = {0.5 * dt, 0.5 * dt, dt};
  const double ts[4] = {t, t + 0.5 * dt, t + 0.5 * dt, t + dt};
  PT_CK(cudaMemcpyAsync(sys->psi_f, sys->psi, sizeof(double2) * n, cudaMemcpyDeviceToDevice, sys->s));
  for (int st = 0; st < 4; ++st) {
    if (st == 0) {
      PT_TRY(set_kinetic_t(sys, ts[0]));
      if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
      PT_TRY(density_scf(sys, sys->rho));
      PT_TRY(local_potential(sys));
      PT_TRY(apply_local_scf(sys, sys->psi, sys->hpsi));
      PT_CK(pt::axpy(kOne, sys->wg, sys->hpsi, n, sys->s));
    } else {
      PT_TRY(h_of_self(sys, sys->tmp, sys->hpsi, ts[st]));
    }
    // acc += w_s (-i) H_s Psi_s; next stage Psi_n + c_s (-i) H_s Psi_s
    PT_CK(pt::axpy(make_double2(0.0, -w[st]), sys->hpsi, sys->psi_f, n, sys->s));
    if (st < 3) {
      PT_CK(cudaMemcpyAsync(sys->tmp, sys->psi, sizeof(double2) * n, cudaMemcpyDeviceToDevice, sys->s));
      PT_CK(pt::axpy(make_double2(0.0, -c[st]), sys->hpsi, sys->tmp, n, sys->s));
    }
  }
  PT_CK(cudaMemcpyAsync(sys->psi, sys->psi_f, sizeof(double2) * n, cudaMemcpyDeviceToDevice, sys->s));
  sys->n_step += 1;
  PT_TRY(set_kinetic(sys, sys->n_step));
  sys->psi_r_current = false;
  PT_TRY(state_from_psi(sys));
  if (info) {
    *info = pt_step_info{};
    info->converged = 1;
    info->time = (double)sys->n_step * dt;
    info->energy = sys->energy;
    for (int k = 0; k < 3; ++k) info->dipole[k] = sys->dipole[k];
  }
  return PT_OK;
}

// ---------------------------------------------------------------------------
// Exchange without device allocation (pt_exchange_static).
//
// Some callers cannot call cudaMalloc: a plug-in whose host application owns
// all device memory through its own allocator, or code that must not
// allocate after its start-up phase (an allocation can synchronise the
// device or fail under memory pressure). pt_exchange_static serves them: it
// keeps every buffer it needs in the file-scope array below, which exists on
// every GPU that loads this library until the process exits.
constexpr size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current).
static pt_status static_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { g_last_error = "pt_exchange_static: cudaGetDevice -> " + pt::cuda_msg(e); return PT_ERR_CUDA; }
  if (dev < 0 || dev >= kMaxDevices) { g_last_error = "pt_exchange_static: device index out of range"; return PT_ERR_INVALID; }
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_addr[dev] == nullptr) {
    void* addr = nullptr;
    e = cudaGetSymbolAddress(&addr, g_static_scratch);
    if (e != cudaSuccess || addr == nullptr) {
      g_last_error = "pt_exchange_static: cudaGetSymbolAddress -> " + pt::cuda_msg(e);
      return PT_ERR_CUDA;
    }
    g_static_addr[dev] = addr;
  }
  *out = g_static_addr[dev];
  return PT_OK;
}

// Layout of the static scratch for one call; returns the bytes needed (base 0 sizes it).
static size_t static_layout(pt_system* t, const pt_params* p, int npw, uintptr_t base, int tpl) {
  Carver c{base};
  const long N = (long)p->n[0] * p->n[1] * p->n[2];
  const long ne = p->n_orb;
  const bool mixed = p->precision == PT_MIXED;
  const size_t cs = mixed ? sizeof(float2) : sizeof(double2);
  const int tile = choose_tile(p);
  const long nb = (ne + tile - 1) / tile;
  t->basis = c.take<int>(npw);
  t->tw64 = c.take<double2>(pt::kTwiddleTotal);
  t->tw32 = c.take<float2>(pt::kTwiddleTotal);
  if (mixed) t->khat32 = c.take<float>(N); else t->khat64 = c.take<double>(N);
  t->psi_r = c.take<double2>((size_t)N * ne);
  if (mixed) t->psi_r32 = c.take<float2>((size_t)N * ne);
  t->w_r = c.take<unsigned char>((size_t)N * ne * cs);
  t->d_tiles_sym = c.take<pt::PairTile>((size_t)(nb * (nb - 1) / 2 + nb));
  t->status = c.take<int>(16);
  t->scratch = c.take<unsigned char>((size_t)tpl * pt::kTileMax * pt::kTileMax * N * cs);
  return c.off + 256;
}

static pt_status exchange_static_body(pt_system* t, const pt_params* p, const std::vector<int>& idx,
                                      const double2* d_psi, double2* d_w) {
  pt_system* sys = t;   // for PT_CK messages
  cudaStream_t s = t->s;
  PT_CK(cudaMemcpyAsync(t->basis, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
  PT_CK(upload_fft_tables(p, t->g, t->mixed, t->tw64, t->tw32, t->khat64, t->khat32, s));
  pt::PairTile* tiles = nullptr;
  int *lf = nullptr, *lc = nullptr, nl = 0;
  const int nt = pt::fock_build_tiles(t->ne, 0, t->plan_sym.tile, 1, t->plan_sym.tiles_per_launch, &tiles, &lf, &lc, &nl);
  if (nt < 0) { t->err = "pt_exchange_static: tile schedule"; return PT_ERR_INVALID; }
  t->plan_sym.n_launch = nl;
  t->plan_sym.launch_first = lf;
  t->plan_sym.launch_count = lc;
  t->plan_sym.n_tiles = nt;
  t->plan_sym.d_tiles = t->d_tiles_sym;
  t->plan_sym.g2_reach = pair_g2_reach(p);
  PT_CK(cudaMemsetAsync(t->status, 0, sizeof(int) * 16, s));
  cudaError_t e = cudaMemcpyAsync(t->d_tiles_sym, tiles, sizeof(pt::PairTile) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  std::free(tiles);
  if (e != cudaSuccess) { t->err = "pt_exchange_static: tile upload -> " + pt::cuda_msg(e); return PT_ERR_CUDA; }
  t->tw.d64 = t->tw64;
  t->tw.d32 = t->tw32;
  // real-space orbitals, then the pair pipeline (it zeroes the accumulators itself)
  PT_TRY(real_orbitals(t, d_psi));
  PT_TRY(exchange_sym(t, d_psi, d_w, 0));
  PT_CK(cudaStreamSynchronize(s));
  return PT_OK;
}

// ---------------------------------------------------------------------------
// C ABI

extern "C" {

pt_status pt_basis_size(const pt_params* p, int* npw) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = why; return st; }
  if (npw == nullptr) { g_last_error = "npw is NULL"; return PT_ERR_INVALID; }
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  *npw = (int)idx.size();
  return PT_OK;
}

pt_status pt_basis_indices(const pt_params* p, int64_t* out_host) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = why; return st; }
  if (out_host == nullptr) { g_last_error = "out is NULL"; return PT_ERR_INVALID; }
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  for (size_t k = 0; k < idx.size(); ++k) out_host[k] = idx[k];
  return PT_OK;
}

pt_status pt_workspace_size(const pt_params* p, size_t* bytes) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = why; return st; }
  if (bytes == nullptr) { g_last_error = "bytes is NULL"; return PT_ERR_INVALID; }
  *bytes = carve(nullptr, p, 0);
  return PT_OK;
}

// Live rows (i0, i1) of the basis sphere in flat order and the live i0 planes of a cubic
// grid of edge L, from the basis flat indices idx (ascending); uploaded to the device.
static pt_status upload_sphere_tables(pt_system* sys, int L, const std::vector<int>& idx, int* d_row_idx,
                                      int* d_row_kbeg, int* d_krow, int* d_planes, unsigned char* d_rowlive,
                                      unsigned char* d_planelive, pt::SphereTables* out) {
  const int npw = (int)idx.size();
  cudaStream_t s = sys->s;
  std::vector<int> row_idx, row_kbeg, krow(npw), planes;
  std::vector<unsigned char> rowlive((size_t)L * L, 0), planelive(L, 0);
  int prev = -1;
  for (int k = 0; k < npw; ++k) {
    const int row = idx[k] / L;
    if (row != prev) {
      row_idx.push_back(row);
      row_kbeg.push_back(k);
      rowlive[row] = 1;
      planelive[row / L] = 1;
      prev = row;
    }
    krow[k] = (int)row_idx.size() - 1;
  }
  row_kbeg.push_back(npw);
  for (int i0 = 0; i0 < L; ++i0)
    if (planelive[i0]) planes.push_back(i0);
  PT_CK(cudaMemcpyAsync(d_row_idx, row_idx.data(), sizeof(int) * row_idx.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(d_row_kbeg, row_kbeg.data(), sizeof(int) * row_kbeg.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(d_krow, krow.data(), sizeof(int) * npw, cudaMemcpyHostToDevice, s));
  if (!planes.empty())
    PT_CK(cudaMemcpyAsync(d_planes, planes.data(), sizeof(int) * planes.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(d_rowlive, rowlive.data(), rowlive.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(d_planelive, planelive.data(), planelive.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaStreamSynchronize(s));
  *out = pt::SphereTables{(int)row_idx.size(), d_row_idx, d_row_kbeg, d_krow, d_rowlive, (int)planes.size(), d_planes,
                          d_planelive};
  return PT_OK;
}

static pt_status init_body(pt_system* sys, const double* psi0_host) {
  const pt_params* p = &sys->p;
  std::vector<int> idx;
  std::vector<double> g2;
  basis_list(p, &idx, &g2);
  const int npw = sys->npw;
  // host tables
  std::vector<double> kin(npw), gk3(3 * (size_t)npw);
  {
    int k = 0;
    for (int t : idx) {
      const int i2 = t % p->n[2], i1 = (t / p->n[2]) % p->n[1], i0 = t / (p->n[1] * p->n[2]);
      const double gk0 = 2.0 * M_PI * freq(i0, p->n[0]) / p->cell[0] + p->kick[0];
      const double gk1 = 2.0 * M_PI * freq(i1, p->n[1]) / p->cell[1] + p->kick[1];
      const double gk2 = 2.0 * M_PI * freq(i2, p->n[2]) / p->cell[2] + p->kick[2];
      gk3[k] = gk0;
      gk3[npw + k] = gk1;
      gk3[2 * (size_t)npw + k] = gk2;
      kin[k++] = 0.5 * (gk0 * gk0 + gk1 * gk1 + gk2 * gk2);
    }
  }
  cudaStream_t s = sys->s;
  PT_CK(cudaMemcpyAsync(sys->basis, idx.data(), sizeof(int) * npw, cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(sys->kin, kin.data(), sizeof(double) * npw, cudaMemcpyHostToDevice, s));
  PT_CK(cudaMemcpyAsync(sys->gk3, gk3.data(), sizeof(double) * gk3.size(), cudaMemcpyHostToDevice, s));
  PT_CK(cudaStreamSynchronize(s));
  // twiddles, and the screened kernel on the Fock grid (scaled by -alpha / N_f)
  PT_CK(upload_fft_tables(p, sys->gf, sys->mixed, sys->tw64, sys->tw32, sys->khat64, sys->khat32, s));
  if (p->n_atoms > 0)
    PT_CK(cudaMemcpyAsync(sys->d_atoms, sys->atoms.data(), sizeof(double) * 3 * p->n_atoms, cudaMemcpyHostToDevice, s));
  if (pt::sphere_fast_supported(sys->g)) {
    PT_TRY(upload_sphere_tables(sys, sys->g.n0, idx, sys->sph_row_idx, sys->sph_row_kbeg, sys->sph_krow,
                                sys->sph_planes, sys->sph_rowlive, sys->sph_planelive, &sys->sph));
    sys->use_sphere = true;
  }
  if (sys->fock_own) {
    // the basis on the Fock grid: the same vectors in the same order (the sphere must fit)
    const pt_params q = fock_params(p);
    std::vector<int> idx_f;
    basis_list(&q, &idx_f, nullptr);
    bool same = (int)idx_f.size() == npw;
    for (int k = 0; same && k < npw; ++k) {
      const int a = idx[k], b = idx_f[k];
      same = freq(a % p->n[2], p->n[2]) == freq(b % q.n[2], q.n[2]) &&
             freq((a / p->n[2]) % p->n[1], p->n[1]) == freq((b / q.n[2]) % q.n[1], q.n[1]) &&
             freq(a / (p->n[1] * p->n[2]), p->n[0]) == freq(b / (q.n[1] * q.n[2]), q.n[0]);
    }
    if (!same) { sys->err = "the basis sphere does not fit on the Fock grid n_fock"; return PT_ERR_INVALID; }
    PT_CK(cudaMemcpyAsync(sys->basis_f, idx_f.data(), sizeof(int) * npw, cudaMemcpyHostToDevice, s));
    if (pt::sphere_fast_supported(sys->gf)) {
      PT_TRY(upload_sphere_tables(sys, sys->gf.n0, idx_f, sys->sphf_row_idx, sys->sphf_row_kbeg, sys->sphf_krow,
                                  sys->sphf_planes, sys->sphf_rowlive, sys->sphf_planelive, &sys->sphf));
      sys->use_sphere_f = true;
    }
    PT_CK(cudaStreamSynchronize(s));
  }
  sys->tw.d64 = sys->tw64;
  sys->tw.d32 = sys->tw32;
  // pair tiles of the symmetric exchange
  {
    pt::PairTile* tiles = nullptr;
    int *lf = nullptr, *lc = nullptr, nl = 0;
    const int tile = choose_tile(p);
    const int tpl = tiles_per_launch(p, sys->Nf, sys->mixed);
    const int nt = pt::fock_build_tiles(sys->ne, 0, tile, 1, tpl, &tiles, &lf, &lc, &nl);
    if (nt < 0) { sys->err = "tile schedule"; return PT_ERR_INVALID; }
    PT_CK(cudaMemcpyAsync(sys->d_tiles_sym, tiles, sizeof(pt::PairTile) * nt, cudaMemcpyHostToDevice, s));
    PT_CK(cudaStreamSynchronize(s));
    std::free(tiles);
    sys->plan_sym.tile = tile;
    sys->plan_sym.tiles_per_launch = tpl;
    sys->plan_sym.n_launch = nl;
    sys->plan_sym.launch_first = lf;
    sys->plan_sym.launch_count = lc;
    sys->plan_sym.d_tiles = sys->d_tiles_sym;
    sys->plan_sym.n_tiles = nt;
    sys->plan_sym.g2_reach = pair_g2_reach(p);
  }
  PT_CK(cudaMemsetAsync(sys->status, 0, sizeof(int) * 16, s));
  PT_CK(cudaStreamSynchronize(s));
  // device tables
  PT_CK(pt::hartree_factor(sys->hfac, sys->g, p->cell, s));
  PT_CK(pt::kerker_factor(sys->kfac, sys->g, p->cell, p->relax_mix, p->relax_q0, s));
  if (p->n_atoms > 0)
    PT_CK(pt::ion_potential(sys->vion, sys->g, p->cell, sys->d_atoms, p->n_atoms, p->well_depth, p->well_sigma, s));
  else
    PT_CK(cudaMemsetAsync(sys->vion, 0, sizeof(double) * sys->N, s));
  // start orbitals
  if (psi0_host == nullptr) { sys->err = "psi0_host is NULL"; return PT_ERR_INVALID; }
  PT_CK(cudaMemcpyAsync(sys->tmp, psi0_host, sizeof(double2) * npw * sys->ne, cudaMemcpyHostToDevice, s));
  PT_TRY(orthonormalize(sys, sys->tmp, sys->psi));
  PT_TRY(relax(sys));
  PT_TRY(state_from_psi(sys));
  PT_CK(cudaStreamSynchronize(s));
  PT_CK(cudaGetLastError());
  return PT_OK;
}

pt_status pt_init_system(const pt_params* p, const double* psi0_host, void* d_workspace, size_t workspace_bytes,
                         void* stream, pt_system** out) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = why; return st; }
  if (out == nullptr || d_workspace == nullptr) { g_last_error = "out / workspace is NULL"; return PT_ERR_INVALID; }
  if (((uintptr_t)d_workspace & 255) != 0) { g_last_error = "workspace must be 256-byte aligned"; return PT_ERR_INVALID; }
  const size_t need = carve(nullptr, p, 0);
  if (workspace_bytes < need) { g_last_error = "workspace too small"; return PT_ERR_OOM; }
  pt_system* sys = new pt_system();
  sys->p = *p;
  if (p->n_atoms > 0) sys->atoms.assign(p->atom_frac, p->atom_frac + 3 * p->n_atoms);
  sys->p.atom_frac = nullptr;
  sys->s = (cudaStream_t)stream;
  sys->g = Grid3{p->n[0], p->n[1], p->n[2]};
  sys->N = sys->g.N();
  {
    const pt_params q = fock_params(p);
    sys->fock_own = fock_is_own(p);
    sys->gf = Grid3{q.n[0], q.n[1], q.n[2]};
    sys->Nf = sys->gf.N();
  }
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  sys->npw = (int)idx.size();
  sys->ne = p->n_orb;
  sys->mdim = p->anderson_dim;
  sys->hb = h_batch(p);
  sys->vol = p->cell[0] * p->cell[1] * p->cell[2];
  sys->dV = sys->vol / (double)sys->N;
  sys->mixed = p->precision == PT_MIXED;
  carve(sys, p, (uintptr_t)d_workspace);
  st = init_body(sys, psi0_host);
  if (st != PT_OK) {
    g_last_error = sys->err;
    pt_destroy(sys);
    return st;
  }
  *out = sys;
  return PT_OK;
}

pt_status pt_build_ace(pt_system* sys) {
  if (sys == nullptr) return invalid_arg(sys, "pt_build_ace", "NULL handle");
  if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  const int saved = sys->p.fock_mode;
  sys->p.fock_mode = PT_FOCK_ACE;
  pt_status st = exchange_data(sys);
  sys->p.fock_mode = saved;
  if (st != PT_OK) return st;
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_apply_h(pt_system* sys, const void* d_X, void* d_Y, int ncols, int fock_mode) {
  if (sys == nullptr) return invalid_arg(sys, "pt_apply_h", "NULL handle");
  if (d_X == nullptr || d_Y == nullptr || ncols < 1 || ncols > sys->ne) {
    sys->err = "pt_apply_h: need 1 <= ncols <= n_orb and non-NULL buffers";
    return PT_ERR_INVALID;
  }
  if (fock_mode == PT_FOCK_ACE && !sys->have_ace) { sys->err = "pt_apply_h: no ACE operator built"; return PT_ERR_INVALID; }
  const double2* X = (const double2*)d_X;
  double2* Y = (double2*)d_Y;
  if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  PT_CK(pt::density(sys->psi_r, sys->N, sys->ne, sys->rho, sys->s));
  PT_TRY(local_potential(sys));
  PT_TRY(apply_local(sys, X, Y, ncols));
  if (sys->p.alpha != 0.0) {
    if (fock_mode == PT_FOCK_EXACT) {
      if (sys->mixed) PT_TRY(exchange_x_t<float>(sys, X, ncols, Y));
      else PT_TRY(exchange_x_t<double>(sys, X, ncols, Y));
    } else if (fock_mode == PT_FOCK_ACE) {
      PT_TRY(ace_apply(sys, X, ncols, Y));
    }
  }
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_exchange(pt_system* sys, void* d_W) {
  if (sys == nullptr) return invalid_arg(sys, "pt_exchange", "NULL handle");
  if (d_W == nullptr) { sys->err = "pt_exchange: NULL output"; return PT_ERR_INVALID; }
  if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  PT_TRY(exchange_sym(sys, sys->psi, (double2*)d_W, 0));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_cn_step(pt_system* sys, pt_step_info* out) {
  if (sys == nullptr) return invalid_arg(sys, "pt_cn_step", "NULL handle");
  pt_step_info info{};
  pt_status st = cn_step(sys, &info);
  if (out) *out = info;
  return st;
}

pt_status pt_rk4_step(pt_system* sys, pt_step_info* out) {
  if (sys == nullptr) return invalid_arg(sys, "pt_rk4_step", "NULL handle");
  pt_step_info info{};
  pt_status st = rk4_step(sys, &info);
  if (out) *out = info;
  return st;
}

pt_status pt_propagate(pt_system* sys, int nsteps, pt_step_info* out_host) {
  if (sys == nullptr || nsteps < 0) return invalid_arg(sys, "pt_propagate", "NULL handle or nsteps < 0");
  pt_status worst = PT_OK;
  for (int k = 0; k < nsteps; ++k) {
    pt_step_info info{};
    pt_status st = cn_step(sys, &info);
    if (out_host) out_host[k] = info;
    if (st == PT_ERR_NOT_CONVERGED) { worst = st; continue; }
    if (st != PT_OK) return st;
  }
  return worst;
}

pt_status pt_get_orbitals(pt_system* sys, double* psi_host) {
  if (sys == nullptr || psi_host == nullptr) return invalid_arg(sys, "pt_get_orbitals", "NULL handle or buffer");
  PT_CK(cudaMemcpyAsync(psi_host, sys->psi, sizeof(double2) * sys->npw * sys->ne, cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_set_orbitals(pt_system* sys, const double* psi_host) {
  if (sys == nullptr || psi_host == nullptr) return invalid_arg(sys, "pt_set_orbitals", "NULL handle or buffer");
  PT_CK(cudaMemcpyAsync(sys->tmp, psi_host, sizeof(double2) * sys->npw * sys->ne, cudaMemcpyHostToDevice, sys->s));
  PT_TRY(orthonormalize(sys, sys->tmp, sys->psi));
  PT_TRY(state_from_psi(sys));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_get_state(pt_system* sys, double* psi_host, double* w_host, int64_t* step) {
  if (sys == nullptr || psi_host == nullptr || w_host == nullptr) return invalid_arg(sys, "pt_get_state", "NULL handle or buffer");
  if (step) *step = sys->n_step;
  const size_t bytes = sizeof(double2) * sys->npw * sys->ne;
  PT_CK(cudaMemcpyAsync(psi_host, sys->psi, bytes, cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaMemcpyAsync(w_host, sys->wg, bytes, cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_set_state(pt_system* sys, const double* psi_host, const double* w_host, int64_t step) {
  if (sys == nullptr || psi_host == nullptr || w_host == nullptr || step < 0)
    return invalid_arg(sys, "pt_set_state", "NULL handle or buffer, or step < 0");
  const size_t bytes = sizeof(double2) * sys->npw * sys->ne;
  sys->n_step = step;
  PT_TRY(set_kinetic(sys, step));
  PT_CK(cudaMemcpyAsync(sys->psi, psi_host, bytes, cudaMemcpyHostToDevice, sys->s));
  PT_CK(cudaMemcpyAsync(sys->wg, w_host, bytes, cudaMemcpyHostToDevice, sys->s));
  PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  PT_TRY(ace_from_w(sys));
  PT_TRY(observables(sys));
  PT_CK(cudaStreamSynchronize(sys->s));
  return PT_OK;
}

pt_status pt_observables(pt_system* sys, double* energy, double* dipole) {
  if (sys == nullptr) return invalid_arg(sys, "pt_observables", "NULL handle");
  if (energy) *energy = sys->energy;
  if (dipole) for (int k = 0; k < 3; ++k) dipole[k] = sys->dipole[k];
  return PT_OK;
}

pt_status pt_orbitals_device(pt_system* sys, void** d_psi) {
  if (sys == nullptr || d_psi == nullptr) return invalid_arg(sys, "pt_orbitals_device", "NULL handle or output");
  *d_psi = sys->psi;
  return PT_OK;
}

pt_status pt_set_timing(pt_system* sys, int enable) {
  if (sys == nullptr) return invalid_arg(sys, "pt_set_timing", "NULL handle");
  if (enable && sys->ev0 == nullptr) {
    PT_CK(cudaEventCreate(&sys->ev0));
    PT_CK(cudaEventCreate(&sys->ev1));
  }
  sys->timing = enable != 0;
  return PT_OK;
}

pt_status pt_get_timing(pt_system* sys, double* pair_ms, int64_t* pairs, int64_t* launch_groups, int reset) {
  if (sys == nullptr) return invalid_arg(sys, "pt_get_timing", "NULL handle");
  if (pair_ms) *pair_ms = sys->t_pair_ms;
  if (pairs) *pairs = sys->t_pairs;
  if (launch_groups) *launch_groups = sys->t_groups;
  if (reset) { sys->t_pair_ms = 0.0; sys->t_pairs = 0; sys->t_groups = 0; }
  return PT_OK;
}

pt_status pt_exchange_static(const pt_params* p, const void* d_psi, void* d_w, void* stream) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = "pt_exchange_static: " + why; return st; }
  if (d_psi == nullptr || d_w == nullptr) { g_last_error = "pt_exchange_static: NULL orbitals or output"; return PT_ERR_INVALID; }
  if (fock_is_own(p)) { g_last_error = "pt_exchange_static: a separate Fock grid (n_fock) is not supported"; return PT_ERR_INVALID; }
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  const long N = (long)p->n[0] * p->n[1] * p->n[2];
  const size_t cs = p->precision == PT_MIXED ? sizeof(float2) : sizeof(double2);
  const int tile = choose_tile(p);
  const int nb = (p->n_orb + tile - 1) / tile;
  pt_system probe;
  const size_t fixed = static_layout(&probe, p, (int)idx.size(), 0, 0);
  const size_t per_tile = (size_t)pt::kTileMax * pt::kTileMax * N * cs;
  if (fixed + per_tile > kStaticScratchBytes) {
    g_last_error = "pt_exchange_static: this system needs " + std::to_string(fixed + per_tile) +
                   " bytes of scratch (orbitals, accumulators, one pair tile); the static array holds " +
                   std::to_string(kStaticScratchBytes) + " bytes. Use pt_exchange with a workspace.";
    return PT_ERR_OOM;
  }
  int tpl = (int)std::min<size_t>((size_t)nb, (kStaticScratchBytes - fixed) / per_tile);
  if (p->pair_tiles_per_launch > 0) tpl = std::min(tpl, p->pair_tiles_per_launch);
  void* base = nullptr;
  st = static_scratch_address(&base);
  if (st != PT_OK) return st;
  pt_system t;
  t.p = *p;
  t.p.atom_frac = nullptr;
  t.s = (cudaStream_t)stream;
  t.g = Grid3{p->n[0], p->n[1], p->n[2]};
  t.N = N;
  t.gf = t.g;
  t.Nf = N;
  t.npw = (int)idx.size();
  t.ne = p->n_orb;
  t.hb = h_batch(p);
  t.vol = p->cell[0] * p->cell[1] * p->cell[2];
  t.dV = t.vol / (double)N;
  t.mixed = p->precision == PT_MIXED;
  t.plan_sym.tile = tile;
  t.plan_sym.tiles_per_launch = tpl;
  static_layout(&t, p, t.npw, (uintptr_t)base, tpl);
  st = exchange_static_body(&t, p, idx, (const double2*)d_psi, (double2*)d_w);
  std::free(t.plan_sym.launch_first);
  std::free(t.plan_sym.launch_count);
  t.plan_sym.launch_first = nullptr;
  t.plan_sym.launch_count = nullptr;
  if (st != PT_OK) g_last_error = t.err;
  return st;
}

pt_status pt_launch_count(uint64_t* count) {
  if (count == nullptr) return invalid_arg(nullptr, "pt_launch_count", "NULL output");
  *count = (uint64_t)pt::launch_count();
  return PT_OK;
}

pt_status pt_destroy(pt_system* sys) {
  if (sys == nullptr) return PT_OK;
  if (sys->ev0) cudaEventDestroy(sys->ev0);
  if (sys->ev1) cudaEventDestroy(sys->ev1);
  std::free(sys->plan_sym.launch_first);
  std::free(sys->plan_sym.launch_count);
  std::free(sys->plan_x.launch_first);
  std::free(sys->plan_x.launch_count);
  delete sys;
  return PT_OK;
}

}  // extern "C"

static pt_status invalid_arg(pt_system* sys, const char* fn, const char* what) {
  const std::string msg = std::string(fn) + ": " + what;
  if (sys != nullptr) sys->err = msg;
  else g_last_error = msg;
  return PT_ERR_INVALID;
}

extern "C" {

const char* pt_last_error(const pt_system* sys) {
  if (sys == nullptr) return g_last_error.c_str();
  return sys->err.empty() ? "no error" : sys->err.c_str();
}

}  // extern "C"
