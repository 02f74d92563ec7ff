// The engine of one PT-CN system: the kernels' drivers for
//   * the exchange operator V_X Psi (Eq. 3, pair pipeline of fock.cu / fock_fast.cu),
//   * ACE: M = Psi^H W, -M = L L^H, xi = W L^{-H}, K_ACE X = -xi (xi^H X),
//   * H Psi (Eq. 2): kinetic diagonal, local potential by FFT, exchange,
//   * the PT-CN step of Eq. 5 / Alg. 1 with the residual of Alg. 3,
//     per-band Anderson mixing and Cholesky orthonormalisation (Sec. 3.4),
//   * the start-state relaxation and the RK4 comparison step.
// All device work is enqueued on the system's stream; host synchronisation
// happens only where a scalar decides control flow (SCF exit, pivots).
#include <mutex>

#include "engine.h"
#include "fft.cuh"

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
pt_status real_orbitals(pt_system* sys, const double2* c) {
  PT_TRY(to_real<double>(sys, c, sys->ne, sys->psi_r));
  if (sys->mixed) PT_CK(pt::convert_c128_to_c64(sys->psi_r, sys->psi_r32, sys->N * sys->ne, sys->s));
  return PT_OK;
}

pt_status local_potential(pt_system* sys, const double* rho) {
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

pt_status local_potential(pt_system* sys) { return local_potential(sys, sys->rho); }

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
pt_status apply_local_from_real(pt_system* sys, const double2* c, double2* out) {
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
pt_status apply_local(pt_system* sys, const double2* X, double2* out, int ncols) {
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

// Device address of the real-space orbitals the pair kernels read (exchange precision, Fock
// grid): fixed for the life of the system, so the pair tiles are bound to it once.
const void* fock_orbitals_addr(const pt_system* sys) {
  if (sys->fock_own) return sys->psi_rf;
  return sys->mixed ? (const void*)sys->psi_r32 : (const void*)sys->psi_r;
}

size_t exchange_cs(const pt_system* sys) { return sys->mixed ? sizeof(float2) : sizeof(double2); }

// The exchange of the orbitals Psi = coef (Eq. 3 on the Fock grid) in three parts, so that
// a batch can run the pair kernels of several systems in shared launches: prepare puts
// the real-space orbitals where the system's pair tiles read them and zeroes the
// accumulators, the pair kernels of the plan accumulate W(r), finish transforms W(r)
// to the basis into out (or adds it).
template <typename T>
static pt_status exchange_prepare_t(pt_system* sys, const double2* coef) {
  const void* pr = nullptr;
  PT_TRY(fock_orbitals<T>(sys, coef, &pr));
  (void)pr;   // the pair tiles are bound to this address (fock_orbitals_addr)
  PT_CK(cudaMemsetAsync(sys->w_r, 0, sizeof(pt::cplx<T>) * fock_grid(sys).N * sys->ne, sys->s));
  return PT_OK;
}

template <typename T>
static pt_status exchange_finish_t(pt_system* sys, double2* out, int accumulate) {
  return to_basis<T>(sys, fock_grid(sys), sys->w_r, sys->ne, out, accumulate, nullptr, nullptr);
}

pt_status exchange_prepare(pt_system* sys, const double2* coef) {
  return sys->mixed ? exchange_prepare_t<float>(sys, coef) : exchange_prepare_t<double>(sys, coef);
}

pt_status exchange_finish(pt_system* sys, double2* out, int accumulate) {
  return sys->mixed ? exchange_finish_t<float>(sys, out, accumulate) : exchange_finish_t<double>(sys, out, accumulate);
}

template <typename T>
static pt_status exchange_sym_t(pt_system* sys, const double2* coef, double2* out, int accumulate) {
  PT_TRY(exchange_prepare_t<T>(sys, coef));
  const T* kt = sys->mixed ? (const T*)(const void*)sys->khat32 : (const T*)(const void*)sys->khat64;
  if (sys->timing) PT_CK(cudaEventRecord(sys->ev0, sys->s));
  PT_CK(pt::fock_pairs<T>(sys->plan_sym, 1, fock_grid(sys).g, kt, sys->scratch, sys->tw, sys->s));
  if (sys->timing) {
    PT_CK(cudaEventRecord(sys->ev1, sys->s));
    PT_CK(cudaEventSynchronize(sys->ev1));
    float ms = 0.f;
    PT_CK(cudaEventElapsedTime(&ms, sys->ev0, sys->ev1));
    sys->t_pair_ms += ms;
    sys->t_pairs += (long long)sys->ne * (sys->ne + 1) / 2;
    sys->t_groups += sys->plan_sym.n_launch;
  }
  return exchange_finish_t<T>(sys, out, accumulate);
}

pt_status exchange_sym(pt_system* sys, const double2* coef, double2* out, int accumulate) {
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
  pt::fock_bind_tiles(tiles, nt, fock_orbitals_addr(sys), sys->x_r, nullptr, sys->w_r, sys->Nf, exchange_cs(sys));
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
  set_pair_reach(&sys->plan_x, &sys->p);
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
  (void)pr;   // the tiles of plan_x are bound to these orbitals, x_r and w_r
  PT_CK(pt::fock_pairs<T>(sys->plan_x, 0, fv.g, kt, sys->scratch, sys->tw, sys->s));
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

// Product of complex64 copies on the tensor cores (mixed precision, 3xTF32 with FP32
// accumulation); C stays complex128. A bounded wait that expires inside the kernel sets
// status[4], which tc_status() reports.
static pt_status gemm32(pt_system* sys, int opA, int opB, int M, int N, int K, double2 alpha, const float2* A, long lda,
                        const float2* B, long ldb, double2 beta, double2* C, long ldc,
                        int structure = pt::GEMM_GENERAL) {
  PT_CK(pt::gemm_tc(opA, opB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, sys->gemm_ws, sys->gemm_ws_elems,
                    sys->status + 4, sys->s, structure));
  return PT_OK;
}

// Small readbacks land in page-locked memory. With a pageable destination the driver
// stages the copy through a buffer it shares across the process, and a copy queued behind
// one stream's long backlog then holds up the readbacks of every other thread's systems.
namespace {
std::mutex g_pinned_mu;
std::vector<void*> g_pinned_free;
}  // namespace

void* pinned_block_get() {
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  if (g_pinned_free.empty()) {
    constexpr int kChunk = 64;
    void* p = nullptr;
    if (cudaHostAlloc(&p, kChunk * kPinnedBytes, cudaHostAllocPortable) != cudaSuccess) return nullptr;
    for (int k = 0; k < kChunk; ++k) g_pinned_free.push_back(static_cast<unsigned char*>(p) + k * kPinnedBytes);
  }
  void* b = g_pinned_free.back();
  g_pinned_free.pop_back();
  return b;
}

void pinned_block_put(void* block) {
  if (block == nullptr) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.push_back(block);
}

pt_status read_small(pt_system* sys, void* dst, const void* d_src, size_t bytes) {
  void* via = (sys->pinned != nullptr && bytes <= kPinnedBytes) ? sys->pinned : dst;
  PT_CK(cudaMemcpyAsync(via, d_src, bytes, cudaMemcpyDeviceToHost, sys->s));
  PT_CK(cudaStreamSynchronize(sys->s));
  if (via != dst) std::memcpy(dst, via, bytes);
  return PT_OK;
}

// PT_ERR_TIMEOUT once a tensor-core product has given up a wait (the flag stays set).
pt_status tc_status(pt_system* sys) {
  int h = 0;
  PT_TRY(read_small(sys, &h, sys->status + 4, sizeof(int)));
  if (h != 0) { sys->err = "tensor-core product: a bounded wait expired"; return PT_ERR_TIMEOUT; }
  return PT_OK;
}

static pt_status to32(pt_system* sys, const double2* src, float2* dst, long n) {
  PT_CK(pt::convert_c128_to_c64(src, dst, n, sys->s));
  return PT_OK;
}

// SCF-iteration forms. In mixed precision the real-space orbitals, the
// density they give and the local-potential product run in FP32; in FP64
// mode these are the FP64 routines above.
pt_status real_orbitals_scf(pt_system* sys, const double2* c) {
  if (!sys->mixed) return real_orbitals(sys, c);
  return to_real<float>(sys, c, sys->ne, sys->psi_r32);
}

pt_status density_scf(pt_system* sys, double* rho) {
  if (sys->mixed) PT_CK(pt::density32(sys->psi_r32, sys->N, sys->ne, rho, sys->s));
  else PT_CK(pt::density(sys->psi_r, sys->N, sys->ne, rho, sys->s));
  return PT_OK;
}

pt_status apply_local_scf(pt_system* sys, const double2* c, double2* out) {
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

// S = A^H B and C -= A S (the PT projection, Alg. 3): on the tensor cores in mixed
// precision unless fp64 is asked for (refinement iterations)
pt_status projection(pt_system* sys, const double2* A, double2* HB, bool fp64) {
  const int ne = sys->ne, npw = sys->npw;
  if (sys->mixed && !fp64) {
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

pt_status read_status(pt_system* sys, int* h) { return read_small(sys, h, sys->status, sizeof(int)); }

// dst = src L^{-H}, L L^H = src^H src  (Sec. 3.4)
pt_status orthonormalize(pt_system* sys, const double2* src, double2* dst) {
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

// ACE data of (psi_src, wg) with psi_src the current orbitals unless given: Mneg =
// -Psi^H W; Cholesky -M = L L^H; xi = W L^{-H} (ACE construction following Eq. 3 and
// the ACE definition; K_ACE Psi = W holds for any Psi with Psi^H W Hermitian negative
// definite, orthonormal or not).
pt_status ace_from_w(pt_system* sys, const double2* psi_src) {
  const int ne = sys->ne, npw = sys->npw;
  const bool ace = sys->p.fock_mode == PT_FOCK_ACE && sys->p.alpha != 0.0;
  const double2* psi = psi_src ? psi_src : sys->psi;
  if (sys->mixed && ace) {
    PT_TRY(to32(sys, psi, sys->ga32, (long)npw * ne));
    PT_TRY(to32(sys, sys->wg, sys->gb32, (long)npw * ne));
    PT_TRY(gemm32(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kMinusOne, sys->ga32, npw, sys->gb32, npw, kZero, sys->Mneg, ne));
  } else
    PT_TRY(gemm<double>(sys, pt::OP_H, pt::OP_N, ne, ne, npw, kMinusOne, psi, npw, sys->wg, npw, kZero, sys->Mneg, ne));
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
pt_status exchange_data(pt_system* sys) {
  Phase phase_("exchange + ACE build");
  PT_TRY(exchange_sym(sys, sys->psi, sys->wg, 0));
  return ace_from_w(sys);
}

// out += -xi (xi^H X); xi is complex128 in both precisions, its complex64 copy feeds the
// tensor-core products of mixed precision (unless fp64 is asked for)
pt_status ace_apply(pt_system* sys, const double2* X, int ncols, double2* out, bool fp64) {
  const int ne = sys->ne, npw = sys->npw;
  if (sys->mixed && !fp64) {
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
pt_status observables(pt_system* sys) {
  PT_CK(pt::density(sys->psi_r, sys->N, sys->ne, sys->rho, sys->s));
  PT_TRY(local_potential(sys));
  PT_CK(pt::energy_sums(sys->rho, sys->vion, sys->vh, sys->p.use_hartree ? 1 : 0, sys->g, sys->p.cell, sys->psi,
                        sys->kin, sys->npw, sys->ne, sys->Mneg, sys->part, sys->red + 8, sys->s));
  double h[8];
  PT_TRY(read_small(sys, h, sys->red + 8, sizeof(h)));
  if (sys->mixed) PT_TRY(tc_status(sys));
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
pt_status relax(pt_system* sys) {
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

pt_status state_from_psi(pt_system* sys) {
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
pt_status set_kinetic_t(pt_system* sys, double t) {
  if (sys->p.laser_amp == 0.0) return PT_OK;
  double a[3];
  laser_field(&sys->p, t, a);
  PT_CK(pt::kinetic_shifted(sys->gk3, sys->npw, a[0], a[1], a[2], sys->kin, sys->s));
  return PT_OK;
}

pt_status set_kinetic(pt_system* sys, int64_t n) { return set_kinetic_t(sys, (double)n * sys->p.dt); }

// ---- one PT-CN step (Eq. 5, Alg. 1), in phases ---------------------------------
// cn_begin enqueues R_n and the half step, cn_iterate one SCF iteration, cn_check reads
// its density change (the only host synchronisation of an iteration), cn_orthonormalize
// forms Psi_{n+1} and its real-space orbitals, and after the exchange of Psi_{n+1}
// (W = V_X Psi_{n+1}, exchange_sym or a batch's shared pair launches) cn_complete builds
// ACE and the observables. cn_step runs them in order; a batch interleaves the phases of
// several systems, each on its own stream, with identical arithmetic.

pt_status cn_begin(pt_system* sys, StepCtx* c) {
  const int ne = sys->ne, npw = sys->npw;
  const long n = (long)npw * ne;
  const double hdt = 0.5 * sys->p.dt;
  *c = StepCtx{};
  if (!sys->psi_r_current) PT_TRY(real_orbitals(sys, sys->psi));
  // Mixed-precision iterative refinement: with a tolerance below scf_fp64_below, R_n
  // and the iterations after the density change has dropped below it run in FP64.
  c->refine = sys->mixed && sys->p.scf_fp64_below > 0.0 && sys->p.scf_tol < sys->p.scf_fp64_below &&
              sys->p.scf_fixed_iters == 0;
  // initial residual R_n = H_n Psi_n - Psi_n (Psi_n^H H_n Psi_n) and the half step (H_n at t_n)
  PT_TRY(set_kinetic(sys, sys->n_step));
  if (c->refine) {
    PT_CK(pt::density(sys->psi_r, sys->N, ne, sys->rho, sys->s));
    PT_TRY(local_potential(sys));
    PT_TRY(apply_local_from_real(sys, sys->psi, sys->hpsi));
  } else {
    PT_TRY(density_scf(sys, sys->rho));
    PT_TRY(local_potential(sys));
    PT_TRY(apply_local_scf(sys, sys->psi, sys->hpsi));
  }
  PT_CK(pt::axpy(kOne, sys->wg, sys->hpsi, n, sys->s));
  PT_TRY(projection(sys, sys->psi, sys->hpsi, c->refine));
  PT_CK(pt::half_step(sys->psi, sys->hpsi, hdt, sys->psi_half, n, sys->s));
  // the SCF loop and the observables of Psi_{n+1} use H at t_{n+1}
  PT_TRY(set_kinetic(sys, sys->n_step + 1));
  PT_CK(cudaMemcpyAsync(sys->psi_f, sys->psi_half, sizeof(double2) * n, cudaMemcpyDeviceToDevice, sys->s));
  PT_TRY(real_orbitals_scf(sys, sys->psi_f));
  sys->psi_r_current = false;
  PT_TRY(density_scf(sys, sys->rho));
  c->fixed = sys->p.scf_fixed_iters;
  c->niter = c->fixed > 0 ? c->fixed : sys->p.scf_max;
  sys->and_count = 0;
  sys->and_order.clear();
  return PT_OK;
}

pt_status cn_iterate(pt_system* sys, StepCtx* c) {
  Phase iter_("SCF iteration");
  const int ne = sys->ne, npw = sys->npw;
  const long n = (long)npw * ne;
  const double hdt = 0.5 * sys->p.dt;
  const int m = sys->p.anderson_dim;
  const long stride = n;
  c->it += 1;
  const bool hi = c->hi;   // this iteration evaluates H Psi and R_f in FP64
  if (hi && !c->hi_prev) {
    // first FP64 iteration: FP64 real-space orbitals (and their FP32 copy) and density of Psi_f
    PT_TRY(real_orbitals(sys, sys->psi_f));
    PT_CK(pt::density(sys->psi_r, sys->N, ne, sys->rho, sys->s));
  }
  c->hi_prev = hi;
  {
    Phase p_("H Psi");
    PT_TRY(local_potential(sys));
    if (hi) PT_TRY(apply_local_from_real(sys, sys->psi_f, sys->hpsi));
    else PT_TRY(apply_local_scf(sys, sys->psi_f, sys->hpsi));
    if (sys->p.alpha != 0.0) {
      Phase x_(sys->p.fock_mode == PT_FOCK_EXACT ? "exchange" : "ACE apply");
      if (sys->p.fock_mode == PT_FOCK_EXACT) PT_TRY(exchange_sym(sys, sys->psi_f, sys->hpsi, 1));
      else PT_TRY(ace_apply(sys, sys->psi_f, ne, sys->hpsi, hi));
    }
  }
  {
    Phase p_("PT residual");
    PT_TRY(projection(sys, sys->psi_f, sys->hpsi, hi));
    PT_CK(pt::pt_residual(sys->psi_f, sys->hpsi, sys->psi_half, hdt, sys->rbuf, n, sys->part, sys->red + 0, sys->s));
  }
  // Anderson (per band)
  {
    Phase and_("Anderson");
    int newslot = -1;
    if (c->have_prev && m > 0) {
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
    c->have_prev = true;
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
  // new density and its change (FP64 real-space orbitals and density once refining)
  Phase rho_("density");
  if (hi) {
    PT_TRY(real_orbitals(sys, sys->psi_f));
    PT_CK(pt::density(sys->psi_r, sys->N, ne, sys->rho2, sys->s));
  } else {
    PT_TRY(real_orbitals_scf(sys, sys->psi_f));
    PT_TRY(density_scf(sys, sys->rho2));
  }
  PT_CK(pt::rho_change(sys->rho2, sys->rho, sys->N, sys->part, sys->red + 1, sys->s));
  std::swap(sys->rho, sys->rho2);
  return PT_OK;
}

pt_status cn_check(pt_system* sys, StepCtx* c) {
  if (c->fixed > 0) {
    if (c->it >= c->niter) { c->done = true; c->converged = true; }
    return PT_OK;
  }
  double h = 0.0;
  PT_TRY(read_small(sys, &h, sys->red + 1, sizeof(double)));
  c->drho = h * sys->dV / (2.0 * sys->ne);
  if (c->drho < sys->p.scf_tol) { c->converged = true; c->done = true; return PT_OK; }
  if (c->refine && c->drho < sys->p.scf_fp64_below) c->hi = true;
  if (c->it >= c->niter) c->done = true;
  return PT_OK;
}

pt_status cn_outer(pt_system* sys, StepCtx* c, bool* again) {
  *again = false;
  if (!c->done || sys->p.fock_mode != PT_FOCK_ACE || sys->p.alpha == 0.0 || c->outer >= sys->p.ace_outer)
    return PT_OK;
  Phase x_("outer ACE rebuild");
  c->outer += 1;
  // W = V_X Psi_f of the converged iterate (its real-space orbitals are current in the
  // exchange precision), ACE from (Psi_f, W), then the SCF again from Psi_f
  PT_TRY(exchange_sym(sys, sys->psi_f, sys->wg, 0));
  PT_TRY(ace_from_w(sys, sys->psi_f));
  c->done = false;
  c->converged = false;
  c->have_prev = false;
  c->niter = c->it + (c->fixed > 0 ? c->fixed : sys->p.scf_max);
  sys->and_count = 0;
  sys->and_order.clear();
  *again = true;
  return PT_OK;
}

pt_status cn_orthonormalize(pt_system* sys, StepCtx* c) {
  PT_TRY(read_small(sys, c->hres, sys->red, sizeof(c->hres)));
  // orthonormalise; the real-space orbitals of Psi_{n+1} for its exchange and density
  PT_TRY(orthonormalize(sys, sys->psi_f, sys->psi));
  PT_TRY(real_orbitals(sys, sys->psi));
  sys->psi_r_current = true;
  return PT_OK;
}

pt_status cn_complete(pt_system* sys, StepCtx* c, pt_step_info* info) {
  PT_TRY(ace_from_w(sys));
  PT_TRY(observables(sys));
  const double drho = c->fixed > 0 ? c->hres[1] * sys->dV / (2.0 * sys->ne) : c->drho;
  sys->n_step += 1;
  if (info) {
    info->time = (double)sys->n_step * sys->p.dt;
    info->scf_iters = c->it;
    info->converged = c->converged ? 1 : 0;
    info->resid_norm = std::sqrt(c->hres[0]);
    info->drho = drho;
    info->energy = sys->energy;
    for (int k = 0; k < 3; ++k) info->dipole[k] = sys->dipole[k];
  }
  return c->converged ? PT_OK : PT_ERR_NOT_CONVERGED;
}

pt_status cn_step(pt_system* sys, pt_step_info* info) {
  Phase phase_("PT-CN step");
  StepCtx c;
  PT_TRY(cn_begin(sys, &c));
  for (bool again = true; again;) {
    while (!c.done) {
      PT_TRY(cn_iterate(sys, &c));
      PT_TRY(cn_check(sys, &c));
    }
    PT_TRY(cn_outer(sys, &c, &again));
  }
  PT_TRY(cn_orthonormalize(sys, &c));
  {
    Phase x_("exchange + ACE build");
    PT_TRY(exchange_sym(sys, sys->psi, sys->wg, 0));
  }
  return cn_complete(sys, &c, info);
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
pt_status rk4_step(pt_system* sys, pt_step_info* info) {
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

// V_X applied to ncols columns X (pair pipeline with the occupied orbitals), added to out
pt_status exchange_x(pt_system* sys, const double2* X, int ncols, double2* out) {
  return sys->mixed ? exchange_x_t<float>(sys, X, ncols, out) : exchange_x_t<double>(sys, X, ncols, out);
}

