// C ABI of include/pt.h: argument checks and the entry points; the work is done by
// the engine (engine.cu), set-up (setup.cu) and the batched stepping (batch.cu).
#include "engine.h"

thread_local std::string g_last_error = "no error";

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

pt_status pt_seeded_coefficients(const pt_params* p, double* out_host) {
  std::string why;
  pt_status st = check_params(p, &why);
  if (st != PT_OK) { g_last_error = why; return st; }
  if (out_host == nullptr) { g_last_error = "pt_seeded_coefficients: out is NULL"; return PT_ERR_INVALID; }
  seeded_coefficients(p, out_host);
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
  sys->pinned = pinned_block_get();   // nullptr (plain copies) if page-locked memory is refused
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
      PT_TRY(exchange_x(sys, X, ncols, Y));
    } else if (fock_mode == PT_FOCK_ACE) {
      PT_TRY(ace_apply(sys, X, ncols, Y));
    }
  }
  PT_CK(cudaStreamSynchronize(sys->s));
  if (sys->mixed) PT_TRY(tc_status(sys));
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

pt_status pt_complex_product(int op_a, int op_b, int M, int N, int K, const double* alpha2, const void* d_A,
                             int64_t lda, const void* d_B, int64_t ldb, const double* beta2, void* d_C, int64_t ldc,
                             int upper_b, void* d_ws, size_t ws_bytes, void* stream) {
  const char* fn = "pt_complex_product";
  if ((op_a != 0 && op_a != 1) || (op_b != 0 && op_b != 1) || M < 0 || N < 0 || K < 0)
    return invalid_arg(nullptr, fn, "op_a / op_b must be 0 or 1 and sizes non-negative");
  if (alpha2 == nullptr || beta2 == nullptr || d_ws == nullptr || ws_bytes < 256 || ((uintptr_t)d_ws & 255) != 0 ||
      (M > 0 && N > 0 && d_C == nullptr) || (M > 0 && N > 0 && K > 0 && (d_A == nullptr || d_B == nullptr)))
    return invalid_arg(nullptr, fn, "NULL argument, or scratch smaller than 256 bytes / not 256-byte aligned");
  const long rows_a = op_a == 0 ? M : K, rows_b = op_b == 0 ? K : N;
  if (lda < std::max<long>(1, rows_a) || ldb < std::max<long>(1, rows_b) || ldc < std::max(1, M))
    return invalid_arg(nullptr, fn, "leading dimension smaller than the rows of its matrix");
  if (upper_b && K != N) return invalid_arg(nullptr, fn, "upper_b needs a square op(B)");
  cudaStream_t s = (cudaStream_t)stream;
  int* flag = (int*)d_ws;
  double2* part = (double2*)((unsigned char*)d_ws + 256);
  const size_t part_elems = (ws_bytes - 256) / sizeof(double2);
  cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = pt::gemm_tc(op_a == 0 ? pt::OP_N : pt::OP_H, op_b == 0 ? pt::OP_N : pt::OP_H, M, N, K,
                    make_double2(alpha2[0], alpha2[1]), (const float2*)d_A, (long)lda, (const float2*)d_B, (long)ldb,
                    make_double2(beta2[0], beta2[1]), (double2*)d_C, (long)ldc, part_elems ? part : nullptr,
                    part_elems, flag, s, upper_b ? pt::GEMM_TRI_B : pt::GEMM_GENERAL);
  int h = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { g_last_error = std::string(fn) + ": " + pt::cuda_msg(e); return PT_ERR_CUDA; }
  if (h != 0) { g_last_error = std::string(fn) + ": a bounded wait inside the kernel expired"; return PT_ERR_TIMEOUT; }
  return PT_OK;
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
  pinned_block_put(sys->pinned);
  std::free(sys->plan_sym.launch_first);
  std::free(sys->plan_sym.launch_count);
  std::free(sys->plan_x.launch_first);
  std::free(sys->plan_x.launch_count);
  delete sys;
  return PT_OK;
}

}  // extern "C"

pt_status invalid_arg(pt_system* sys, const char* fn, const char* what) {
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

