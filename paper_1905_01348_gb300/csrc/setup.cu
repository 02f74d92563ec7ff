// Set-up of a PT-CN system: parameter checks, the planewave basis (Sec. 3.1 / Sec. 4),
// the kernel and twiddle tables, the layout of the caller's workspace, the start
// state (orthonormalisation and relaxation), and the exchange without device
// allocation (pt_exchange_static).
#include <mutex>

#include "engine.h"
#include "fft.cuh"

// ---------------------------------------------------------------------------
// parameter checks and host tables

static bool supported_n(int n) { return pt::fft_length_supported(n); }

pt_status check_params(const pt_params* p, std::string* why) {
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
  if (!(p->scf_fp64_below >= 0.0)) { *why = "scf_fp64_below must be >= 0"; return PT_ERR_INVALID; }
  if (p->ace_outer < 0 || p->ace_outer > 8) { *why = "ace_outer must be in [0, 8]"; return PT_ERR_INVALID; }
  {
    const bool any = p->n_fock[0] || p->n_fock[1] || p->n_fock[2];
    for (int k = 0; k < 3 && any; ++k)
      if (!supported_n(p->n_fock[k])) { *why = "n_fock must be all 0 or supported grid sizes"; return PT_ERR_INVALID; }
  }
  return PT_OK;
}

inline int freq(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

void basis_list(const pt_params* p, std::vector<int>* idx, std::vector<double>* g2out) {
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
pt_params fock_params(const pt_params* p) {
  pt_params q = *p;
  if (p->n_fock[0] || p->n_fock[1] || p->n_fock[2])
    for (int k = 0; k < 3; ++k) q.n[k] = p->n_fock[k];
  return q;
}

bool fock_is_own(const pt_params* p) {
  const pt_params q = fock_params(p);
  return q.n[0] != p->n[0] || q.n[1] != p->n[1] || q.n[2] != p->n[2];
}

static long fock_points(const pt_params* p) {
  const pt_params q = fock_params(p);
  return (long)q.n[0] * q.n[1] * q.n[2];
}

// k-th output (k = 0, 1, ...) of SplitMix64 started from the state `seed` (Steele, Lea
// and Flood, 2014): the state advances by the golden-ratio increment, the output is its
// variant-13 mix. Counter-based: output k depends only on seed and k.
static inline uint64_t splitmix64_at(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// the top 53 bits as a uniform number in (0, 1), never 0
static inline double unit_open(uint64_t x) { return ((double)(x >> 11) + 0.5) * 0x1.0p-53; }

void seeded_coefficients(const pt_params* p, double* out) {
  std::vector<int> idx;
  std::vector<double> g2;
  basis_list(p, &idx, &g2);
  const uint64_t npw = idx.size();
  for (int b = 0; b < p->n_orb; ++b)
    for (uint64_t m = 0; m < npw; ++m) {
      const uint64_t j = (uint64_t)b * npw + m;
      const double u1 = unit_open(splitmix64_at(p->seed, 2 * j));
      const double u2 = unit_open(splitmix64_at(p->seed, 2 * j + 1));
      const double r = std::sqrt(-2.0 * std::log(u1)), t = 2.0 * M_PI * u2;
      const double w = std::exp(-0.25 * g2[m]);
      out[2 * j] = r * std::cos(t) * w;
      out[2 * j + 1] = r * std::sin(t) * w;
    }
}

// The reach of pair products along axis 2 (Eq. 3: products of two basis-limited
// orbitals): twice the largest |g2| index of the basis.
void set_pair_reach(pt::FockPlan* plan, const pt_params* p) {
  std::vector<int> idx;
  basis_list(p, &idx, nullptr);
  int m = 0;
  for (int v : idx) m = std::max(m, std::abs(freq(v % p->n[2], p->n[2])));
  plan->g2_reach = 2 * m;
}

// Screened kernel K(G) = 4 pi (1 - exp(-G^2 / (4 w^2))) / G^2, K(0) = pi / w^2 (its limit),
// on the grid g in the pair-intermediate layout [i2][i0][i1], scaled by -alpha / N (the
// inverse-FFT factor) so that the pair kernels multiply by it directly (Eq. 3).
std::vector<double> khat_table(const pt_params* p, Grid3 g) {
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
cudaError_t upload_fft_tables(const pt_params* p, Grid3 g, bool mixed, double2* tw64, float2* tw32,
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

int choose_tile(const pt_params* p) {
  if (p->pair_tile > 0) return p->pair_tile;
  return std::min(pt::kTileMax, p->n_orb);
}

int tiles_per_launch(const pt_params* p, long N, bool mixed) {
  const int tile = choose_tile(p);
  const int nb = (p->n_orb + tile - 1) / tile;
  const double per_tile = (double)pt::kTileMax * pt::kTileMax * N * (mixed ? 8.0 : 16.0);
  const double budget = 16.0e9;
  int cap = (int)std::max(1.0, std::floor(budget / per_tile));
  if (p->pair_tiles_per_launch > 0) cap = std::min(cap, p->pair_tiles_per_launch);
  return std::max(1, std::min(nb, cap));
}

int h_batch(const pt_params* p) { return std::min(p->n_orb, 32); }

// Carve (or size, when base == 0) the workspace.
size_t carve(pt_system* sys, const pt_params* p, uintptr_t base) {
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

pt_status init_body(pt_system* sys, const double* psi0_host) {
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
    pt::fock_bind_tiles(tiles, nt, fock_orbitals_addr(sys), nullptr, sys->w_r, nullptr, sys->Nf, exchange_cs(sys));
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
    set_pair_reach(&sys->plan_sym, p);
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
  // start orbitals: the caller's, or the seeded ones (kept alive until the copy has landed)
  std::vector<double> seeded;
  if (psi0_host == nullptr) {
    seeded.resize(2 * (size_t)npw * sys->ne);
    seeded_coefficients(p, seeded.data());
    psi0_host = seeded.data();
  }
  PT_CK(cudaMemcpyAsync(sys->tmp, psi0_host, sizeof(double2) * npw * sys->ne, cudaMemcpyHostToDevice, s));
  if (!seeded.empty()) PT_CK(cudaStreamSynchronize(s));
  PT_TRY(orthonormalize(sys, sys->tmp, sys->psi));
  PT_TRY(relax(sys));
  PT_TRY(state_from_psi(sys));
  PT_CK(cudaStreamSynchronize(s));
  PT_CK(cudaGetLastError());
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
extern const size_t kStaticScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
static std::mutex g_static_mu;
static void* g_static_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device. In host code the
// array's name is only a host-side stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress (with that device current).
pt_status static_scratch_address(void** out) {
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
size_t static_layout(pt_system* t, const pt_params* p, int npw, uintptr_t base, int tpl) {
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

pt_status exchange_static_body(pt_system* t, const pt_params* p, const std::vector<int>& idx,
                                      const double2* d_psi, double2* d_w) {
  pt_system* sys = t;   // for PT_CK messages
  cudaStream_t s = t->s;
  PT_CK(cudaMemcpyAsync(t->basis, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice, s));
  PT_CK(upload_fft_tables(p, t->g, t->mixed, t->tw64, t->tw32, t->khat64, t->khat32, s));
  pt::PairTile* tiles = nullptr;
  int *lf = nullptr, *lc = nullptr, nl = 0;
  const int nt = pt::fock_build_tiles(t->ne, 0, t->plan_sym.tile, 1, t->plan_sym.tiles_per_launch, &tiles, &lf, &lc, &nl);
  if (nt < 0) { t->err = "pt_exchange_static: tile schedule"; return PT_ERR_INVALID; }
  pt::fock_bind_tiles(tiles, nt, fock_orbitals_addr(t), nullptr, t->w_r, nullptr, t->N, exchange_cs(t));
  t->plan_sym.n_launch = nl;
  t->plan_sym.launch_first = lf;
  t->plan_sym.launch_count = lc;
  t->plan_sym.n_tiles = nt;
  t->plan_sym.d_tiles = t->d_tiles_sym;
  set_pair_reach(&t->plan_sym, p);
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

