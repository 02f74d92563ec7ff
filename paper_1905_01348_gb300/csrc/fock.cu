// Fock exchange by orbital pairs (Eq. 3; the pair loop of Alg. 2).
//
// For every pair (i, j) the pair density rho_ij = conj(psi_i) psi_j goes
// through a forward 3D FFT, is multiplied by the screened kernel
// Khat(G) = 4 pi (1 - exp(-G^2 / (4 w^2))) / G^2 (scaled by -alpha / N), goes
// back through an inverse FFT and is multiplied by psi_i and accumulated
// into W_j. Because Khat is real and even, v_ji = conj(v_ij): one solve per
// unordered pair also feeds W_i += psi_j conj(v_ij) ("sym" mode).
//
// Pairs are grouped into tiles (up to kTileMax orbitals on each side) and a
// launch holds tiles whose output orbitals are all distinct, so every W
// element has a single writer per launch (deterministic, no atomics). One
// launch is three kernels over an intermediate X in global memory:
//   F1  rows: product of two orbitals' rows, FFT along axis 2; the block owns
//       `rr` rows of all pairs of its tile and stores X[pair][i2][i0][i1]
//       (axis 1 fastest, so F2 reads a contiguous slab);
//   F2  slab (pair, i2): FFT along axis 1 and axis 0, multiply by Khat,
//       inverse along axis 0 and axis 1, all in shared memory;
//   F3  rows: inverse FFT along axis 2 of all pairs of the tile, then each
//       output orbital sums its pair contributions in a fixed order and
//       updates its W row once.
// X traffic is four passes of the pair volume (write, read+write, read).
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace pt {

template <typename T>
static const cplx<T>* twp(const DevTwiddles& tw, int L) {
  return reinterpret_cast<const cplx<T>*>(tw.base<T>()) + twiddle_offset(L);
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_fock_f1(const PairTile* __restrict__ tiles, int tile0, cplx<T>* __restrict__ X, int n0, int n1,
                          int n2, int rr, const cplx<T>* __restrict__ tw_g) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairTile tl;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rowlen = rr * n2;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* orb = tw + n2;
  C* work = orb + 2 * kTileMax * rowlen;
  if (tid == 0) tl = tiles[tile0 + blockIdx.y];
  for (int t = tid; t < n2; t += nthr) tw[t] = tw_g[t];
  __syncthreads();
  const int nb1 = n1 / rr;
  const int i0 = blockIdx.x / nb1;
  const int i1s = (blockIdx.x - i0 * nb1) * rr;
  const long roff = ((long)i0 * n1 + i1s) * n2;
  for (int o = 0; o < tl.n_orb; ++o) {
    const C* src = (const C*)tl.in[o] + roff;
    for (int e = tid; e < rowlen; e += nthr) orb[o * rowlen + e] = src[e];
  }
  __syncthreads();
  const int np = tl.n_pairs;
  for (int idx = tid; idx < np * rowlen; idx += nthr) {
    const int p = idx / rowlen, e = idx - p * rowlen;
    work[idx] = cmulc(orb[tl.pi[p] * rowlen + e], orb[tl.pj[p] * rowlen + e]);
  }
  __syncthreads();
  fft_lines<T, false, true>(work, n2, np * rr, n2, 1, tw, tid, nthr);
  // store X[slot][i2][i0][i1s + r]; consecutive threads take consecutive r
  const long slot0 = (long)blockIdx.y * kTileMax * kTileMax;
  for (int idx = tid; idx < np * rowlen; idx += nthr) {
    const int r = idx % rr;
    const int rest = idx / rr;
    const int i2 = rest % n2;
    const int p = rest / n2;
    X[(((slot0 + p) * n2 + i2) * n0 + i0) * n1 + i1s + r] = work[(p * rr + r) * n2 + i2];
  }
}

template <typename T>
__global__ void __launch_bounds__(768, 1) k_fock_f2(cplx<T>* __restrict__ X, const PairTile* __restrict__ tiles, int tile0, int n0, int n1,
                          int n2, const T* __restrict__ khat_t, const cplx<T>* __restrict__ tw0_g,
                          const cplx<T>* __restrict__ tw1_g) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int slot = blockIdx.y;
  const int p = slot % (kTileMax * kTileMax);
  if (p >= tiles[tile0 + slot / (kTileMax * kTileMax)].n_pairs) return;
  const int i2 = blockIdx.x;
  C* tw0 = reinterpret_cast<C*>(smem_raw);
  C* tw1 = tw0 + n0;
  C* buf = tw1 + n1;
  for (int t = tid; t < n0; t += nthr) tw0[t] = tw0_g[t];
  for (int t = tid; t < n1; t += nthr) tw1[t] = tw1_g[t];
  const int cnt = n0 * n1;
  C* slab = X + ((long)slot * n2 + i2) * cnt;
  for (int e = tid; e < cnt; e += nthr) buf[e] = slab[e];
  __syncthreads();
  fft_lines<T, false, true>(buf, n1, n0, n1, 1, tw1, tid, nthr);    // axis 1
  fft_lines<T, false, false>(buf, n0, n1, 1, n1, tw0, tid, nthr);   // axis 0
  const T* kt = khat_t + (long)i2 * cnt;
  for (int e = tid; e < cnt; e += nthr) buf[e] = cscale(buf[e], kt[e]);
  __syncthreads();
  fft_lines<T, true, false>(buf, n0, n1, 1, n1, tw0, tid, nthr);
  fft_lines<T, true, true>(buf, n1, n0, n1, 1, tw1, tid, nthr);
  for (int e = tid; e < cnt; e += nthr) slab[e] = buf[e];
}

template <typename T>
__global__ void k_fock_f3(const PairTile* __restrict__ tiles, int tile0, const cplx<T>* __restrict__ X, int n0, int n1,
                          int n2, int rr, int sym,
                          const cplx<T>* __restrict__ tw_g) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairTile tl;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int rowlen = rr * n2;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* orb = tw + n2;
  C* work = orb + 2 * kTileMax * rowlen;
  if (tid == 0) tl = tiles[tile0 + blockIdx.y];
  for (int t = tid; t < n2; t += nthr) tw[t] = tw_g[t];
  __syncthreads();
  const int nb1 = n1 / rr;
  const int i0 = blockIdx.x / nb1;
  const int i1s = (blockIdx.x - i0 * nb1) * rr;
  const long roff = ((long)i0 * n1 + i1s) * n2;
  const int np = tl.n_pairs;
  const long slot0 = (long)blockIdx.y * kTileMax * kTileMax;
  for (int idx = tid; idx < np * rowlen; idx += nthr) {
    const int r = idx % rr;
    const int rest = idx / rr;
    const int i2 = rest % n2;
    const int p = rest / n2;
    work[(p * rr + r) * n2 + i2] = X[(((slot0 + p) * n2 + i2) * n0 + i0) * n1 + i1s + r];
  }
  for (int o = 0; o < tl.n_orb; ++o) {
    const C* src = (const C*)tl.in[o] + roff;
    for (int e = tid; e < rowlen; e += nthr) orb[o * rowlen + e] = src[e];
  }
  __syncthreads();
  fft_lines<T, true, true>(work, n2, np * rr, n2, 1, tw, tid, nthr);
  // each output orbital: fixed-order sum over the tile's pairs, one RMW of its row
  for (int o = 0; o < tl.n_orb; ++o) {
    if (!tl.is_out[o]) continue;
    C* dst = (C*)tl.out[o] + roff;
    for (int e = tid; e < rowlen; e += nthr) {
      C acc = mk((T)0, (T)0);
      for (int p = 0; p < np; ++p) {
        const C v = work[p * rowlen + e];
        if (tl.pj[p] == o) acc = cadd(acc, cmul(orb[tl.pi[p] * rowlen + e], v));
        if (sym && tl.pi[p] == o && tl.pi[p] != tl.pj[p]) acc = cadd(acc, cmul_conj(orb[tl.pj[p] * rowlen + e], v));
      }
      dst[e] = cadd(dst[e], acc);
    }
  }
}

// ---------------------------------------------------------------------------
static int rows_per_block(int n1, bool fp64) {
  const int want = fp64 ? 2 : 4;
  for (int r = want; r >= 1; r /= 2)
    if (n1 % r == 0) return r;
  return 1;
}

static int round_threads(int t) {
  t = ((t + 31) / 32) * 32;
  return std::max(64, std::min(1024, t));
}

template <typename T>
cudaError_t fock_pairs(const FockPlan& plan, int sym, Grid3 g, const T* khat_t, void* scratch, const DevTwiddles& tw,
                       cudaStream_t s) {
  using C = cplx<T>;
  if constexpr (sizeof(T) == 4) {
    if (fock_fast_supported(g)) return fock_pairs_fast(plan, g, khat_t, scratch, twp<float>(tw, g.n0), s);
  }
  const bool fp64 = sizeof(T) == 8;
  const int rr = rows_per_block(g.n1, fp64);
  const int rowlen = rr * g.n2;
  const int lines13 = kTileMax * kTileMax * rr;
  const int thr13 = round_threads(std::max(fft_threads_needed(g.n2, lines13, fp64), 128));
  const size_t smem13 = (size_t)(g.n2 + 2 * kTileMax * rowlen + kTileMax * kTileMax * rowlen) * sizeof(C);
  const int thr2 = round_threads(std::max(fft_threads_needed(g.n1, g.n0, fp64), fft_threads_needed(g.n0, g.n1, fp64)));
  const size_t smem2 = (size_t)(g.n0 + g.n1 + g.n0 * g.n1) * sizeof(C);
  if (thr13 > 1024 || thr2 > 768) return cudaErrorInvalidConfiguration;
  cudaError_t e;
  static std::atomic<unsigned long long> attr_done{0};
  if (const unsigned long long bit = device_bit_todo(attr_done)) {
    e = cudaFuncSetAttribute(k_fock_f1<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fock_f2<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fock_f3<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit, std::memory_order_release);
  }
  if (smem13 > 200 * 1024 || smem2 > 200 * 1024) return cudaErrorInvalidConfiguration;
  const C* tw0 = twp<T>(tw, g.n0);
  const C* tw1 = twp<T>(tw, g.n1);
  const C* tw2 = twp<T>(tw, g.n2);
  C* X = (C*)scratch;
  for (int l = 0; l < plan.n_launch; ++l) {
    const int t0 = plan.launch_first[l], nt = plan.launch_count[l];
    dim3 g13((unsigned)(g.n0 * (g.n1 / rr)), (unsigned)nt);
    k_fock_f1<T><<<g13, thr13, smem13, s>>>(plan.d_tiles, t0, X, g.n0, g.n1, g.n2, rr, tw2); launched();
    dim3 g2((unsigned)g.n2, (unsigned)(nt * kTileMax * kTileMax));
    k_fock_f2<T><<<g2, thr2, smem2, s>>>(X, plan.d_tiles, t0, g.n0, g.n1, g.n2, khat_t, tw0, tw1); launched();
    k_fock_f3<T><<<g13, thr13, smem13, s>>>(plan.d_tiles, t0, X, g.n0, g.n1, g.n2, rr, sym, tw2); launched();
  }
  return cudaGetLastError();
}

template cudaError_t fock_pairs<float>(const FockPlan&, int, Grid3, const float*, void*, const DevTwiddles&,
                                       cudaStream_t);
template cudaError_t fock_pairs<double>(const FockPlan&, int, Grid3, const double*, void*, const DevTwiddles&,
                                        cudaStream_t);

void fock_bind_tiles(PairTile* tiles, int n, const void* psi_r, const void* x_r, void* w_occ, void* w_x, long N,
                     size_t cs) {
  for (int t = 0; t < n; ++t) {
    PairTile& tl = tiles[t];
    for (int o = 0; o < 2 * kTileMax; ++o) {
      tl.in[o] = nullptr;
      tl.out[o] = nullptr;
      if (o >= tl.n_orb) continue;
      const size_t off = (size_t)tl.orb[o] * (size_t)N * cs;
      tl.in[o] = (const unsigned char*)(tl.src[o] == 0 ? psi_r : x_r) + off;
      if (tl.is_out[o]) tl.out[o] = (unsigned char*)(tl.src[o] == 0 ? w_occ : w_x) + off;
    }
  }
}

// ---------------------------------------------------------------------------
// Tile schedule. Symmetric: blocks of `tile` orbitals; rounds of a
// round-robin tournament pair the blocks so each block appears once per
// round (off-diagonal tiles: all |A| x |B| pairs), then one round of the
// diagonal tiles (pairs a <= b inside a block). Non-symmetric (V_X applied to
// other vectors): round r pairs X-block b with occupied block (b + r) mod nbo.
int fock_build_tiles(int n_occ, int n_x, int tile, int sym, int tiles_per_launch, PairTile** tiles_out,
                     int** launch_first, int** launch_count, int* n_launch) {
  if (tile < 1 || tile > kTileMax || n_occ < 1 || tiles_per_launch < 1) return -1;
  std::vector<PairTile> tiles;
  std::vector<std::vector<int>> rounds;   // tile indices per round
  auto block_range = [&](int b, int n, int* lo) { *lo = b * tile; return std::min(n, (b + 1) * tile) - b * tile; };
  auto make_tile = [&](int a_lo, int a_n, int a_src, int b_lo, int b_n, int b_src, bool diag, int out_a,
                       int out_b) {
    PairTile t;
    std::memset(&t, 0, sizeof(t));
    for (int i = 0; i < a_n; ++i) { t.orb[t.n_orb] = a_lo + i; t.src[t.n_orb] = (signed char)a_src; t.is_out[t.n_orb] = (signed char)out_a; ++t.n_orb; }
    if (!diag)
      for (int i = 0; i < b_n; ++i) { t.orb[t.n_orb] = b_lo + i; t.src[t.n_orb] = (signed char)b_src; t.is_out[t.n_orb] = (signed char)out_b; ++t.n_orb; }
    if (diag) {
      for (int a = 0; a < a_n; ++a)
        for (int b = a; b < a_n; ++b) { t.pi[t.n_pairs] = (signed char)a; t.pj[t.n_pairs] = (signed char)b; ++t.n_pairs; }
    } else {
      for (int a = 0; a < a_n; ++a)
        for (int b = 0; b < b_n; ++b) { t.pi[t.n_pairs] = (signed char)a; t.pj[t.n_pairs] = (signed char)(a_n + b); ++t.n_pairs; }
    }
    for (int o = 0; o < t.n_orb; ++o) {
      if (!t.is_out[o]) continue;
      int c = 0;
      for (int q = 0; q < t.n_pairs; ++q) {
        if (t.pj[q] == o) { t.out_pair[o][c] = (signed char)q; t.out_other[o][c] = t.pi[q]; t.out_conj[o][c] = 0; ++c; }
        if (sym && t.pi[q] == o && t.pi[q] != t.pj[q]) {
          t.out_pair[o][c] = (signed char)q; t.out_other[o][c] = t.pj[q]; t.out_conj[o][c] = 1; ++c;
        }
      }
      t.out_n[o] = (signed char)c;
    }
    tiles.push_back(t);
    return (int)tiles.size() - 1;
  };
  if (sym) {
    const int nb = (n_occ + tile - 1) / tile;
    const int nbp = nb + (nb & 1);
    for (int r = 0; r < nbp - 1; ++r) {
      std::vector<int> rd;
      for (int i = 0; i < nbp / 2; ++i) {
        int a, b;
        if (i == 0) { a = r; b = nbp - 1; }
        else { a = (r + i) % (nbp - 1); b = (r - i + nbp - 1) % (nbp - 1); }
        if (a >= nb || b >= nb) continue;
        if (a > b) std::swap(a, b);
        int alo, blo;
        const int an = block_range(a, n_occ, &alo), bn = block_range(b, n_occ, &blo);
        rd.push_back(make_tile(alo, an, 0, blo, bn, 0, false, 1, 1));
      }
      if (!rd.empty()) rounds.push_back(rd);
    }
    std::vector<int> rd;
    for (int b = 0; b < nb; ++b) {
      int lo;
      const int bn = block_range(b, n_occ, &lo);
      rd.push_back(make_tile(lo, bn, 0, 0, 0, 0, true, 1, 0));
    }
    rounds.push_back(rd);
  } else {
    const int nbo = (n_occ + tile - 1) / tile, nbx = (n_x + tile - 1) / tile;
    for (int r = 0; r < nbo; ++r) {
      std::vector<int> rd;
      for (int bx = 0; bx < nbx; ++bx) {
        const int bo = (bx + r) % nbo;
        int alo, blo;
        const int an = block_range(bo, n_occ, &alo), bn = block_range(bx, n_x, &blo);
        rd.push_back(make_tile(alo, an, 0, blo, bn, 1, false, 0, 1));
      }
      rounds.push_back(rd);
    }
  }
  // order tiles by round and split rounds into launches of at most tiles_per_launch
  std::vector<PairTile> ordered;
  std::vector<int> lf, lc;
  for (auto& rd : rounds) {
    for (size_t k = 0; k < rd.size(); k += tiles_per_launch) {
      const int cnt = (int)std::min<size_t>(tiles_per_launch, rd.size() - k);
      lf.push_back((int)ordered.size());
      lc.push_back(cnt);
      for (int q = 0; q < cnt; ++q) ordered.push_back(tiles[rd[k + q]]);
    }
  }
  *tiles_out = (PairTile*)std::malloc(sizeof(PairTile) * ordered.size());
  std::memcpy(*tiles_out, ordered.data(), sizeof(PairTile) * ordered.size());
  *launch_first = (int*)std::malloc(sizeof(int) * lf.size());
  *launch_count = (int*)std::malloc(sizeof(int) * lc.size());
  std::memcpy(*launch_first, lf.data(), sizeof(int) * lf.size());
  std::memcpy(*launch_count, lc.data(), sizeof(int) * lc.size());
  *n_launch = (int)lf.size();
  return (int)ordered.size();
}

}  // namespace pt
