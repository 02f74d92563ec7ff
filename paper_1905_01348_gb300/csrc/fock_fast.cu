// FP32 pair pipeline for cubic grids of 32, 64 or 96 points per edge (the
// Si8 / Si64 / Si216 workloads): the same three passes as fock.cu (Eq. 3,
// pair loop of Alg. 2) with compile-time line lengths and two-stage radix
// plans, padded shared memory, the screened-kernel multiply fused between the
// last forward and the first inverse stage of axis 0, and accumulation
// through per-output contribution lists.
#include <algorithm>

#include "common.cuh"
#include "fft_ct.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int TT = kTileMax;   // orbitals per tile edge
constexpr int RR = 4;          // grid rows per block in F1 / F3
constexpr int NPAIR = TT * TT;

template <int L> struct Cfg;
template <> struct Cfg<32> { static constexpr int NT13 = 256, NT2 = 128, MIN2 = 4; };
template <> struct Cfg<64> { static constexpr int NT13 = 256, NT2 = 512, MIN2 = 1; };
template <> struct Cfg<96> { static constexpr int NT13 = 256, NT2 = 768, MIN2 = 1; };

template <int L> constexpr size_t smem13() {
  return sizeof(float2) * (size_t)(L + 2 * TT * RR * L + padded(NPAIR * RR * L));
}
template <int L> constexpr size_t smem2() { return sizeof(float2) * (size_t)(L + padded(L * L)); }

}  // namespace

// F1: pair products of RR grid rows for every pair of the tile, forward FFT
// along axis 2, store X[slot][i2][i0][i1].
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13) k_fast_f1(const float2* __restrict__ psi_r,
                                                          const float2* __restrict__ x_r,
                                                          const PairTile* __restrict__ tiles, int tile0,
                                                          float2* __restrict__ X, const float2* __restrict__ tw_g) {
  constexpr int NT = Cfg<L>::NT13;
  constexpr int ROW = RR * L;
  constexpr long N = (long)L * L * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairTile tl;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* orb = tw + L;
  float2* work = orb + 2 * TT * ROW;
  const int tid = threadIdx.x;
  if (tid == 0) tl = tiles[tile0 + blockIdx.y];
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  __syncthreads();
  constexpr int NB1 = L / RR;
  const int i0 = blockIdx.x / NB1;
  const int i1s = (blockIdx.x % NB1) * RR;
  const long roff = ((long)i0 * L + i1s) * L;
  for (int o = 0; o < tl.n_orb; ++o) {
    const float4* src = reinterpret_cast<const float4*>((tl.src[o] == 0 ? psi_r : x_r) + (long)tl.orb[o] * N + roff);
    float4* dst = reinterpret_cast<float4*>(orb + o * ROW);
    for (int e = tid; e < ROW / 2; e += NT) dst[e] = src[e];
  }
  __syncthreads();
  const int np = tl.n_pairs;
  for (int idx = tid; idx < np * ROW; idx += NT) {
    const int p = idx / ROW, e = idx % ROW;
    work[pidx(idx)] = cmulc(orb[tl.pi[p] * ROW + e], orb[tl.pj[p] * ROW + e]);
  }
  __syncthreads();
  ct_forward<float2, L, NPAIR * RR, NT, true, L, 1>(work, np * RR, tw, tid);
  const long slot0 = (long)blockIdx.y * NPAIR;
  for (int idx = tid; idx < np * ROW; idx += NT) {
    const int r = idx % RR;
    const int rest = idx / RR;
    const int i2 = rest % L;
    const int p = rest / L;
    X[(((slot0 + p) * L + i2) * L + i0) * L + i1s + r] = work[pidx((p * RR + r) * L + i2)];
  }
}

// F2: one (pair, i2) slab: FFT along axis 1 and axis 0, multiply by the
// screened kernel, inverse along axis 0 and axis 1.
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT2, Cfg<L>::MIN2) k_fast_f2(float2* __restrict__ X, const PairTile* __restrict__ tiles,
                                                         int tile0, const float* __restrict__ khat_t,
                                                         const float2* __restrict__ tw_g) {
  constexpr int NT = Cfg<L>::NT2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int slot = blockIdx.y;
  if (slot % NPAIR >= tiles[tile0 + slot / NPAIR].n_pairs) return;
  const int i2 = blockIdx.x;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* buf = tw + L;
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  float2* slab = X + ((long)slot * L + i2) * (L * L);
  for (int e = tid; e < L * L; e += NT) buf[pidx(e)] = slab[e];
  __syncthreads();
  ct_forward<float2, L, L, NT, true, L, 1>(buf, L, tw, tid);          // axis 1 (rows)
  ct_forward_stage1<float2, L, L, NT, false, 1, L>(buf, L, tw, tid);  // axis 0 (columns)
  const float* kt = khat_t + (long)i2 * (L * L);
  ct_fused<float2, L, L, NT, false, 1, L>(buf, L, tw, tid, [kt](int line, int e) { return kt[e * L + line]; });
  ct_inverse_stage2<float2, L, L, NT, false, 1, L>(buf, L, tw, tid);
  ct_inverse<float2, L, L, NT, true, L, 1>(buf, L, tw, tid);
  for (int e = tid; e < L * L; e += NT) slab[e] = buf[pidx(e)];
}

// F3: inverse FFT along axis 2 for all pairs of the tile, then each output
// orbital adds its listed contributions to its W rows (one writer per row).
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13) k_fast_f3(const float2* __restrict__ psi_r,
                                                          const float2* __restrict__ x_r, float2* __restrict__ w_occ,
                                                          float2* __restrict__ w_x, const PairTile* __restrict__ tiles,
                                                          int tile0, const float2* __restrict__ X,
                                                          const float2* __restrict__ tw_g) {
  constexpr int NT = Cfg<L>::NT13;
  constexpr int ROW = RR * L;
  constexpr long N = (long)L * L * L;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ PairTile tl;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* orb = tw + L;
  float2* work = orb + 2 * TT * ROW;
  const int tid = threadIdx.x;
  if (tid == 0) tl = tiles[tile0 + blockIdx.y];
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  __syncthreads();
  constexpr int NB1 = L / RR;
  const int i0 = blockIdx.x / NB1;
  const int i1s = (blockIdx.x % NB1) * RR;
  const long roff = ((long)i0 * L + i1s) * L;
  const int np = tl.n_pairs;
  const long slot0 = (long)blockIdx.y * NPAIR;
  for (int idx = tid; idx < np * ROW; idx += NT) {
    const int r = idx % RR;
    const int rest = idx / RR;
    const int i2 = rest % L;
    const int p = rest / L;
    work[pidx((p * RR + r) * L + i2)] = X[(((slot0 + p) * L + i2) * L + i0) * L + i1s + r];
  }
  for (int o = 0; o < tl.n_orb; ++o) {
    const float4* src = reinterpret_cast<const float4*>((tl.src[o] == 0 ? psi_r : x_r) + (long)tl.orb[o] * N + roff);
    float4* dst = reinterpret_cast<float4*>(orb + o * ROW);
    for (int e = tid; e < ROW / 2; e += NT) dst[e] = src[e];
  }
  __syncthreads();
  ct_inverse<float2, L, NPAIR * RR, NT, true, L, 1>(work, np * RR, tw, tid);
  for (int o = 0; o < tl.n_orb; ++o) {
    const int n = tl.out_n[o];
    if (!tl.is_out[o] || n == 0) continue;
    float2* dst = (tl.src[o] == 0 ? w_occ : w_x) + (long)tl.orb[o] * N + roff;
    for (int e = tid; e < ROW; e += NT) {
      float2 acc = make_float2(0.f, 0.f);
      for (int c = 0; c < n; ++c) {
        const float2 v = work[pidx(tl.out_pair[o][c] * ROW + e)];
        const float2 a = orb[tl.out_other[o][c] * ROW + e];
        acc = cadd(acc, tl.out_conj[o][c] ? cmul_conj(a, v) : cmul(a, v));
      }
      dst[e] = cadd(dst[e], acc);
    }
  }
}

template <int L>
static cudaError_t launch_fast(const void* psi_r, const void* x_r, void* w_occ, void* w_x, const FockPlan& plan,
                               const float* khat_t, void* scratch, const float2* tw, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_fast_f1<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f2<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<L>());
    if (e != cudaSuccess) return e;
    attr = true;
  }
  float2* X = (float2*)scratch;
  for (int l = 0; l < plan.n_launch; ++l) {
    const int t0 = plan.launch_first[l], nt = plan.launch_count[l];
    dim3 g13((unsigned)(L * (L / RR)), (unsigned)nt);
    k_fast_f1<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>((const float2*)psi_r, (const float2*)x_r, plan.d_tiles, t0, X,
                                                         tw);
    dim3 g2((unsigned)L, (unsigned)(nt * NPAIR));
    k_fast_f2<L><<<g2, Cfg<L>::NT2, smem2<L>(), s>>>(X, plan.d_tiles, t0, khat_t, tw);
    k_fast_f3<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>((const float2*)psi_r, (const float2*)x_r, (float2*)w_occ,
                                                         (float2*)w_x, plan.d_tiles, t0, X, tw);
    launched(3);
  }
  return cudaGetLastError();
}

bool fock_fast_supported(Grid3 g) {
  return g.n0 == g.n1 && g.n1 == g.n2 && (g.n0 == 32 || g.n0 == 64 || g.n0 == 96);
}

cudaError_t fock_pairs_fast(const void* psi_r, const void* x_r, void* w_occ, void* w_x, const FockPlan& plan, Grid3 g,
                            const float* khat_t, void* scratch, const float2* tw_L, cudaStream_t s) {
  switch (g.n0) {
    case 32: return launch_fast<32>(psi_r, x_r, w_occ, w_x, plan, khat_t, scratch, tw_L, s);
    case 64: return launch_fast<64>(psi_r, x_r, w_occ, w_x, plan, khat_t, scratch, tw_L, s);
    case 96: return launch_fast<96>(psi_r, x_r, w_occ, w_x, plan, khat_t, scratch, tw_L, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pt
