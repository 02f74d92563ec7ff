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

// NT2 threads transform SUB lines of a slab per stage call (L / SUB calls per stage).
template <int L> struct Cfg;
template <> struct Cfg<32> { static constexpr int NT13 = 256, NT2 = 128, SUB = 32; };
template <> struct Cfg<64> { static constexpr int NT13 = 256, NT2 = 512, SUB = 64; };
template <> struct Cfg<96> { static constexpr int NT13 = 256, NT2 = 576, SUB = 48; };

template <int L> constexpr int WS = L + 1;   // work-buffer row stride (complex values)
template <int L> constexpr int LS = L + 2;   // landing-buffer row stride (16-byte multiple)

template <int L> constexpr size_t smem13() { return sizeof(float2) * (size_t)(L + NPAIR * RR * WS<L>); }
template <int L> constexpr size_t smem2() { return sizeof(float2) * (size_t)(L * LS<L> + L + L * WS<L>); }

__device__ __forceinline__ const float2* orb_ptr(const PairTile& tl, int o, const float2* psi_r, const float2* x_r,
                                                 long N) {
  return (tl.src[o] == 0 ? psi_r : x_r) + (long)tl.orb[o] * N;
}

// Warp 0 brings one (i0, i1) slab into the landing buffer, one bulk copy per row.
template <int L>
__device__ __forceinline__ void issue_slab(float2* land, const float2* slab, unsigned long long* bar) {
  constexpr uint32_t ROWB = L * sizeof(float2);
  const int lane = threadIdx.x;
  if (lane == 0) mbar_expect_tx(bar, ROWB * L);
  __syncwarp();
  for (int row = lane; row < L; row += 32) bulk_load(land + row * LS<L>, slab + (long)row * L, ROWB, bar);
}

}  // namespace

// F1: pair products of RR grid rows for every pair of the tile (orbital rows
// read through the read-only cache), forward FFT along axis 2, store
// X[slot][i2][i0][i1].
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13, 4) k_fast_f1(const float2* __restrict__ psi_r,
                                                          const float2* __restrict__ x_r,
                                                          const PairTile* __restrict__ tiles, int tile0,
                                                          float2* __restrict__ X, const float2* __restrict__ tw_g) {
  constexpr int NT = Cfg<L>::NT13;
  constexpr int ROW = RR * L;
  constexpr long N = (long)L * L * L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ PairTile tl;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* work = tw + L;
  const int tid = threadIdx.x;
  if (tid == 0) tl = tiles[tile0 + blockIdx.y];
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  __syncthreads();
  constexpr int NB1 = L / RR;
  const int i0 = blockIdx.x / NB1;
  const int i1s = (blockIdx.x % NB1) * RR;
  const long roff = ((long)i0 * L + i1s) * L;
  const int np = tl.n_pairs;
  for (int idx = tid; idx < np * ROW; idx += NT) {
    const int p = idx / ROW, e = idx % ROW;
    const float2 a = __ldg(orb_ptr(tl, tl.pi[p], psi_r, x_r, N) + roff + e);
    const float2 b = __ldg(orb_ptr(tl, tl.pj[p], psi_r, x_r, N) + roff + e);
    work[(p * RR + e / L) * WS<L> + e % L] = cmulc(a, b);
  }
  __syncthreads();
  ct_forward<float2, L, NPAIR * RR, NT, WS<L>, 1>(work, np * RR, tw, tid);
  const long slot0 = (long)blockIdx.y * NPAIR;
  for (int idx = tid; idx < np * ROW; idx += NT) {
    const int r = idx % RR;
    const int rest = idx / RR;
    const int i2 = rest % L;
    const int p = rest / L;
    X[(((slot0 + p) * L + i2) * L + i0) * L + i1s + r] = work[(p * RR + r) * WS<L> + i2];
  }
}

// F2: persistent blocks walk the (pair slot, i2) slabs of the launch. The
// next slab is brought into the landing buffer by bulk copies (TMA) as soon
// as the current one has been read out of it, so the load overlaps the
// transforms: FFT along axis 1 and axis 0, multiply by the screened kernel,
// inverse along axis 0 and axis 1. A wait that exceeds its iteration cap sets
// *err and ends the block after a second bounded wait for its copy in flight.
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT2, 1) k_fast_f2(float2* __restrict__ X, const PairTile* __restrict__ tiles,
                                                            int tile0, int nslot, const float* __restrict__ khat_t,
                                                            const float2* __restrict__ tw_g, int* __restrict__ err) {
  constexpr int NT = Cfg<L>::NT2;
  constexpr int SUB = Cfg<L>::SUB;
  constexpr int SLAB = L * L;
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  constexpr int W = WS<L>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) unsigned long long bar;
  __shared__ int s_abort;
  float2* land = reinterpret_cast<float2*>(smem_raw);
  float2* tw = land + L * LS<L>;
  float2* buf = tw + L;
  const int tid = threadIdx.x;
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  if (tid == 0) {
    mbar_init(&bar, 1);
    s_abort = 0;
  }
  __syncthreads();
  const long total = (long)nslot * L;
  auto active = [&](long sl) {
    const int slot = (int)(sl / L);
    return (slot % NPAIR) < tiles[tile0 + slot / NPAIR].n_pairs;
  };
  long s = blockIdx.x;
  while (s < total && !active(s)) s += gridDim.x;
  uint32_t phase = 0;
  bool in_flight = s < total;
  if (tid < 32 && s < total) issue_slab<L>(land, X + s * SLAB, &bar);
  while (s < total) {
    long nxt = s + gridDim.x;
    while (nxt < total && !active(nxt)) nxt += gridDim.x;
    if (!mbar_wait_bounded(&bar, phase)) atomicExch(&s_abort, 1);
    __syncthreads();
    if (s_abort) break;
    phase ^= 1u;
    in_flight = false;
    const int i2 = (int)(s % L);
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)   // axis 1 (rows), stage 1: landing buffer -> work buffer
      ct_stage_io<float2, false, L, R1, 1, SUB, NT, LS<L>, 1, W, 1>(land, buf, SUB, tw, tid, l0);
    if (nxt < total) {
      if (tid < 32) {
        if (tid == 0) fence_proxy_async_smem();
        __syncwarp();
        issue_slab<L>(land, X + nxt * SLAB, &bar);
      }
      in_flight = true;
    }
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_stage<float2, false, L, R2, R1, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);     // axis 1, stage 2
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_stage<float2, false, L, R1, 1, SUB, NT, 1, W>(buf, SUB, tw, tid, l0);      // axis 0, stage 1
    const float* kt = khat_t + (long)i2 * SLAB;
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_fused<float2, L, SUB, NT, 1, W>(buf, SUB, tw, tid,
                                        [kt](int line, int e) { return __ldg(kt + e * L + line); }, l0);
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_stage<float2, true, L, R1, R2, SUB, NT, 1, W>(buf, SUB, tw, tid, l0);      // axis 0, inverse stage 2
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_stage<float2, true, L, R2, 1, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);       // axis 1, inverse stage 1
#pragma unroll 1
    for (int l0 = 0; l0 < L; l0 += SUB)
      ct_stage<float2, true, L, R1, R2, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);      // axis 1, inverse stage 2
    float2* slab = X + s * SLAB;
    for (int e = tid; e < SLAB; e += NT) slab[e] = buf[(e / L) * W + e % L];
    s = nxt;
  }
  if (s_abort) {
    if (tid == 0) atomicExch(err, 1);
    if (in_flight) (void)mbar_wait_bounded(&bar, phase);
  }
}

// F3: inverse FFT along axis 2 for all pairs of the tile, then each output
// orbital adds its listed contributions to its W rows (one writer per row).
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13, 4) k_fast_f3(const float2* __restrict__ psi_r,
                                                          const float2* __restrict__ x_r, float2* __restrict__ w_occ,
                                                          float2* __restrict__ w_x, const PairTile* __restrict__ tiles,
                                                          int tile0, const float2* __restrict__ X,
                                                          const float2* __restrict__ tw_g) {
  constexpr int NT = Cfg<L>::NT13;
  constexpr int ROW = RR * L;
  constexpr long N = (long)L * L * L;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ PairTile tl;
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* work = tw + L;
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
    work[(p * RR + r) * WS<L> + i2] = X[(((slot0 + p) * L + i2) * L + i0) * L + i1s + r];
  }
  __syncthreads();
  ct_inverse<float2, L, NPAIR * RR, NT, WS<L>, 1>(work, np * RR, tw, tid);
  for (int o = 0; o < tl.n_orb; ++o) {
    const int n = tl.out_n[o];
    if (!tl.is_out[o] || n == 0) continue;
    float2* dst = (tl.src[o] == 0 ? w_occ : w_x) + (long)tl.orb[o] * N + roff;
    for (int e = tid; e < ROW; e += NT) {
      const int r = e / L, i2 = e % L;
      float2 acc = make_float2(0.f, 0.f);
      for (int c = 0; c < n; ++c) {
        const float2 v = work[(tl.out_pair[o][c] * RR + r) * WS<L> + i2];
        const float2 a = __ldg(orb_ptr(tl, tl.out_other[o][c], psi_r, x_r, N) + roff + e);
        acc = cadd(acc, tl.out_conj[o][c] ? cmul_conj(a, v) : cmul(a, v));
      }
      dst[e] = cadd(dst[e], acc);
    }
  }
}

template <int L>
static cudaError_t launch_fast(const void* psi_r, const void* x_r, void* w_occ, void* w_x, const FockPlan& plan,
                               const float* khat_t, void* scratch, const float2* tw, cudaStream_t s) {
  static bool init = false;
  static int grid2 = 0;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(k_fast_f1<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f2<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<L>());
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fast_f2<L>, Cfg<L>::NT2, smem2<L>());
    if (e != cudaSuccess) return e;
    grid2 = sms * std::max(1, per_sm);
    init = true;
  }
  if (plan.d_err == nullptr) return cudaErrorInvalidValue;
  float2* X = (float2*)scratch;
  for (int l = 0; l < plan.n_launch; ++l) {
    const int t0 = plan.launch_first[l], nt = plan.launch_count[l];
    dim3 g13((unsigned)(L * (L / RR)), (unsigned)nt);
    k_fast_f1<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>((const float2*)psi_r, (const float2*)x_r, plan.d_tiles, t0, X,
                                                         tw);
    k_fast_f2<L><<<grid2, Cfg<L>::NT2, smem2<L>(), s>>>(X, plan.d_tiles, t0, nt * NPAIR, khat_t, tw, plan.d_err);
    k_fast_f3<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>((const float2*)psi_r, (const float2*)x_r, (float2*)w_occ,
                                                         (float2*)w_x, plan.d_tiles, t0, X, tw);
    launched(3);
  }
  return cudaGetLastError();
}

// Self-test of the bounded wait: one block announces a transfer that is never
// issued and waits for it with a small cap; the wait must give up and the
// kernel must report it through *flag (no copy is ever in flight).
__global__ void k_selftest_wait(int* flag, int cap) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_expect_tx(&bar, 16);
  }
  __syncthreads();
  const bool ok = mbar_wait_bounded(&bar, 0, cap);
  if (threadIdx.x == 0) *flag = ok ? 0 : 1;
}

cudaError_t selftest_bounded_wait(int* d_flag, cudaStream_t s) {
  k_selftest_wait<<<1, 32, 0, s>>>(d_flag, 1 << 14);
  launched();
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
