// FP32 pair pipeline for cubic grids of 32, 48, 64 or 96 points per edge (the
// Si8 / Si64 / Si216 workloads, and 48 for the Si216 wavefunction grid): the same three passes as fock.cu (Eq. 3,
// pair loop of Alg. 2) with compile-time line lengths and two-stage radix
// plans, padded and transposed shared-memory rows (no bank conflicts), the
// screened-kernel multiply fused between the last forward and the first
// inverse stage of axis 0, accumulation through per-output contribution
// lists, asynchronous global->shared copies for the pair intermediate, and
// no work on the axis-2 frequency slabs that pair products cannot reach.
#include <algorithm>

#include "common.cuh"
#include "fft_ct.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int TT = kTileMax;   // orbitals per tile edge
constexpr int RR = 4;          // grid rows per block in F1 / F3
constexpr int NPAIR = TT * TT;

template <int L> struct Cfg { static constexpr int NT13 = 256; };

template <int L> constexpr int WS = L + 1;   // work-buffer row stride (complex values)

template <int L> constexpr size_t smem13() { return sizeof(float2) * (size_t)(L + NPAIR * RR * WS<L>); }

// Row layout of the F1 / F3 work buffer: row l (pair p, grid row r) at stride
// L + 1, and inside each aligned group of 16 elements the 4 x 4 block is
// transposed (element 4a + b sits at 4b + a). FFT stages access one element of
// 16 consecutive rows per half-warp (distinct banks through the odd stride);
// the X loads and stores access 4 rows x 4 consecutive elements per half-warp,
// which the transpose also spreads over 16 distinct bank pairs.
template <int L> struct RowsT {
  __device__ __forceinline__ static int at(int l, int e) {
    return l * WS<L> + ((e & ~15) | ((e & 3) << 2) | ((e >> 2) & 3));
  }
};

__device__ __forceinline__ void cp_async8(void* smem_dst, const void* gsrc) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Axis-2 slab i2 is dead when its frequency lies beyond the pair reach R:
// the pair products have no component there (the slab stays unwritten in X).
template <int L> __device__ __forceinline__ bool dead_slab(int i2, int reach) { return i2 > reach && i2 < L - reach; }

// An off-diagonal tile of two full orbital blocks: orbitals 0..3 and 4..7,
// pair 4a + b = (a, 4 + b).
__device__ __forceinline__ bool full_tile(const PairTile& tl) { return tl.n_orb == 2 * TT && tl.n_pairs == NPAIR; }

__device__ __forceinline__ const float2* orb_ptr(const PairTile& tl, int o) {
  return static_cast<const float2*>(tl.in[o]);
}
__device__ __forceinline__ float2* acc_ptr(const PairTile& tl, int o) { return static_cast<float2*>(tl.out[o]); }

}  // namespace

// F1: pair products of RR grid rows for every pair of the tile (orbital rows
// read through the read-only cache, four products per thread per round with
// all their loads issued first), forward FFT along axis 2, store the live
// slabs of X[slot][i2][i0][i1].
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13, 4) k_fast_f1(const PairTile* __restrict__ tiles, int tile0,
                                                          float2* __restrict__ X, const float2* __restrict__ tw_g,
                                                          int reach) {
  using A = RowsT<L>;
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
  if (full_tile(tl)) {
    // off-diagonal 4 x 4 tile: pair 4a + b is (a, 4 + b); the eight orbital
    // values of an element are loaded once (eight loads in flight)
    for (int e = tid; e < ROW; e += NT) {
      float2 v[2 * TT];
#pragma unroll
      for (int o = 0; o < 2 * TT; ++o) v[o] = __ldg(orb_ptr(tl, o) + roff + e);
      const int row = e / L, col = e % L;
#pragma unroll
      for (int a = 0; a < TT; ++a)
#pragma unroll
        for (int b = 0; b < TT; ++b) work[A::at((a * TT + b) * RR + row, col)] = cmulc(v[a], v[TT + b]);
    }
  } else {
    // any tile: four products per thread per round, all eight loads issued before the first use
    constexpr int U = 4;
    for (int base = tid; base < np * ROW; base += U * NT) {
      float2 a[U], b[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NT;
        if (idx < np * ROW) {
          const int p = idx / ROW, e = idx % ROW;
          a[u] = __ldg(orb_ptr(tl, tl.pi[p]) + roff + e);
          b[u] = __ldg(orb_ptr(tl, tl.pj[p]) + roff + e);
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = base + u * NT;
        if (idx < np * ROW) {
          const int p = idx / ROW, e = idx % ROW;
          work[A::at(p * RR + e / L, e % L)] = cmulc(a[u], b[u]);
        }
      }
    }
  }
  __syncthreads();
  ct_forward_lay<float2, L, NPAIR * RR, NT, A>(work, np * RR, tw, tid);
  // lanes: r fastest, then i2, so each (pair, i2) writes one run of RR values along i1
  const long slot0 = (long)blockIdx.y * NPAIR;
  const int r = tid % RR;
  for (int p = 0; p < np; ++p) {
    float2* xp = X + (slot0 + p) * N + (long)i0 * L + i1s + r;
    for (int i2 = tid / RR; i2 < L; i2 += NT / RR)
      if (!dead_slab<L>(i2, reach)) xp[(long)i2 * L * L] = work[A::at(p * RR + r, i2)];
  }
}

// Register-line transforms of 96-point lines (L = 96 = 12 x 8, n = n1 + 12 n2,
// k = k2 + 8 k1): two threads share a line, thread half h holding n1 in [6h, 6h + 6)
// (48 values); the partner is the lane XM apart. Used by F2 at 96^3.
namespace l96 {
constexpr int L = 96, W = L + 1;

// Twiddle indices n1 k2 stay below 96 (n1 < 12, k2 < 8), so they need no reduction.

// 8-point DFTs over n2 of the owned n1 = 6h + a, then the twiddle W96^(n1 k2) (forward)
__device__ __forceinline__ void stage_a_fwd(float2 (&v)[6][8], int h, const float2* tw) {
  const int h6 = 6 * h;
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    dft<8, false>(v[a]);
#pragma unroll
    for (int k2 = 1; k2 < 8; ++k2) v[a][k2] = cmul(v[a][k2], tw[a * k2 + h6 * k2]);
  }
}

// inverse 8-point DFTs over k2: v[a][n2] = x[6h + a + 12 n2]
__device__ __forceinline__ void stage_a_inv(float2 (&v)[6][8]) {
#pragma unroll
  for (int a = 0; a < 6; ++a) dft<8, true>(v[a]);
}

// forward exchange for k2 = 4h + b: z[n1], n1 = 0..11, from the owned v[.][b or 4 + b] and the partner's
template <int XM = 1>
__device__ __forceinline__ void exch_fwd(const float2 (&v)[6][8], int h, int b, float2 (&z)[12]) {
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float2 mine = h ? v[a][4 + b] : v[a][b];   // my k2 = 4h + b
    const float2 send = h ? v[a][b] : v[a][4 + b];   // the partner's k2 = 4(1 - h) + b
    float2 got;
    got.x = __shfl_xor_sync(0xffffffffu, send.x, XM);
    got.y = __shfl_xor_sync(0xffffffffu, send.y, XM);
    z[a] = h ? got : mine;        // n1 = a (owned by half 0)
    z[6 + a] = h ? mine : got;    // n1 = 6 + a (owned by half 1)
  }
}

// inverse twiddle of Z[n1][k2], k2 = 4h + b, then the exchange back into v[a][b], v[a][4 + b]
template <int XM = 1>
__device__ __forceinline__ void exch_inv(float2 (&z)[12], int h, int b, const float2* tw, float2 (&v)[6][8]) {
  const int h4 = 4 * h;
#pragma unroll
  for (int n1 = 1; n1 < 12; ++n1) {
    float2 w = tw[n1 * b + n1 * h4];
    w.y = -w.y;
    z[n1] = cmul(z[n1], w);
  }
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float2 mine = h ? z[6 + a] : z[a];          // my n1 = 6h + a
    const float2 send = h ? z[a] : z[6 + a];          // the partner's n1
    float2 got;
    got.x = __shfl_xor_sync(0xffffffffu, send.x, XM);
    got.y = __shfl_xor_sync(0xffffffffu, send.y, XM);  // my n1, the partner's k2 = 4(1 - h) + b
    v[a][b] = h ? got : mine;
    v[a][4 + b] = h ? mine : got;
  }
}
}  // namespace l96

// F2: one live (pair, i2) slab per block: asynchronous copies into the padded
// work buffer, FFT along axis 1 and axis 0, multiply by the screened kernel
// (fused between the last forward and first inverse stage of axis 0), inverse
// along axis 0 and axis 1, store. Blocks are small so that two or more are
// resident per SM and one block's barrier waits overlap another's work (this
// beat a single persistent block per SM fed by bulk-copy prefetch, and one
// block of 384 threads without sub-batches).
template <int L> struct Cfg2;
template <> struct Cfg2<32> { static constexpr int NT = 128, SUB = 32, MINB = 4; };
template <> struct Cfg2<48> { static constexpr int NT = 192, SUB = 48, MINB = 4; };
template <> struct Cfg2<64> { static constexpr int NT = 256, SUB = 32, MINB = 3; };
// 96: 192 threads balance both radices (48 lines x 12 radix-8 or 8 radix-12
// butterflies = 3 or 2 per thread) and leave room for 152 registers without spills.
template <> struct Cfg2<96> { static constexpr int NT = 192, SUB = 48, MINB = 2; };
template <int L> constexpr size_t smem2() { return sizeof(float2) * (size_t)(L + L * WS<L>); }

template <int L>
__global__ void __launch_bounds__(Cfg2<L>::NT, Cfg2<L>::MINB) k_fast_f2(float2* __restrict__ X,
                                                                         const PairTile* __restrict__ tiles, int tile0,
                                                                         const float* __restrict__ khat_t,
                                                                         const float2* __restrict__ tw_g, int reach) {
  constexpr int NT = Cfg2<L>::NT;
  constexpr int SUB = Cfg2<L>::SUB;
  static_assert(L % SUB == 0, "the sub-batches of SUB lines must tile the L lines of a slab exactly");
  constexpr int SLAB = L * L;
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  constexpr int W = WS<L>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int tid = threadIdx.x;
  const int slot = blockIdx.y;
  if (slot % NPAIR >= tiles[tile0 + slot / NPAIR].n_pairs) return;
  // live slabs only: blockIdx.x in [0, n_live) maps to frequencies 0..R, then -R..-1
  const int i2 = (int)blockIdx.x <= reach ? (int)blockIdx.x : (int)blockIdx.x + (L - (int)gridDim.x);
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* buf = tw + L;
  for (int t = tid; t < L; t += NT) tw[t] = tw_g[t];
  float2* slab = X + ((long)slot * L + i2) * SLAB;
  for (int e = tid; e < SLAB; e += NT) cp_async8(buf + (e / L) * W + e % L, slab + e);
  cp_async_wait_all();
  __syncthreads();
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, false, L, R1, 1, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, false, L, R2, R1, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, false, L, R1, 1, SUB, NT, 1, W>(buf, SUB, tw, tid, l0);
  const float* kt = khat_t + (long)i2 * SLAB;
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB)
    ct_fused<float2, L, SUB, NT, 1, W>(buf, SUB, tw, tid, [kt](int line, int e) { return __ldg(kt + e * L + line); },
                                      l0);
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, true, L, R1, R2, SUB, NT, 1, W>(buf, SUB, tw, tid, l0);
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, true, L, R2, 1, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);
#pragma unroll 1
  for (int l0 = 0; l0 < L; l0 += SUB) ct_stage<float2, true, L, R1, R2, SUB, NT, W, 1>(buf, SUB, tw, tid, l0);
  for (int e = tid; e < SLAB; e += NT) slab[e] = buf[(e / L) * W + e % L];
}

// F2 for 96-point lines with the lines in registers. Two threads share a line of
// L = 96 = 12 x 8 points, n = n1 + 12 n2, k = k2 + 8 k1: thread half h holds the
// points of n1 in [6h, 6h + 6) (48 values). Forward: 8-point DFTs over n2 in registers
// (twiddle W96^(n1 k2)), then the two halves exchange by warp shuffles so that half h
// holds k2 in [4h, 4h + 4) for all twelve n1, and 12-point DFTs over n1 give the outputs
// k2 + 8 k1. The inverse runs the same steps backwards. The slab arrives by cp.async
// into a shared buffer (rows padded to 97) and leaves from it; between the passes the
// lines cross shared memory once per pass instead of once per radix stage. Column
// pass: for each owned k2, forward 12-point DFT, kernel multiply, inverse 12-point DFT,
// all in registers.

template <int L>
__global__ void __launch_bounds__(192, 2) k_fast_f2r(float2* __restrict__ X, const PairTile* __restrict__ tiles,
                                                     int tile0, const float* __restrict__ khat_t,
                                                     const float2* __restrict__ tw_g, int reach) {
  static_assert(L == l96::L, "register-line F2 is written for 96-point lines");
  using namespace l96;
  constexpr int SLAB = L * L;
  constexpr int XM = 16;                      // the two halves of a line are the lanes 16 apart
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float2* tw = reinterpret_cast<float2*>(smem_raw);
  float2* buf = tw + L;                       // [row][W]
  const int tid = threadIdx.x, lane = tid & 31;
  // a half-warp holds the same half h of 16 consecutive lines: its shared-memory accesses
  // (one row of 16 lines, or 16 columns of one row) fall on distinct banks
  const int line = (tid >> 5) * 16 + (lane & 15), h = lane >> 4;
  const int slot = blockIdx.y;
  if (slot % NPAIR >= tiles[tile0 + slot / NPAIR].n_pairs) return;
  const int i2 = (int)blockIdx.x <= reach ? (int)blockIdx.x : (int)blockIdx.x + (L - (int)gridDim.x);
  for (int t = tid; t < L; t += 192) tw[t] = tw_g[t];
  float2* slab = X + ((long)slot * L + i2) * SLAB;
  for (int e = tid; e < SLAB; e += 192) cp_async8(buf + (e / L) * W + e % L, slab + e);
  cp_async_wait_all();
  __syncthreads();
  float2 v[6][8];
  // ---- forward along axis 1 (rows): v[a][n2] = x[6h + a + 12 n2] of row `line`; outputs
  // k = k2 + 8 k1 back into the row
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2)
#pragma unroll
    for (int a = 0; a < 6; ++a) v[a][n2] = buf[line * W + 6 * h + a + 12 * n2];
  __syncthreads();   // every row is in registers before any is overwritten
  stage_a_fwd(v, h, tw);
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    float2 z[12];
    exch_fwd<XM>(v, h, b, z);
    dft12<false>(z);
#pragma unroll
    for (int k1 = 0; k1 < 12; ++k1) buf[line * W + 4 * h + b + 8 * k1] = z[k1];
  }
  __syncthreads();
  // ---- axis 0 (columns): column c = line; forward, kernel multiply, inverse, in registers
  {
    const int c = line;
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2)
#pragma unroll
      for (int a = 0; a < 6; ++a) v[a][n2] = buf[(6 * h + a + 12 * n2) * W + c];
    stage_a_fwd(v, h, tw);
    const float* kt = khat_t + (long)i2 * SLAB + c;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float2 z[12];
      exch_fwd<XM>(v, h, b, z);
      dft12<false>(z);                                   // frequency k0 = 4h + b + 8 k1 along axis 0
#pragma unroll
      for (int k1 = 0; k1 < 12; ++k1) z[k1] = cscale(z[k1], __ldg(kt + (4 * h + b + 8 * k1) * L));
      dft12<true>(z);                                    // back to n1, this k2
      exch_inv<XM>(z, h, b, tw, v);
    }
    stage_a_inv(v);
#pragma unroll
    for (int n2 = 0; n2 < 8; ++n2)
#pragma unroll
      for (int a = 0; a < 6; ++a) buf[(6 * h + a + 12 * n2) * W + c] = v[a][n2];
  }
  __syncthreads();
  // ---- inverse along axis 1 (rows): inputs k2 + 8 k1 of row `line`, outputs back into it
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    float2 z[12];
#pragma unroll
    for (int k1 = 0; k1 < 12; ++k1) z[k1] = buf[line * W + 4 * h + b + 8 * k1];
    dft12<true>(z);
    exch_inv<XM>(z, h, b, tw, v);
  }
  stage_a_inv(v);
  __syncthreads();   // every row is in registers before any is overwritten
#pragma unroll
  for (int n2 = 0; n2 < 8; ++n2)
#pragma unroll
    for (int a = 0; a < 6; ++a) buf[line * W + 6 * h + a + 12 * n2] = v[a][n2];
  __syncthreads();
  for (int e = tid; e < SLAB; e += 192) slab[e] = buf[(e / L) * W + e % L];
}

// F3: inverse FFT along axis 2 for all pairs of the tile, then each output
// orbital adds its listed contributions to its W rows (one writer per row).
// The live slabs of X arrive by asynchronous copies straight into shared
// memory (no registers held while the loads are in flight); dead slabs are zero.
// Three resident blocks per SM (rather than F1's four) leave F3 the registers to keep the
// orbital and W loads of its accumulation in flight together (9% faster at 96^3).
template <int L>
__global__ void __launch_bounds__(Cfg<L>::NT13, 3) k_fast_f3(const PairTile* __restrict__ tiles, int tile0,
                                                          const float2* __restrict__ X,
                                                          const float2* __restrict__ tw_g, int reach) {
  using A = RowsT<L>;
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
  const int r = tid % RR;
  for (int p = 0; p < np; ++p) {
    const float2* xp = X + (slot0 + p) * N + (long)i0 * L + i1s + r;
    for (int i2 = tid / RR; i2 < L; i2 += NT / RR) {
      float2* dst = work + A::at(p * RR + r, i2);
      if (dead_slab<L>(i2, reach)) *dst = make_float2(0.f, 0.f);
      else cp_async8(dst, xp + (long)i2 * L * L);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  ct_inverse_lay<float2, L, NPAIR * RR, NT, A>(work, np * RR, tw, tid);
  if (full_tile(tl)) {
    // off-diagonal 4 x 4 tile: output a (< 4) takes psi_{4+b} conj(v_ab) over b, output
    // 4 + b takes psi_a v_ab over a, in the order of the contribution lists; all orbital
    // and W loads of an element are issued together
    for (int e = tid; e < ROW; e += NT) {
      const int row = e / L, col = e % L;
      float2 v[2 * TT], w[2 * TT];
      float2* dst[2 * TT];
#pragma unroll
      for (int o = 0; o < 2 * TT; ++o) {
        v[o] = __ldg(orb_ptr(tl, o) + roff + e);
        dst[o] = tl.is_out[o] ? acc_ptr(tl, o) + roff + e : nullptr;
        if (tl.is_out[o]) w[o] = *dst[o];
      }
#pragma unroll
      for (int a = 0; a < TT; ++a) {
        if (!tl.is_out[a]) continue;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int b = 0; b < TT; ++b) acc = cadd(acc, cmul_conj(v[TT + b], work[A::at((a * TT + b) * RR + row, col)]));
        *dst[a] = cadd(w[a], acc);
      }
#pragma unroll
      for (int b = 0; b < TT; ++b) {
        if (!tl.is_out[TT + b]) continue;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 0; a < TT; ++a) acc = cadd(acc, cmul(v[a], work[A::at((a * TT + b) * RR + row, col)]));
        *dst[TT + b] = cadd(w[TT + b], acc);
      }
    }
    return;
  }
  for (int o = 0; o < tl.n_orb; ++o) {
    const int n = tl.out_n[o];
    if (!tl.is_out[o] || n == 0) continue;
    float2* dst = acc_ptr(tl, o) + roff;
    for (int e = tid; e < ROW; e += NT) {
      const int r = e / L, i2 = e % L;
      float2 acc = make_float2(0.f, 0.f);
      for (int c = 0; c < n; ++c) {
        const float2 v = work[A::at(tl.out_pair[o][c] * RR + r, i2)];
        const float2 a = __ldg(orb_ptr(tl, tl.out_other[o][c]) + roff + e);
        acc = cadd(acc, tl.out_conj[o][c] ? cmul_conj(a, v) : cmul(a, v));
      }
      dst[e] = cadd(dst[e], acc);
    }
  }
}

template <int L>
static cudaError_t launch_fast(const FockPlan& plan, const float* khat_t, void* scratch, const float2* tw,
                               cudaStream_t s) {
  static std::atomic<unsigned long long> attr_done{0};
  if (const unsigned long long bit = device_bit_todo(attr_done)) {
    cudaError_t e = cudaFuncSetAttribute(k_fast_f1<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f3<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem13<L>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_fast_f2<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<L>());
    if (e != cudaSuccess) return e;
    if constexpr (L == 96) {
      e = cudaFuncSetAttribute(k_fast_f2r<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2<L>());
      if (e != cudaSuccess) return e;
    }
    attr_done.fetch_or(bit, std::memory_order_release);
  }
  float2* X = (float2*)scratch;
  const int reach = 2 * plan.g2_reach + 1 < L ? plan.g2_reach : L;
  const int n_live = reach >= L ? L : 2 * reach + 1;
  for (int l = 0; l < plan.n_launch; ++l) {
    const int t0 = plan.launch_first[l], nt = plan.launch_count[l];
    dim3 g13((unsigned)(L * (L / RR)), (unsigned)nt);
    k_fast_f1<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>(plan.d_tiles, t0, X, tw, reach);
    dim3 g2((unsigned)n_live, (unsigned)(nt * NPAIR));
    if constexpr (L == 96) k_fast_f2r<L><<<g2, 192, smem2<L>(), s>>>(X, plan.d_tiles, t0, khat_t, tw, reach);
    else k_fast_f2<L><<<g2, Cfg2<L>::NT, smem2<L>(), s>>>(X, plan.d_tiles, t0, khat_t, tw, reach);
    k_fast_f3<L><<<g13, Cfg<L>::NT13, smem13<L>(), s>>>(plan.d_tiles, t0, X, tw, reach);
    launched(3);
  }
  return cudaGetLastError();
}

bool fock_fast_supported(Grid3 g) {
  return g.n0 == g.n1 && g.n1 == g.n2 && (g.n0 == 32 || g.n0 == 48 || g.n0 == 64 || g.n0 == 96);
}

cudaError_t fock_pairs_fast(const FockPlan& plan, Grid3 g, const float* khat_t, void* scratch, const float2* tw_L,
                            cudaStream_t s) {
  switch (g.n0) {
    case 32: return launch_fast<32>(plan, khat_t, scratch, tw_L, s);
    case 48: return launch_fast<48>(plan, khat_t, scratch, tw_L, s);
    case 64: return launch_fast<64>(plan, khat_t, scratch, tw_L, s);
    case 96: return launch_fast<96>(plan, khat_t, scratch, tw_L, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace pt
