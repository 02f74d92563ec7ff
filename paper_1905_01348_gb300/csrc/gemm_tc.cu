// Complex products of ACE and the PT projection on the 5th-generation tensor cores.
//
// C = alpha op(A) op(B) + beta C with complex64 inputs (the mixed-precision
// copies of Psi, W, xi, H Psi, X and the small N_e x N_e factors) and a
// complex128 C: M = Psi^H W and xi = W L^{-H} of the ACE build, xi^H X and
// -xi (xi^H X) of its application, S = Psi^H (H Psi) and H Psi - Psi S of the
// PT residual (Alg. 3). FP64 stays on the CUDA cores for the overlap, the
// Cholesky factorisations and the orthonormalisation (Sec. 3.4).
//
// Complex to real. With a_k = op(A)(m, k) and b_k = op(B)(k, n),
//   C_r = sum_k a_r b_r - a_i b_i,   C_i = sum_k a_r b_i + a_i b_r,
// is one real product over 2K: row m of A' interleaves (a_r, a_i) along k
// (the storage order of complex64 when op(A) reads along k), and B' holds for
// every output column two rows, (b_r, -b_i) for C_r and (b_i, b_r) for C_i.
// A tile of 128 complex output columns is therefore a 128 x 256 real tile.
//
// Precision (3xTF32): every operand value x is split into hi = tf32(x) and
// lo = tf32(x - hi) (round to nearest), and hi*hi + hi*lo + lo*hi is
// accumulated in FP32 in tensor memory (lo*lo, below 2^-22 relative, is
// dropped). Single-pass TF32 would keep only 11 significant bits.
//
// Kernel: one CTA per 128 x 128 complex output tile and K chunk (split-K for
// the long reductions over the basis, summed afterwards in a fixed order).
// Warps 0-3 load their row of A and column of B for a stage of 8 complex k,
// split and expand them, and store them into shared memory in the canonical
// K-major layout without swizzle (core matrices of 8 rows x 16 bytes); a ring
// of two stages is guarded by mbarriers. One thread of warp 4 issues
// tcgen05.mma (kind::tf32, M = 128, N = 256, K = 8) and releases each stage
// with tcgen05.commit. Warps 0-3 read the accumulators with tcgen05.ld (warp w
// owns TMEM lanes 32w..32w+31, i.e. output rows) and write C or the
// split-K partials. The accumulator is promoted into round-to-nearest FP32
// sums every 8 stages (see the kernel). Every wait is bounded: on expiry the
// kernel sets an error flag, stops issuing work and frees its tensor memory.
#include <algorithm>
#include <atomic>
#include <cstdint>

#include "common.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int TC_M = 128;            // output rows per tile (TMEM lanes)
constexpr int TC_NC = 128;           // complex output columns per tile (256 real accumulator columns)
constexpr int TC_KC = 8;             // complex k per stage (16 real k: two MMAs of K = 8)
constexpr int TC_NS = 2;             // ring stages
constexpr int TC_WIN = 8;            // stages per accumulation window (48 MMAs)
constexpr int TC_PF = 4;             // stages of operand loads in flight per producer thread
static_assert(TC_WIN % TC_PF == 0, "the producer loop steps through windows in groups of TC_PF stages");
constexpr int TC_PROD = 256;         // producer / drain threads (warps 0-7), two per tile row
constexpr int TC_THREADS = 288;      // + warp 8: tensor-memory allocation and MMA issue
constexpr uint32_t TC_TMEM_COLS = 512;                      // two accumulators of 256 columns
constexpr uint32_t A_BYTES = TC_M * 2 * TC_KC * 4;           // 128 rows x 16 floats
constexpr uint32_t B_BYTES = 2 * TC_NC * 2 * TC_KC * 4;      // 256 rows x 16 floats
constexpr uint32_t STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;  // [A hi][A lo][B hi][B lo]
constexpr uint32_t SUM_BYTES = 2 * TC_NC * TC_M * 4;         // FP32 window sums, [256 columns][128 rows]
constexpr uint32_t TC_SMEM = TC_NS * STAGE_BYTES + SUM_BYTES;  // 224 KB: one CTA per SM
constexpr long long kWaitCycles = 4000000000LL;              // about 2 s at 2 GHz

// Instruction descriptor of tcgen05.mma kind::tf32: FP32 accumulator (bits 4-5 = 1),
// A and B TF32 (bits 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at
// bits 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(2 * TC_NC) >> 3 << 17) |
                            ((uint32_t)TC_M >> 4 << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


// Shared-memory matrix descriptor, K-major without swizzle: the 8 x 16-byte core
// matrices are 128 contiguous bytes; LBO = 128 bytes to the next core matrix along K,
// SBO = 512 bytes to the next group of 8 rows (four core matrices of a stage row block
// lie along K). Bits 46-47 carry the descriptor version (1) of tcgen05.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)(128u >> 4) << 16;
  d |= (uint64_t)(512u >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(smem_u32(bar)) : "memory");
}

// Waits for the phase of the given parity to complete; false after kWaitCycles (the
// error flag is set then).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > kWaitCycles) {
      atomicOr(err, 1);
      return false;
    }
  }
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 16 consecutive columns: register i of lane l = column col + i of
// TMEM lane (lane base + l).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory"); }

// x = hi + lo with hi, lo TF32 values (round to nearest, ties away); x - hi is exact in FP32.
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  uint32_t h, l;
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(h) : "f"(x));
  hi = __uint_as_float(h);
  asm("cvt.rna.tf32.f32 %0, %1;\n" : "=r"(l) : "f"(x - hi));
  lo = __uint_as_float(l);
}

__device__ __forceinline__ void st_split(unsigned char* hi_base, unsigned char* lo_base, uint32_t off, float a, float b,
                                         float c, float d) {
  float4 h, l;
  split_tf32(a, h.x, l.x);
  split_tf32(b, h.y, l.y);
  split_tf32(c, h.z, l.z);
  split_tf32(d, h.w, l.w);
  *reinterpret_cast<float4*>(hi_base + off) = h;
  *reinterpret_cast<float4*>(lo_base + off) = l;
}

// byte offset of row r, core-matrix column kc (4 floats) inside an operand tile
__device__ __forceinline__ uint32_t core_off(int r, int kc) {
  return (uint32_t)(((r >> 3) * 4 + kc) * 128 + (r & 7) * 16);
}

}  // namespace

// One 128 x 128 complex tile of C over complex k in [kz * kchunk, min(K, (kz + 1) kchunk))
// (and k < n0 + 128 when op(B) is upper triangular). ksplit > 1: the raw sums go to
// part[(kz N + j) M + i]; otherwise C = alpha sum + beta C.
//
// Threads: warps 0-7 produce and drain, two threads per tile row r = 32 (w % 4) + lane
// (warp w reaches TMEM lanes 32 (w % 4)..+31); thread half h = w / 4 loads and converts
// complex k 4h..4h+3 of each stage (TC_PF stages ahead, in registers) and owns
// accumulator columns 128h..128h+127 (C_r for h = 0, C_i for h = 1). Warp 8 allocates
// tensor memory and one of its threads issues the MMAs.
//
// Accumulation. The tensor core adds into its FP32 accumulator with truncation, so its
// error grows linearly with the number of MMAs into one accumulator (measured: 4e-5
// relative after 2250 MMAs). Each window of TC_WIN stages (48 MMAs) therefore starts a
// fresh accumulator, and the producer threads add the finished window into FP32 sums in
// shared memory (round to nearest), one slice of 16 columns after each stage they
// produce. Two TMEM accumulators alternate, so the MMAs of window w run while window
// w - 1 is drained.
template <int OPA, int OPB>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_cgemm_tf32x3(int M, int N, int K, int kchunk, int ksplit, int tri_b, double2 alpha,
                   const float2* __restrict__ A, long lda, const float2* __restrict__ B, long ldb, double2 beta,
                   double2* __restrict__ Cm, long ldc, double2* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t bar_full[TC_NS];
  __shared__ __align__(8) uint64_t bar_empty[TC_NS];
  __shared__ __align__(8) uint64_t bar_acc_full[2];
  __shared__ __align__(8) uint64_t bar_acc_empty[2];
  __shared__ uint32_t tmem_base;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * TC_M, n0 = blockIdx.y * TC_NC, kz = blockIdx.z;
  const int kbeg = kz * kchunk;
  int kend = min(K, kbeg + kchunk);
  if (tri_b) kend = min(kend, n0 + TC_NC);
  const int nst = kend > kbeg ? (kend - kbeg + TC_KC - 1) / TC_KC : 0;
  const int nwin = (nst + TC_WIN - 1) / TC_WIN;
  float* sums = reinterpret_cast<float*>(smem + TC_NS * STAGE_BYTES);   // [256 columns][128 rows]

  if (tid == 0) {
    for (int s = 0; s < TC_NS; ++s) {
      mbar_init(&bar_full[s], TC_PROD);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_acc_full[b], 1);
      mbar_init(&bar_acc_empty[b], TC_PROD);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
  }
  if (warp == TC_PROD / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_base)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp < TC_PROD / 32) {
    const int q = warp & 3, h = warp >> 2;
    const int r = 32 * q + lane;                 // tile row of op(A), tile column of op(B)
    const int m = m0 + r, n = n0 + r;
    const uint32_t tlane = (uint32_t)(32 * q) << 16;
    float* my_sums = sums + (TC_NC * h) * TC_M + r;   // column j of this thread: my_sums[j * TC_M]
    float2 pa[TC_PF][4], pb[TC_PF][4];           // stages st .. st + TC_PF - 1 in flight (buffer st % TC_PF)
    auto load = [&](int st, float2 (&a)[4], float2 (&b)[4]) {
      const int kb = kbeg + st * TC_KC + 4 * h;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int kk = kb + j;
        float2 va = make_float2(0.f, 0.f), vb = make_float2(0.f, 0.f);
        if (st < nst && m < M && kk < kend) {
          if (OPA == OP_N) va = __ldg(A + m + (long)kk * lda);
          else { va = __ldg(A + kk + (long)m * lda); va.y = -va.y; }
        }
        if (st < nst && n < N && kk < kend) {
          if (OPB == OP_N) vb = __ldg(B + kk + (long)n * ldb);
          else { vb = __ldg(B + n + (long)kk * ldb); vb.y = -vb.y; }
        }
        a[j] = va;
        b[j] = vb;
      }
    };
    // store stage st (from a, b) into its ring slot
    auto produce = [&](int st, const float2 (&a)[4], const float2 (&b)[4]) {
      const int s = st % TC_NS;
      const uint32_t ph = (uint32_t)(st / TC_NS) & 1u;
      if (ok) ok = mbar_wait(&bar_empty[s], ph ^ 1u, err);
      unsigned char* Ahi = smem + s * STAGE_BYTES;
      unsigned char* Alo = Ahi + A_BYTES;
      unsigned char* Bhi = Alo + A_BYTES;
      unsigned char* Blo = Bhi + B_BYTES;
      if (ok) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {   // core-matrix columns kc = 2h + c: complex k 4h + 2c, +1
          const int kc = 2 * h + c;
          const float2 a0 = a[2 * c], a1 = a[2 * c + 1], b0 = b[2 * c], b1 = b[2 * c + 1];
          st_split(Ahi, Alo, core_off(r, kc), a0.x, a0.y, a1.x, a1.y);
          st_split(Bhi, Blo, core_off(r, kc), b0.x, -b0.y, b1.x, -b1.y);          // -> C_r
          st_split(Bhi, Blo, core_off(r + TC_NC, kc), b0.y, b0.x, b1.y, b1.x);    // -> C_i
        }
      }
      asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
      mbar_arrive(&bar_full[s]);
    };
    // slice pos (16 columns) of window dw's accumulator into the sums
    auto drain = [&](int dw, int pos) {
      const int b = dw & 1;
      if (pos == 0 && ok) ok = mbar_wait(&bar_acc_full[b], (uint32_t)(dw >> 1) & 1u, err);
      tc_fence_after();
      uint32_t v[16];
      // tcgen05.ld is warp-collective: the whole warp reads the accumulator, or none of it
      if (__all_sync(0xffffffffu, ok)) {
        tmem_ld16(tmem + tlane + (uint32_t)(b * 2 * TC_NC + TC_NC * h + 16 * pos), v);
        tmem_ld_wait();
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0u;
      }
      float* sp = my_sums + (16 * pos) * TC_M;
#pragma unroll
      for (int i = 0; i < 16; ++i) sp[i * TC_M] = dw == 0 ? __uint_as_float(v[i]) : sp[i * TC_M] + __uint_as_float(v[i]);
      if (pos == TC_WIN - 1) {
        tc_fence_before();
        mbar_arrive(&bar_acc_empty[b]);
      }
    };
#pragma unroll
    for (int e = 0; e < TC_PF; ++e) load(e, pa[e], pb[e]);
    // stages in groups of TC_PF (stage st in buffer st % TC_PF); after producing stage
    // st = TC_WIN win + pos, drain slice pos of window win - 1
#pragma unroll 1
    for (int st0 = 0; st0 < TC_WIN * (nwin + 1); st0 += TC_PF) {
#pragma unroll
      for (int e = 0; e < TC_PF; ++e) {
        const int st = st0 + e;
        if (st < nst) {
          float2 a[4], b[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) { a[j] = pa[e][j]; b[j] = pb[e][j]; }
          load(st + TC_PF, pa[e], pb[e]);   // TC_PF stages ahead, in flight while this one is stored
          produce(st, a, b);
        }
        const int win = st / TC_WIN, pos = st % TC_WIN;
        if (win >= 1 && win - 1 < nwin) drain(win - 1, pos);
      }
    }
    // ---- output ----------------------------------------------------------------------
    asm volatile("bar.sync 1, %0;\n" ::"r"(TC_PROD) : "memory");   // both halves of every row drained
    if (m < M) {
      for (int j0 = (TC_NC / 2) * h; j0 < (TC_NC / 2) * (h + 1); ++j0) {
        const int j = n0 + j0;
        if (j >= N) break;
        double2 v = make_double2(0.0, 0.0);
        if (nst > 0) v = make_double2((double)sums[j0 * TC_M + r], (double)sums[(TC_NC + j0) * TC_M + r]);
        if (ksplit > 1) {
          part[((long)kz * N + j) * (long)M + m] = v;
        } else {
          double2* c = Cm + m + (long)j * ldc;
          double2 o2 = make_double2(alpha.x * v.x - alpha.y * v.y, alpha.x * v.y + alpha.y * v.x);
          if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 o = *c;
            o2.x += beta.x * o.x - beta.y * o.y;
            o2.y += beta.x * o.y + beta.y * o.x;
          }
          *c = o2;
        }
      }
    }
  } else if (lane == 0) {
    // ---- MMA issue (one thread of warp 8) --------------------------------------------
    const uint32_t sbase = smem_u32(smem);
    for (int st = 0; st < nst; ++st) {
      const int s = st % TC_NS;
      const uint32_t ph = (uint32_t)(st / TC_NS) & 1u;
      const int win = st / TC_WIN, pos = st % TC_WIN, b = win & 1;
      if (pos == 0 && win >= 2 && ok) ok = mbar_wait(&bar_acc_empty[b], (uint32_t)((win - 2) >> 1) & 1u, err);
      if (ok) ok = mbar_wait(&bar_full[s], ph, err);
      tc_fence_after();
      if (ok) {
        const uint32_t d = tmem + (uint32_t)(b * 2 * TC_NC);
        const uint32_t ahi = sbase + s * STAGE_BYTES, alo = ahi + A_BYTES, bhi = alo + A_BYTES, blo = bhi + B_BYTES;
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {   // K = 8 real values = two core matrices along K
          const uint32_t o = qq * 256;
          tc_mma(d, smem_desc(ahi + o), smem_desc(bhi + o), (pos > 0 || qq > 0) ? 1u : 0u);
          tc_mma(d, smem_desc(ahi + o), smem_desc(blo + o), 1u);
          tc_mma(d, smem_desc(alo + o), smem_desc(bhi + o), 1u);
        }
      }
      tc_commit(&bar_empty[s]);                                            // stage s is free once read
      if (pos == TC_WIN - 1 || st == nst - 1) tc_commit(&bar_acc_full[b]);   // window complete
    }
  }
  if (warp == TC_PROD / 32) __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == TC_PROD / 32) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

template <int OPA, int OPB>
static cudaError_t launch_tc(int M, int N, int K, int kchunk, int ksplit, int tri_b, double2 alpha, const float2* A,
                             long lda, const float2* B, long ldb, double2 beta, double2* C, long ldc, double2* ws,
                             int* err, cudaStream_t s) {
  static std::atomic<unsigned long long> attr_done{0};
  if (const unsigned long long bit = device_bit_todo(attr_done)) {
    cudaError_t e = cudaFuncSetAttribute(k_cgemm_tf32x3<OPA, OPB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit, std::memory_order_release);
  }
  dim3 grid((unsigned)((M + TC_M - 1) / TC_M), (unsigned)((N + TC_NC - 1) / TC_NC), (unsigned)ksplit);
  k_cgemm_tf32x3<OPA, OPB><<<grid, TC_THREADS, TC_SMEM, s>>>(M, N, K, kchunk, ksplit, tri_b, alpha, A, lda, B, ldb,
                                                             beta, C, ldc, ws, err);
  launched();
  return cudaGetLastError();
}

cudaError_t gemm_tc(int opA, int opB, int M, int N, int K, double2 alpha, const float2* A, long lda, const float2* B,
                    long ldb, double2 beta, double2* C, long ldc, double2* ws, size_t ws_elems, int* d_err,
                    cudaStream_t s, int structure) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (structure == GEMM_HERM || d_err == nullptr) return cudaErrorInvalidValue;
  const int tri_b = structure == GEMM_TRI_B ? 1 : 0;
  const long tiles = (long)((M + TC_M - 1) / TC_M) * ((N + TC_NC - 1) / TC_NC);
  // split the reduction over the basis so that the tiles fill the SMs (one CTA each) about once
  static std::atomic<int> sm_count[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  int sms = sm_count[dev & 63].load(std::memory_order_relaxed);
  if (sms == 0) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    sms = std::max(1, sms);
    sm_count[dev & 63].store(sms, std::memory_order_relaxed);
  }
  const long slots = sms;
  int ksplit = 1;
  if (K > 1024 && tiles < slots && ws != nullptr) {
    ksplit = (int)std::max<long>(1, std::min<long>(slots / tiles, (K + 511) / 512));
    while (ksplit > 1 && (size_t)ksplit * M * N > ws_elems) --ksplit;
  }
  int kchunk = (K + ksplit - 1) / ksplit;
  kchunk = ((kchunk + TC_KC - 1) / TC_KC) * TC_KC;
  ksplit = std::max(1, (K + kchunk - 1) / kchunk);
  if (K <= 0) { ksplit = 1; kchunk = TC_KC; }
  cudaError_t e;
  if (opA == OP_N && opB == OP_N) e = launch_tc<OP_N, OP_N>(M, N, K, kchunk, ksplit, tri_b, alpha, A, lda, B, ldb, beta, C, ldc, ws, d_err, s);
  else if (opA == OP_N) e = launch_tc<OP_N, OP_H>(M, N, K, kchunk, ksplit, tri_b, alpha, A, lda, B, ldb, beta, C, ldc, ws, d_err, s);
  else if (opB == OP_N) e = launch_tc<OP_H, OP_N>(M, N, K, kchunk, ksplit, tri_b, alpha, A, lda, B, ldb, beta, C, ldc, ws, d_err, s);
  else e = launch_tc<OP_H, OP_H>(M, N, K, kchunk, ksplit, tri_b, alpha, A, lda, B, ldb, beta, C, ldc, ws, d_err, s);
  if (e != cudaSuccess || ksplit == 1) return e;
  return splitk_reduce(M, N, ksplit, alpha, ws, beta, C, ldc, s);
}

}  // namespace pt
