// Dense complex linear algebra of the PT-CN step and ACE:
//   overlap / projection products S = Psi^H (H Psi), Psi S (Alg. 3),
//   M = Psi^H W, xi^H X, xi Y (ACE), Psi^H Psi and Psi L^{-H} (Sec. 3.4),
//   Cholesky factorisations (orthonormalisation, -M of ACE) and L^{-1}.
// GEMM: 64 x 64 output tiles, 256 threads with 4 x 4 complex micro-tiles,
// operands staged in shared memory in the compute precision (double-buffered,
// next slice prefetched into registers); the long reduction over the basis is
// split over blocks (split-K) into a workspace and summed in a fixed order, so
// results are deterministic. Hermitian products (Psi^H Psi) compute half the
// tiles; products with a triangular factor stop the reduction at the diagonal.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace pt {

constexpr int GBM = 64, GBN = 64;
template <typename C> __device__ __forceinline__ C to_compute(double2 v) { return cvt<C>(v); }
template <typename C> __device__ __forceinline__ C to_compute(float2 v);
template <> __device__ __forceinline__ float2 to_compute<float2>(float2 v) { return v; }
template <typename Tc> struct GemmK { static constexpr int V = 16; };
template <> struct GemmK<double> { static constexpr int V = 8; };

// Output structure the caller promises (skipped work is exactly zero or implied):
//   GEMM_HERM   C = A^H A is Hermitian: only tiles on or below the diagonal are
//               computed; the upper triangle is written as the conjugate mirror.
//   GEMM_TRI_B  op(B) is upper triangular (op(B)[k][j] = 0 for k > j): the
//               reduction for output columns [n0, n0 + 64) stops at n0 + 64.
// One block computes a 64 x 64 tile over its K chunk with 256 threads (4 x 4
// complex register tiles). The next K slice is fetched into registers while the
// current one is multiplied from the other of two shared-memory buffers, so
// there is one barrier per K slice. TI is the storage type of A and B
// (complex128, or complex64 mirrors for FP32 products: converting FP64 inputs
// inside the product loop would run every re-read element through the FP64
// pipe, which on this GPU is as costly as the products themselves).
template <typename Tc, typename TI>
__global__ void __launch_bounds__(256) k_gemm(int opA, int opB, int M, int N, int K, int kchunk, int ksplit, int structure,
                                              double2 alpha, const TI* __restrict__ A, long lda, long sA,
                                              const TI* __restrict__ B, long ldb, long sB, double2 beta,
                                              double2* __restrict__ Cm, long ldc, long sC,
                                              double2* __restrict__ part) {
  using C = cplx<Tc>;
  constexpr int GK = GemmK<Tc>::V;
  constexpr int PA = GBM * GK / 256;   // A elements per thread per slice
  constexpr int PB = GBN * GK / 256;
  __shared__ C As[2][GK][GBM + 1];
  __shared__ C Bs[2][GK][GBN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * GBM, n0 = blockIdx.y * GBN;
  if (structure == GEMM_HERM && m0 + GBM <= n0) return;   // strictly above the diagonal
  const int bz = blockIdx.z / ksplit, kz = blockIdx.z % ksplit;
  const TI* Ab = A + (long)bz * sA;
  const TI* Bb = B + (long)bz * sB;
  const int kbeg = kz * kchunk;
  int kend = min(K, kbeg + kchunk);
  if (structure == GEMM_TRI_B) kend = min(kend, n0 + GBN);
  C acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = mk((Tc)0, (Tc)0);
  C ra[PA], rb[PB];   // next slice, already in the compute precision
  auto fetch = [&](int k0) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int idx = tid + q * 256;
      int i, k;
      if (opA == OP_N) { i = idx % GBM; k = idx / GBM; }
      else { k = idx % GK; i = idx / GK; }
      const int gi = m0 + i, gk = k0 + k;
      TI v{};
      if (gi < M && gk < kend) {
        if (opA == OP_N) v = Ab[gi + (long)gk * lda];
        else { v = Ab[gk + (long)gi * lda]; v.y = -v.y; }
      }
      ra[q] = to_compute<C>(v);
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int idx = tid + q * 256;
      int j, k;
      if (opB == OP_N) { k = idx % GK; j = idx / GK; }
      else { j = idx % GBN; k = idx / GBN; }
      const int gj = n0 + j, gk = k0 + k;
      TI v{};
      if (gj < N && gk < kend) {
        if (opB == OP_N) v = Bb[gk + (long)gj * ldb];
        else { v = Bb[gj + (long)gk * ldb]; v.y = -v.y; }
      }
      rb[q] = to_compute<C>(v);
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < PA; ++q) {
      const int idx = tid + q * 256;
      int i, k;
      if (opA == OP_N) { i = idx % GBM; k = idx / GBM; }
      else { k = idx % GK; i = idx / GK; }
      As[buf][k][i] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < PB; ++q) {
      const int idx = tid + q * 256;
      int j, k;
      if (opB == OP_N) { k = idx % GK; j = idx / GK; }
      else { j = idx % GBN; k = idx / GBN; }
      Bs[buf][k][j] = rb[q];
    }
  };
  int buf = 0;
  if (kbeg < kend) {
    fetch(kbeg);
    stash(0);
  }
  __syncthreads();
  for (int k0 = kbeg; k0 < kend; k0 += GK) {
    const bool more = k0 + GK < kend;
    if (more) fetch(k0 + GK);   // in flight during the products below
#pragma unroll
    for (int k = 0; k < GK; ++k) {
      C av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[buf][k][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[buf][k][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          acc[a][b].x = fma(av[a].x, bv[b].x, acc[a][b].x);
          acc[a][b].x = fma(-av[a].y, bv[b].y, acc[a][b].x);
          acc[a][b].y = fma(av[a].x, bv[b].y, acc[a][b].y);
          acc[a][b].y = fma(av[a].y, bv[b].x, acc[a][b].y);
        }
    }
    if (more) stash(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int i = m0 + tx + 16 * a, j = n0 + ty + 16 * b;
      if (i < M && j < N) {
        if (structure == GEMM_HERM && i < j) continue;   // mirrored from (j, i)
        const double2 v = to_d(acc[a][b]);
        if (ksplit > 1) {
          part[(((long)kz * gridDim.z / ksplit + bz) * N + j) * (long)M + i] = v;
        } else {
          double2 r = make_double2(alpha.x * v.x - alpha.y * v.y, alpha.x * v.y + alpha.y * v.x);
          double2* c = Cm + (long)bz * sC + i + (long)j * ldc;
          if (beta.x != 0.0 || beta.y != 0.0) {
            const double2 o = *c;
            r.x += beta.x * o.x - beta.y * o.y;
            r.y += beta.x * o.y + beta.y * o.x;
          }
          *c = r;
          if (structure == GEMM_HERM && i != j) {
            double2* cm = Cm + (long)bz * sC + j + (long)i * ldc;
            double2 rm = make_double2(alpha.x * v.x + alpha.y * v.y, alpha.y * v.x - alpha.x * v.y);  // alpha conj(v)
            if (beta.x != 0.0 || beta.y != 0.0) {
              const double2 o = *cm;
              rm.x += beta.x * o.x - beta.y * o.y;
              rm.y += beta.x * o.y + beta.y * o.x;
            }
            *cm = rm;
          }
        }
      }
    }
}

// Sums the split-K partials in a fixed order. For GEMM_HERM the partials exist
// on and below the diagonal; an entry above it is the conjugate of its mirror.
__global__ void k_splitk_reduce(int M, int N, int batch, int ksplit, int structure, double2 alpha,
                                const double2* __restrict__ part, double2 beta, double2* __restrict__ Cm, long ldc,
                                long sC) {
  const long total = (long)batch * M * N;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t % M);
    const long rest = t / M;
    const int j = (int)(rest % N);
    const int bz = (int)(rest / N);
    const bool mirror = structure == GEMM_HERM && i < j;
    const int pi = mirror ? j : i, pj = mirror ? i : j;
    double2 s = make_double2(0.0, 0.0);
    for (int kz = 0; kz < ksplit; ++kz) {
      const double2 v = part[(((long)kz * batch + bz) * N + pj) * (long)M + pi];
      s.x += v.x;
      s.y += v.y;
    }
    if (mirror) s.y = -s.y;
    double2* c = Cm + (long)bz * sC + i + (long)j * ldc;
    double2 r = make_double2(alpha.x * s.x - alpha.y * s.y, alpha.x * s.y + alpha.y * s.x);
    if (beta.x != 0.0 || beta.y != 0.0) {
      const double2 o = *c;
      r.x += beta.x * o.x - beta.y * o.y;
      r.y += beta.x * o.y + beta.y * o.x;
    }
    *c = r;
  }
}

template <typename Tc, typename TI>
static cudaError_t gemm_impl(int opA, int opB, int M, int N, int K, double2 alpha, const TI* A, long lda, long strideA,
                             const TI* B, long ldb, long strideB, double2 beta, double2* C, long ldc, long strideC,
                             int batch, double2* ws, size_t ws_elems, cudaStream_t s, int structure) {
  constexpr int GK = GemmK<Tc>::V;
  if (M <= 0 || N <= 0 || batch <= 0) return cudaSuccess;
  if (structure == GEMM_HERM && M != N) return cudaErrorInvalidValue;
  const int tm = (M + GBM - 1) / GBM, tn = (N + GBN - 1) / GBN;
  const long tiles = structure == GEMM_HERM ? (long)tm * (tm + 1) / 2 * batch : (long)tm * tn * batch;
  // split the reduction so that tiles x ksplit fills the resident block slots once
  // (a second, mostly empty wave would cost as much as the first)
  static std::atomic<int> slot_count[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  int slots = slot_count[dev & 63].load(std::memory_order_relaxed);
  if (slots == 0) {
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gemm<Tc, TI>, 256, 0);
    slots = std::max(1, sms * std::max(1, per_sm));
    slot_count[dev & 63].store(slots, std::memory_order_relaxed);
  }
  int ksplit = 1;
  if (K > 1024 && tiles < slots) {
    ksplit = (int)std::max<long>(1, std::min<long>(slots / tiles, (K + 511) / 512));
    while (ksplit > 1 && (size_t)ksplit * batch * M * N > ws_elems) --ksplit;
  }
  int kchunk = (K + ksplit - 1) / ksplit;
  kchunk = ((kchunk + GK - 1) / GK) * GK;
  ksplit = std::max(1, (K + kchunk - 1) / kchunk);
  if (K == 0) { ksplit = 1; kchunk = GK; }
  dim3 grid(tm, tn, (unsigned)(batch * ksplit));
  k_gemm<Tc, TI><<<grid, 256, 0, s>>>(opA, opB, M, N, K, kchunk, ksplit, structure, alpha, A, lda, strideA, B, ldb,
                                  strideB, beta, C, ldc, strideC, ws); launched();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || ksplit == 1) return e;
  const long total = (long)batch * M * N;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_splitk_reduce<<<blocks, 256, 0, s>>>(M, N, batch, ksplit, structure, alpha, ws, beta, C, ldc, strideC); launched();
  return cudaGetLastError();
}

template <typename Tc>
cudaError_t gemm(int opA, int opB, int M, int N, int K, double2 alpha, const double2* A, long lda, long strideA,
                 const double2* B, long ldb, long strideB, double2 beta, double2* C, long ldc, long strideC, int batch,
                 double2* ws, size_t ws_elems, cudaStream_t s, int structure) {
  return gemm_impl<Tc, double2>(opA, opB, M, N, K, alpha, A, lda, strideA, B, ldb, strideB, beta, C, ldc, strideC,
                                batch, ws, ws_elems, s, structure);
}

template cudaError_t gemm<double>(int, int, int, int, int, double2, const double2*, long, long, const double2*, long,
                                  long, double2, double2*, long, long, int, double2*, size_t, cudaStream_t, int);

cudaError_t splitk_reduce(int M, int N, int ksplit, double2 alpha, const double2* part, double2 beta, double2* C,
                          long ldc, cudaStream_t s) {
  const long total = (long)M * N;
  const int blocks = (int)std::min<long>((total + 255) / 256, 152L * 16);
  k_splitk_reduce<<<blocks, 256, 0, s>>>(M, N, 1, ksplit, GEMM_GENERAL, alpha, part, beta, C, ldc, 0); launched();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cholesky, right-looking, one column per pair of launches (pivot, update).
__global__ void k_chol_pivot(double2* A, int n, int j, int* status) {
  __shared__ double djj;
  if (*status != 0) return;
  if (threadIdx.x == 0) {
    const double d = A[j + (long)j * n].x;
    if (!(d > 0.0)) { *status = 1; djj = 0.0; }
    else { djj = sqrt(d); A[j + (long)j * n] = make_double2(djj, 0.0); }
  }
  __syncthreads();
  if (djj == 0.0) return;
  const double inv = 1.0 / djj;
  for (int i = j + 1 + threadIdx.x; i < n; i += blockDim.x) {
    double2 v = A[i + (long)j * n];
    A[i + (long)j * n] = make_double2(v.x * inv, v.y * inv);
  }
}

// A[i][k] -= A[i][j] conj(A[k][j]) for j < k <= i
__global__ void k_chol_update(double2* A, int n, int j, const int* status) {
  if (*status != 0) return;
  const int k = j + 1 + blockIdx.x;
  if (k >= n) return;
  const double2 akj = A[k + (long)j * n];
  for (int i = k + threadIdx.x; i < n; i += blockDim.x) {
    const double2 aij = A[i + (long)j * n];
    double2* t = A + i + (long)k * n;
    double2 v = *t;
    v.x -= aij.x * akj.x + aij.y * akj.y;
    v.y -= aij.y * akj.x - aij.x * akj.y;
    *t = v;
  }
}

__global__ void k_zero_upper(double2* A, int n) {
  const long total = (long)n * n;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
    const int i = (int)(t % n), k = (int)(t / n);
    if (i < k) A[t] = make_double2(0.0, 0.0);
  }
}

cudaError_t cholesky(double2* A, int n, int* d_status, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  for (int j = 0; j < n; ++j) {
    k_chol_pivot<<<1, 256, 0, s>>>(A, n, j, d_status); launched();
    if (j + 1 < n) { k_chol_update<<<n - j - 1, 128, 0, s>>>(A, n, j, d_status); launched(); }
  }
  k_zero_upper<<<std::max(1, std::min(1024, (n * n + 255) / 256)), 256, 0, s>>>(A, n); launched();
  return cudaGetLastError();
}

// Column c of L^{-1}: solve L x = e_c by forward substitution (one block per column).
__global__ void k_tri_inverse(const double2* __restrict__ L, double2* __restrict__ Li, int n) {
  extern __shared__ double2 b[];
  const int c = blockIdx.x;
  for (int i = threadIdx.x; i < n; i += blockDim.x) b[i] = make_double2(i == c ? 1.0 : 0.0, 0.0);
  __syncthreads();
  for (int i = c; i < n; ++i) {
    const double2 lii = L[i + (long)i * n];
    // x_i = b_i / L_ii  (L_ii real positive for a Cholesky factor, kept general)
    const double den = lii.x * lii.x + lii.y * lii.y;
    const double2 bi = b[i];
    const double2 xi = make_double2((bi.x * lii.x + bi.y * lii.y) / den, (bi.y * lii.x - bi.x * lii.y) / den);
    __syncthreads();
    for (int k = i + 1 + threadIdx.x; k < n; k += blockDim.x) {
      const double2 lki = L[k + (long)i * n];
      double2 v = b[k];
      v.x -= lki.x * xi.x - lki.y * xi.y;
      v.y -= lki.x * xi.y + lki.y * xi.x;
      b[k] = v;
    }
    if (threadIdx.x == 0) b[i] = xi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Li[i + (long)c * n] = i < c ? make_double2(0.0, 0.0) : b[i];
}

cudaError_t tri_inverse(const double2* L, double2* Linv, int n, cudaStream_t s) {
  k_tri_inverse<<<n, 128, sizeof(double2) * n, s>>>(L, Linv, n); launched();
  return cudaGetLastError();
}

}  // namespace pt
