// Generic batched 3D transforms between the planewave basis and the real-space
// grid (orbitals, density, local potential of Eq. 2; Sec. 3.2 and 3.4).
// A 3D FFT is three passes over global memory, one per axis:
//   rows   (axis 2, contiguous lines): a block owns whole rows,
//   cols   (axis 1 or 0): a block owns an L x C tile of C consecutive i2
//          columns so that every global access is a run of C elements.
// The axis-0 pass can fuse "inverse, multiply by a real field, forward"
// (local potential times orbital) or "forward, multiply by a reciprocal-space
// factor, inverse" (Hartree solve), so those operations cost no extra pass.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "common.cuh"
#include "fft.cuh"
#include "internal.h"

namespace pt {

int twiddle_offset(int L) {
  int off = 0;
  for (int i = 0; i < kNumLengths; ++i) {
    if (kLengths[i] == L) return off;
    off += kLengths[i];
  }
  return -1;
}

void twiddle_host(double2* out) {
  int off = 0;
  for (int i = 0; i < kNumLengths; ++i) {
    const int L = kLengths[i];
    for (int t = 0; t < L; ++t) {
      const double a = 2.0 * M_PI * (double)t / (double)L;
      out[off + t] = make_double2(std::cos(a), -std::sin(a));
    }
    off += L;
  }
}

template <> const void* DevTwiddles::base<double>() const { return d64; }
template <> const void* DevTwiddles::base<float>() const { return d32; }

template <typename T>
static const cplx<T>* tw_for(const DevTwiddles& tw, int L) {
  return reinterpret_cast<const cplx<T>*>(tw.base<T>()) + twiddle_offset(L);
}

static int round_threads(int t) {
  t = ((t + 31) / 32) * 32;
  return std::max(64, std::min(1024, t));
}

// ---------------------------------------------------------------------------
template <typename T, bool INV>
__global__ void k_rows(const cplx<T>* __restrict__ in, cplx<T>* __restrict__ out, long nrows, int L, int rpc,
                       const cplx<T>* __restrict__ tw_g, T scale, const T* __restrict__ mul, long rows_per_vol) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int t = tid; t < L; t += nthr) tw[t] = tw_g[t];
  const long r0 = (long)blockIdx.x * rpc;
  const int nr = (int)min((long)rpc, nrows - r0);
  const int cnt = nr * L;
  const C* src = in + r0 * L;
  for (int e = tid; e < cnt; e += nthr) {
    C v = src[e];
    if (mul != nullptr) {
      const long row = r0 + e / L;
      v = cscale(v, mul[(row % rows_per_vol) * L + (e % L)]);
    }
    buf[e] = v;
  }
  __syncthreads();
  fft_lines<T, INV, true>(buf, L, nr, L, 1, tw, tid, nthr);
  C* dst = out + r0 * L;
  for (int e = tid; e < cnt; e += nthr) dst[e] = cscale(buf[e], scale);
}

template <typename T, bool INV, int MODE>
__global__ void k_cols(cplx<T>* __restrict__ data, int n0, int n1, int n2, int axis, int chunk,
                       const cplx<T>* __restrict__ tw_g, T scale, const T* __restrict__ mul) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = axis == 0 ? n0 : n1;
  const long S = axis == 0 ? (long)n1 * n2 : (long)n2;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  for (int t = tid; t < L; t += nthr) tw[t] = tw_g[t];
  const int i2s = blockIdx.x * chunk;
  const int nc = min(chunk, n2 - i2s);
  const int u = blockIdx.y;
  const long N = (long)n0 * n1 * n2;
  C* base = data + (long)blockIdx.z * N + (axis == 1 ? (long)u * n1 * n2 : (long)u * n2) + i2s;
  const int cnt = L * nc;
  for (int idx = tid; idx < cnt; idx += nthr) {
    const int e = idx / nc, c = idx - e * nc;
    buf[e * chunk + c] = base[e * S + c];
  }
  __syncthreads();
  fft_lines<T, INV, false>(buf, L, nc, 1, chunk, tw, tid, nthr);
  if (MODE != 0) {
    for (int idx = tid; idx < cnt; idx += nthr) {
      const int e = idx / nc, c = idx - e * nc;
      // axis 0 only: point (e, u, i2s + c)
      const long flat = ((long)e * n1 + u) * n2 + i2s + c;
      buf[e * chunk + c] = cscale(buf[e * chunk + c], mul[flat]);
    }
    __syncthreads();
    fft_lines<T, !INV, false>(buf, L, nc, 1, chunk, tw, tid, nthr);
  }
  for (int idx = tid; idx < cnt; idx += nthr) {
    const int e = idx / nc, c = idx - e * nc;
    base[e * S + c] = cscale(buf[e * chunk + c], scale);
  }
}

template <typename T>
cudaError_t fft_rows(const void* in, void* out, long nvol, Grid3 g, int inverse, double scale, const T* mul_real,
                     const DevTwiddles& tw, cudaStream_t s) {
  using C = cplx<T>;
  const int L = g.n2;
  if (!fft_length_supported(L)) return cudaErrorInvalidValue;
  const long nrows = nvol * g.n0 * g.n1;
  // rows per block: aim at ~4-8 KB of data per block
  int rpc = std::max(1, (int)(8192 / (L * (int)sizeof(C))));
  rpc = std::min<long>(rpc, nrows);
  const bool fp64 = sizeof(T) == 8;
  const int nthr = round_threads(fft_threads_needed(L, rpc, fp64));
  const size_t smem = (size_t)(L + rpc * L) * sizeof(C);
  const long nblk = (nrows + rpc - 1) / rpc;
  const T sc = (T)scale;
  const long rpv = (long)g.n0 * g.n1;
  if (inverse)
    k_rows<T, true><<<(unsigned)nblk, nthr, smem, s>>>((const C*)in, (C*)out, nrows, L, rpc, tw_for<T>(tw, L), sc,
                                                      mul_real, rpv);
  else
    k_rows<T, false><<<(unsigned)nblk, nthr, smem, s>>>((const C*)in, (C*)out, nrows, L, rpc, tw_for<T>(tw, L), sc,
                                                       mul_real, rpv);
  launched();
  return cudaGetLastError();
}

template <typename T>
cudaError_t fft_cols(void* data, long nvol, Grid3 g, int axis, int inverse, int mode, double scale, const T* mul_real,
                     const DevTwiddles& tw, cudaStream_t s) {
  using C = cplx<T>;
  const int L = axis == 0 ? g.n0 : g.n1;
  if (!fft_length_supported(L)) return cudaErrorInvalidValue;
  if (mode != 0 && (axis != 0 || mul_real == nullptr)) return cudaErrorInvalidValue;
  int chunk = sizeof(T) == 4 ? 16 : 8;
  chunk = std::min(chunk, g.n2);
  const bool fp64 = sizeof(T) == 8;
  const int nthr = round_threads(fft_threads_needed(L, chunk, fp64));
  const size_t smem = (size_t)(L + L * chunk) * sizeof(C);
  dim3 grid((g.n2 + chunk - 1) / chunk, axis == 0 ? g.n1 : g.n0, (unsigned)nvol);
  const T sc = (T)scale;
  const C* twp = tw_for<T>(tw, L);
#define PT_COLS(INV, MODE) k_cols<T, INV, MODE><<<grid, nthr, smem, s>>>((C*)data, g.n0, g.n1, g.n2, axis, chunk, twp, sc, mul_real)
  if (mode == 0) {
    if (inverse) PT_COLS(true, 0); else PT_COLS(false, 0);
  } else if (mode == 1) {
    PT_COLS(true, 1);   // inverse, multiply, forward
  } else {
    PT_COLS(false, 2);  // forward, multiply, inverse
  }
#undef PT_COLS
  launched();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void k_scatter(const double2* __restrict__ in, long in_ld, cplx<T>* __restrict__ out, long N,
                          const int* __restrict__ basis, int npw, double scale) {
  const long v = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npw; k += gridDim.x * blockDim.x) {
    const double2 c = in[v * in_ld + k];
    out[v * N + basis[k]] = cvt<cplx<T>>(make_double2(c.x * scale, c.y * scale));
  }
}

template <typename T>
__global__ void k_gather(const cplx<T>* __restrict__ in, double2* __restrict__ out, long out_ld, long N,
                         const int* __restrict__ basis, int npw, double scale, const double* __restrict__ kin,
                         const double2* __restrict__ x, long x_ld, int accumulate) {
  const long v = blockIdx.y;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npw; k += gridDim.x * blockDim.x) {
    const double2 f = to_d(in[v * N + basis[k]]);
    double2 r = make_double2(f.x * scale, f.y * scale);
    if (kin != nullptr) {
      const double2 c = x[v * x_ld + k];
      r.x += kin[k] * c.x;
      r.y += kin[k] * c.y;
    }
    double2* o = out + v * out_ld + k;
    if (accumulate) { r.x += o->x; r.y += o->y; }
    *o = r;
  }
}

template <typename T>
cudaError_t scatter_basis(const double2* in, long in_ld, void* out, long nvol, Grid3 g, const int* basis, int npw,
                          double scale, cudaStream_t s) {
  using C = cplx<T>;
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(C) * g.N() * nvol, s);
  if (e != cudaSuccess) return e;
  dim3 grid((npw + 255) / 256, (unsigned)nvol);
  k_scatter<T><<<grid, 256, 0, s>>>(in, in_ld, (C*)out, g.N(), basis, npw, scale); launched();
  return cudaGetLastError();
}

template <typename T>
cudaError_t gather_basis(const void* in, double2* out, long out_ld, long nvol, Grid3 g, const int* basis, int npw,
                         double scale, const double* kin, const double2* x, long x_ld, int accumulate, cudaStream_t s) {
  using C = cplx<T>;
  dim3 grid((npw + 255) / 256, (unsigned)nvol);
  k_gather<T><<<grid, 256, 0, s>>>((const C*)in, out, out_ld, g.N(), basis, npw, scale, kin, x, x_ld, accumulate); launched();
  return cudaGetLastError();
}

__global__ void k_c128_to_c64(const double2* __restrict__ in, float2* __restrict__ out, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    out[i] = make_float2((float)in[i].x, (float)in[i].y);
}

cudaError_t convert_c128_to_c64(const double2* in, float2* out, long n, cudaStream_t s) {
  long blocks = std::min<long>((n + 255) / 256, 152L * 32);
  k_c128_to_c64<<<(unsigned)std::max<long>(blocks, 1), 256, 0, s>>>(in, out, n); launched();
  return cudaGetLastError();
}

// explicit instantiations
template cudaError_t fft_rows<float>(const void*, void*, long, Grid3, int, double, const float*, const DevTwiddles&, cudaStream_t);
template cudaError_t fft_rows<double>(const void*, void*, long, Grid3, int, double, const double*, const DevTwiddles&, cudaStream_t);
template cudaError_t fft_cols<float>(void*, long, Grid3, int, int, int, double, const float*, const DevTwiddles&, cudaStream_t);
template cudaError_t fft_cols<double>(void*, long, Grid3, int, int, int, double, const double*, const DevTwiddles&, cudaStream_t);
template cudaError_t scatter_basis<float>(const double2*, long, void*, long, Grid3, const int*, int, double, cudaStream_t);
template cudaError_t scatter_basis<double>(const double2*, long, void*, long, Grid3, const int*, int, double, cudaStream_t);
template cudaError_t gather_basis<float>(const void*, double2*, long, long, Grid3, const int*, int, double, const double*, const double2*, long, int, cudaStream_t);
template cudaError_t gather_basis<double>(const void*, double2*, long, long, Grid3, const int*, int, double, const double*, const double2*, long, int, cudaStream_t);

static std::atomic<unsigned long long> g_launches{0};
void launched(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }
unsigned long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

std::string cuda_msg(cudaError_t e) { return std::string(cudaGetErrorName(e)) + ": " + cudaGetErrorString(e); }

}  // namespace pt
