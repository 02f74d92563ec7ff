// Compile-time-sized line FFTs for the pair pipeline (lengths 32, 64, 96).
//
// Each length L = R1 * R2 is transformed by two Stockham stages (radix R1,
// then radix R2 with sub-transform length R1), so one line costs two
// shared-memory round trips. The inverse uses the reversed plan (R2, R1):
// the forward stage 2 butterfly j reads and writes elements j + r R1, which
// are exactly the inputs of inverse stage 1 butterfly j, so "forward stage 2,
// multiply by the kernel, inverse stage 1" runs in registers (ct_fused).
// Shared-memory line buffers use a padded index i + i / 8, which spreads the
// radix-8 stride of stage-1 writes over all banks.
#pragma once

#include "common.cuh"
#include "fft.cuh"

namespace pt {

// ---- radix 12 = 4 x 3 codelet ---------------------------------------------------
// X[k1 + 4 k2] = sum_l W3^{l k2} (W12^{l k1} Y_l[k1]),  Y_l = DFT4(x[l], x[l+3], x[l+6], x[l+9])
template <bool INV, typename C> __device__ __forceinline__ void dft12(C* x) {
  using R = typename real_of<C>::type;
  const R c30 = (R)0.86602540378443864676, s30 = (R)0.5;   // W12^1 = cos30 - i sin30
  C y[3][4];
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    y[l][0] = x[l]; y[l][1] = x[l + 3]; y[l][2] = x[l + 6]; y[l][3] = x[l + 9];
    dft4<INV>(y[l][0], y[l][1], y[l][2], y[l][3]);
  }
  // twiddles W12^{l k1}: l = 1: k1 = 1,2,3 -> W^1, W^2, W^3; l = 2: -> W^2, W^4, W^6
  auto tw = [&](C a, R c, R s) {   // a * (c - i s) forward, a * (c + i s) inverse
    return INV ? mk(a.x * c - a.y * s, a.x * s + a.y * c) : mk(a.x * c + a.y * s, a.y * c - a.x * s);
  };
  y[1][1] = tw(y[1][1], c30, s30);             // W^1
  y[1][2] = tw(y[1][2], s30, c30);             // W^2 = cos60 - i sin60
  y[1][3] = mul_mi<INV>(y[1][3]);              // W^3 = -i
  y[2][1] = tw(y[2][1], s30, c30);             // W^2
  y[2][2] = tw(y[2][2], -s30, c30);            // W^4 = cos120 - i sin120
  y[2][3] = mk(-y[2][3].x, -y[2][3].y);        // W^6 = -1
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    C a = y[0][k1], b = y[1][k1], c = y[2][k1];
    dft3<INV>(a, b, c);
    x[k1] = a; x[k1 + 4] = b; x[k1 + 8] = c;
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dftc(C* v) {
  if constexpr (R == 12) dft12<INV>(v);
  else dft<R, INV>(v);
}

template <int L> struct Plan2;
template <> struct Plan2<32> { static constexpr int R1 = 8, R2 = 4; };
template <> struct Plan2<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Plan2<96> { static constexpr int R1 = 8, R2 = 12; };

// Line buffers in shared memory are laid out with a row stride of L + 1
// complex values (rows = lines of the row-wise transforms), and every stage
// maps consecutive threads to consecutive lines with the same butterfly
// index. A half-warp then touches 16 different rows whose addresses differ by
// L + 1 = 1 (mod 16) complex values: the 64-bit accesses of a half-warp fall
// on 16 distinct bank pairs for row- and column-wise stages alike, and the
// twiddle index is uniform across the warp (a shared-memory broadcast).

// One Stockham stage over lines [line0, line0 + nl) of length L. Element e of
// line l of `src` is src[l * SLS + e * SES]; the output goes to `dst` with
// strides (DLS, DES). src == dst gives the in-place form (all reads of the
// stage finish before the first write). Lines at or beyond nl are skipped
// (NL is the compile-time line capacity of one call).
template <typename C, bool INV, int L, int R, int NS, int NL, int NT, int SLS, int SES, int DLS, int DES>
__device__ __forceinline__ void ct_stage_io(const C* src, C* dst, int nl, const C* __restrict__ tw, int tid,
                                            int line0 = 0) {
  constexpr int NBL = L / R;
  constexpr int MB = (NL * NBL + NT - 1) / NT;
  constexpr int TWS = L / (NS * R);
  C v[MB][R];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    const int ll = b % NL, j = b / NL;
    if (j < NBL && ll < nl) {
      const int base = (line0 + ll) * SLS;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[base + (j + r * NBL) * SES];
      if (NS > 1) {
        const int k = j % NS;
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[r * k * TWS];
          if (INV) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dftc<R, INV>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    const int ll = b % NL, j = b / NL;
    if (j < NBL && ll < nl) {
      const int base = (line0 + ll) * DLS;
      const int k = j % NS;
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[base + (o + r * NS) * DES] = v[q][r];
    }
  }
  __syncthreads();
}

template <typename C, bool INV, int L, int R, int NS, int NL, int NT, int LS, int ES>
__device__ __forceinline__ void ct_stage(C* buf, int nl, const C* __restrict__ tw, int tid, int line0 = 0) {
  ct_stage_io<C, INV, L, R, NS, NL, NT, LS, ES, LS, ES>(buf, buf, nl, tw, tid, line0);
}

// Forward stage 2 of plan (R1, R2), multiply each element by mul(line, e),
// inverse stage 1 of plan (R2, R1); all in registers between one read and one write.
template <typename C, int L, int NL, int NT, int LS, int ES, class Mul>
__device__ __forceinline__ void ct_fused(C* buf, int nl, const C* __restrict__ tw, int tid, Mul mul, int line0 = 0) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  constexpr int NBL = R1;   // = L / R2
  constexpr int MB = (NL * NBL + NT - 1) / NT;
  C v[MB][R2];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    const int ll = b % NL, j = b / NL;
    if (j < NBL && ll < nl) {
      const int line = line0 + ll;
      const int base = line * LS;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q][r] = buf[base + (j + r * R1) * ES];
#pragma unroll
      for (int r = 1; r < R2; ++r) v[q][r] = cmul(v[q][r], tw[r * j]);
      dftc<R2, false>(v[q]);
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q][r] = cscale(v[q][r], mul(line, j + r * R1));
      dftc<R2, true>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    const int ll = b % NL, j = b / NL;
    if (j < NBL && ll < nl) {
      const int base = (line0 + ll) * LS;
#pragma unroll
      for (int r = 0; r < R2; ++r) buf[base + (j * R2 + r) * ES] = v[q][r];
    }
  }
  __syncthreads();
}

// ---- bulk copies (TMA, non-tensor) and mbarriers --------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one arrival that also announces `bytes` of incoming transaction
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// global -> shared bulk copy completing on `bar`; addresses 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
               : "=r"(ok)
               : "r"(smem_u32(bar)), "r"(parity)
               : "memory");
  return ok != 0;
}

// Wait for phase `parity` with an iteration cap; false when the cap is hit.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, uint32_t parity, int cap = 1 << 22) {
  for (int it = 0; it < cap; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// order earlier generic-proxy accesses of shared memory before later async-proxy ones
__device__ __forceinline__ void fence_proxy_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Full forward (plan R1, R2) and inverse (plan R2, R1) line transforms in place.
template <typename C, int L, int NL, int NT, int LS, int ES>
__device__ __forceinline__ void ct_forward(C* buf, int nl, const C* tw, int tid, int line0 = 0) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage<C, false, L, R1, 1, NL, NT, LS, ES>(buf, nl, tw, tid, line0);
  ct_stage<C, false, L, R2, R1, NL, NT, LS, ES>(buf, nl, tw, tid, line0);
}

template <typename C, int L, int NL, int NT, int LS, int ES>
__device__ __forceinline__ void ct_inverse(C* buf, int nl, const C* tw, int tid, int line0 = 0) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage<C, true, L, R2, 1, NL, NT, LS, ES>(buf, nl, tw, tid, line0);
  ct_stage<C, true, L, R1, R2, NL, NT, LS, ES>(buf, nl, tw, tid, line0);
}

}  // namespace pt
