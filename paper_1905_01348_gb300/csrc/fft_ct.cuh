// Compile-time-sized line FFTs for the pair pipeline (lengths 32, 48, 64, 96).
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
template <> struct Plan2<48> { static constexpr int R1 = 4, R2 = 12; };
template <> struct Plan2<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct Plan2<96> { static constexpr int R1 = 8, R2 = 12; };

// Line buffers in shared memory are laid out with a row stride of L + 1
// complex values (rows = lines of the row-wise transforms), and every stage
// maps consecutive threads to consecutive lines with the same butterfly
// index. A half-warp then touches 16 different rows whose addresses differ by
// L + 1 = 1 (mod 16) complex values: the 64-bit accesses of a half-warp fall
// on 16 distinct bank pairs for row- and column-wise stages alike, and the
// twiddle index is uniform across the warp (a shared-memory broadcast).

// Shared-memory layouts: Strided<LS, ES> puts element e of line l at
// l * LS + e * ES; kernels may define their own (a struct with a static at(l, e)).
template <int LS, int ES> struct Strided {
  __device__ __forceinline__ static int at(int l, int e) { return l * LS + e * ES; }
};

// One Stockham stage over lines [line0, line0 + nl) of length L, reading
// through layout SA from `src` and writing through layout DA to `dst`
// (src == dst: in place; every read of the stage finishes before the first
// write). Lines at or beyond nl are skipped (NL is the per-call capacity).
template <typename C, bool INV, int L, int R, int NS, int NL, int NT, class SA, class DA>
__device__ __forceinline__ void ct_stage_lay(const C* src, C* dst, int nl, const C* __restrict__ tw, int tid,
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
      const int line = line0 + ll;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = src[SA::at(line, j + r * NBL)];
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
      const int line = line0 + ll;
      const int k = j % NS;
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[DA::at(line, o + r * NS)] = v[q][r];
    }
  }
  __syncthreads();
}

template <typename C, bool INV, int L, int R, int NS, int NL, int NT, int SLS, int SES, int DLS, int DES>
__device__ __forceinline__ void ct_stage_io(const C* src, C* dst, int nl, const C* __restrict__ tw, int tid,
                                            int line0 = 0) {
  ct_stage_lay<C, INV, L, R, NS, NL, NT, Strided<SLS, SES>, Strided<DLS, DES>>(src, dst, nl, tw, tid, line0);
}

template <typename C, int L, int NL, int NT, class A>
__device__ __forceinline__ void ct_forward_lay(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage_lay<C, false, L, R1, 1, NL, NT, A, A>(buf, buf, nl, tw, tid);
  ct_stage_lay<C, false, L, R2, R1, NL, NT, A, A>(buf, buf, nl, tw, tid);
}

template <typename C, int L, int NL, int NT, class A>
__device__ __forceinline__ void ct_inverse_lay(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage_lay<C, true, L, R2, 1, NL, NT, A, A>(buf, buf, nl, tw, tid);
  ct_stage_lay<C, true, L, R1, R2, NL, NT, A, A>(buf, buf, nl, tw, tid);
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
