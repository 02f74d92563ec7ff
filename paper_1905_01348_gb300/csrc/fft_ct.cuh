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

__device__ __forceinline__ int pidx(int i) { return i + (i >> 3); }
constexpr int padded(int n) { return n + n / 8 + 1; }

// One Stockham stage over lines of length L. Element e of line l is
// buf[pidx(l * LSTR + e * ESTR)]. LM: consecutive threads walk along a line
// (line count nl may be below NL); otherwise across lines (nl == NL).
template <typename C, bool INV, int L, int R, int NS, int NL, int NT, bool LM, int LSTR, int ESTR>
__device__ __forceinline__ void ct_stage(C* buf, int nl, const C* __restrict__ tw, int tid) {
  constexpr int NBL = L / R;
  constexpr int MB = (NL * NBL + NT - 1) / NT;
  constexpr int TWS = L / (NS * R);
  const int total = nl * NBL;
  C v[MB][R];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    if (b < total) {
      const int line = LM ? b / NBL : b % NL;
      const int j = LM ? b % NBL : b / NL;
      const int base = line * LSTR;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[pidx(base + (j + r * NBL) * ESTR)];
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
    if (b < total) {
      const int line = LM ? b / NBL : b % NL;
      const int j = LM ? b % NBL : b / NL;
      const int base = line * LSTR;
      const int k = j % NS;
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[pidx(base + (o + r * NS) * ESTR)] = v[q][r];
    }
  }
  __syncthreads();
}

// Forward stage 2 of plan (R1, R2), multiply each element by mul(line, e),
// inverse stage 1 of plan (R2, R1); all in registers between one read and one write.
template <typename C, int L, int NL, int NT, bool LM, int LSTR, int ESTR, class Mul>
__device__ __forceinline__ void ct_fused(C* buf, int nl, const C* __restrict__ tw, int tid, Mul mul) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  constexpr int NBL = R1;   // = L / R2
  constexpr int MB = (NL * NBL + NT - 1) / NT;
  const int total = nl * NBL;
  C v[MB][R2];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * NT;
    if (b < total) {
      const int line = LM ? b / NBL : b % NL;
      const int j = LM ? b % NBL : b / NL;
      const int base = line * LSTR;
#pragma unroll
      for (int r = 0; r < R2; ++r) v[q][r] = buf[pidx(base + (j + r * R1) * ESTR)];
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
    if (b < total) {
      const int line = LM ? b / NBL : b % NL;
      const int j = LM ? b % NBL : b / NL;
      const int base = line * LSTR;
#pragma unroll
      for (int r = 0; r < R2; ++r) buf[pidx(base + (j * R2 + r) * ESTR)] = v[q][r];
    }
  }
  __syncthreads();
}

// Full forward (plan R1, R2) and inverse (plan R2, R1) line transforms.
template <typename C, int L, int NL, int NT, bool LM, int LSTR, int ESTR>
__device__ __forceinline__ void ct_forward(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage<C, false, L, R1, 1, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
  ct_stage<C, false, L, R2, R1, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
}

template <typename C, int L, int NL, int NT, bool LM, int LSTR, int ESTR>
__device__ __forceinline__ void ct_inverse(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage<C, true, L, R2, 1, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
  ct_stage<C, true, L, R1, R2, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
}

// inverse stage 2 alone (after ct_fused)
template <typename C, int L, int NL, int NT, bool LM, int LSTR, int ESTR>
__device__ __forceinline__ void ct_inverse_stage2(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1, R2 = Plan2<L>::R2;
  ct_stage<C, true, L, R1, R2, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
}

template <typename C, int L, int NL, int NT, bool LM, int LSTR, int ESTR>
__device__ __forceinline__ void ct_forward_stage1(C* buf, int nl, const C* tw, int tid) {
  constexpr int R1 = Plan2<L>::R1;
  ct_stage<C, false, L, R1, 1, NL, NT, LM, LSTR, ESTR>(buf, nl, tw, tid);
}

}  // namespace pt
