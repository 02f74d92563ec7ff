// Batched 1D FFTs of short lines held in shared memory (building block of
// every 3D transform in the library: the pair-density transforms of Eq. 3 and
// the orbital / density transforms of Sec. 3.2-3.4).
//
// A line of length L = R_1 R_2 ... R_s is transformed in place by s Stockham
// (self-sorting) stages. Stage with radix R, sub-transform length Ns so far:
//   butterfly j in [0, L/R): v_r = x[j + r L/R], k = j mod Ns,
//   v_r *= W_{Ns R}^{r k}, v = DFT_R(v), x[(j - k) R + k + r Ns] = v_r.
// Every thread reads all its butterflies into registers, the block
// synchronises, then writes: the stage is in place without a second buffer.
// Forward = exp(-2 pi i ...), inverse = exp(+2 pi i ...) unnormalised.
// Twiddles W_L^t = exp(-2 pi i t / L) come from a table built on the host in
// double precision with the C library's cos / sin.
#pragma once

#include "common.cuh"

namespace pt {

// ---- radix codelets (in registers) ---------------------------------------
template <bool INV, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
  C t = a;
  a = cadd(t, b);
  b = csub(t, b);
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C& x0, C& x1, C& x2) {
  using R = typename real_of<C>::type;
  const R s3 = (R)0.86602540378443864676;  // sin(2 pi / 3)
  C s = cadd(x1, x2);
  C d = cscale(csub(x1, x2), s3);
  C t = csub(x0, cscale(s, (R)0.5));
  x0 = cadd(x0, s);
  C md = mul_mi<INV>(d);
  x1 = cadd(t, md);
  x2 = csub(t, md);
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
  C a = cadd(x0, x2), b = csub(x0, x2), c = cadd(x1, x3), d = mul_mi<INV>(csub(x1, x3));
  x0 = cadd(a, c);
  x2 = csub(a, c);
  x1 = cadd(b, d);
  x3 = csub(b, d);
}

// multiply by W_8^1 = (1 -+ i)/sqrt(2)
template <bool INV, typename C> __device__ __forceinline__ C mul_w8(C o) {
  using R = typename real_of<C>::type;
  const R h = (R)0.70710678118654752440;
  return INV ? mk((o.x - o.y) * h, (o.x + o.y) * h) : mk((o.x + o.y) * h, (o.y - o.x) * h);
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* x) {
  dft4<INV>(x[0], x[2], x[4], x[6]);
  dft4<INV>(x[1], x[3], x[5], x[7]);
  C o1 = mul_w8<INV>(x[3]);
  C o2 = mul_mi<INV>(x[5]);
  C o3 = mul_mi<INV>(mul_w8<INV>(x[7]));
  C e0 = x[0], e1 = x[2], e2 = x[4], e3 = x[6], o0 = x[1];
  x[0] = cadd(e0, o0); x[4] = csub(e0, o0);
  x[1] = cadd(e1, o1); x[5] = csub(e1, o1);
  x[2] = cadd(e2, o2); x[6] = csub(e2, o2);
  x[3] = cadd(e3, o3); x[7] = csub(e3, o3);
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C* v) {
  if constexpr (R == 2) dft2<INV>(v[0], v[1]);
  else if constexpr (R == 3) dft3<INV>(v[0], v[1], v[2]);
  else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
  else if constexpr (R == 8) dft8<INV>(v);
}

// Butterflies a thread may hold in registers per stage.
template <typename T, int R> struct MaxB;
template <> struct MaxB<float, 8> { static constexpr int v = 2; };
template <> struct MaxB<float, 4> { static constexpr int v = 4; };
template <> struct MaxB<float, 3> { static constexpr int v = 6; };
template <> struct MaxB<float, 2> { static constexpr int v = 8; };
template <> struct MaxB<double, 4> { static constexpr int v = 3; };
template <> struct MaxB<double, 3> { static constexpr int v = 4; };
template <> struct MaxB<double, 2> { static constexpr int v = 6; };

// One Stockham stage over `nlines` lines. Element e of line l sits at
// buf[l * lstride + e * estride]. LM (line-major): consecutive threads walk
// along a line (use when estride == 1); otherwise across lines.
template <typename T, bool INV, bool LM, int R>
__device__ __forceinline__ void stage(cplx<T>* buf, int L, int Ns, int nlines, int lstride, int estride,
                                      const cplx<T>* tw, int tid, int nthr) {
  using C = cplx<T>;
  constexpr int MB = MaxB<T, R>::v;
  const int nbl = L / R;
  const int total = nlines * nbl;
  const int twstep = L / (Ns * R);
  C v[MB][R];
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * nthr;
    if (b < total) {
      int line, j;
      if (LM) { line = b / nbl; j = b - line * nbl; }
      else { j = b / nlines; line = b - j * nlines; }
      const C* base = buf + (size_t)line * lstride;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = base[(j + r * nbl) * estride];
      const int k = j % Ns;
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          C w = tw[r * k * twstep];
          if (INV) w.y = -w.y;
          v[q][r] = cmul(v[q][r], w);
        }
      }
      dft<R, INV>(v[q]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MB; ++q) {
    const int b = tid + q * nthr;
    if (b < total) {
      int line, j;
      if (LM) { line = b / nbl; j = b - line * nbl; }
      else { j = b / nlines; line = b - j * nlines; }
      C* base = buf + (size_t)line * lstride;
      const int k = j % Ns;
      const int o = (j - k) * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) base[(o + r * Ns) * estride] = v[q][r];
    }
  }
  __syncthreads();
}

// Radix plans. FP32 favours radix 8 (fewer shared-memory round trips); FP64
// keeps radix <= 4 to bound registers (FP64 work is ALU-bound on this part).
template <typename T, bool INV, bool LM>
__device__ __forceinline__ void fft_lines(cplx<T>* buf, int L, int nlines, int lstride, int estride,
                                          const cplx<T>* tw, int tid, int nthr) {
#define PT_ST(R, NS) stage<T, INV, LM, R>(buf, L, NS, nlines, lstride, estride, tw, tid, nthr)
  if constexpr (sizeof(T) == 4) {
    switch (L) {
      case 8: PT_ST(8, 1); break;
      case 12: PT_ST(4, 1); PT_ST(3, 4); break;
      case 16: PT_ST(4, 1); PT_ST(4, 4); break;
      case 24: PT_ST(8, 1); PT_ST(3, 8); break;
      case 32: PT_ST(8, 1); PT_ST(4, 8); break;
      case 48: PT_ST(4, 1); PT_ST(4, 4); PT_ST(3, 16); break;
      case 64: PT_ST(8, 1); PT_ST(8, 8); break;
      case 96: PT_ST(8, 1); PT_ST(4, 8); PT_ST(3, 32); break;
      default: break;
    }
  } else {
    switch (L) {
      case 8: PT_ST(4, 1); PT_ST(2, 4); break;
      case 12: PT_ST(4, 1); PT_ST(3, 4); break;
      case 16: PT_ST(4, 1); PT_ST(4, 4); break;
      case 24: PT_ST(4, 1); PT_ST(3, 4); PT_ST(2, 12); break;
      case 32: PT_ST(4, 1); PT_ST(4, 4); PT_ST(2, 16); break;
      case 48: PT_ST(4, 1); PT_ST(4, 4); PT_ST(3, 16); break;
      case 64: PT_ST(4, 1); PT_ST(4, 4); PT_ST(4, 16); break;
      case 96: PT_ST(4, 1); PT_ST(4, 4); PT_ST(3, 16); PT_ST(2, 48); break;
      default: break;
    }
  }
#undef PT_ST
}

// Host-side mirror of the plans: minimum threads for `nlines` lines of length L.
inline int fft_threads_needed(int L, int nlines, bool fp64) {
  struct S { int r, mb; };
  S st[4];
  int ns = 0;
  auto add = [&](int r) {
    int mb;
    if (!fp64) mb = r == 8 ? 2 : r == 4 ? 4 : r == 3 ? 6 : 8;
    else mb = r == 4 ? 3 : r == 3 ? 4 : 6;
    st[ns++] = S{r, mb};
  };
  if (!fp64) {
    switch (L) {
      case 8: add(8); break;
      case 12: add(4); add(3); break;
      case 16: add(4); add(4); break;
      case 24: add(8); add(3); break;
      case 32: add(8); add(4); break;
      case 48: add(4); add(4); add(3); break;
      case 64: add(8); add(8); break;
      case 96: add(8); add(4); add(3); break;
      default: return -1;
    }
  } else {
    switch (L) {
      case 8: add(4); add(2); break;
      case 12: add(4); add(3); break;
      case 16: add(4); add(4); break;
      case 24: add(4); add(3); add(2); break;
      case 32: add(4); add(4); add(2); break;
      case 48: add(4); add(4); add(3); break;
      case 64: add(4); add(4); add(4); break;
      case 96: add(4); add(4); add(3); add(2); break;
      default: return -1;
    }
  }
  int need = 1;
  for (int i = 0; i < ns; ++i) {
    long tot = (long)nlines * (L / st[i].r);
    int t = (int)((tot + st[i].mb - 1) / st[i].mb);
    if (t > need) need = t;
  }
  return need;
}

inline bool fft_length_supported(int L) {
  return L == 8 || L == 12 || L == 16 || L == 24 || L == 32 || L == 48 || L == 64 || L == 96;
}

}  // namespace pt
