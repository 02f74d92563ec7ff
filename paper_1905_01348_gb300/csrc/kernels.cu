// Elementwise and reduction kernels of the PT-CN step (Alg. 1, Alg. 3,
// Sec. 3.4) and of the local part of the Hamiltonian (Eq. 2).
// Reductions are two-level (block partials, then one block sums the
// partials in order), so every sum is deterministic.
#include <algorithm>
#include <cmath>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "kernels.h"

namespace pt {

static inline unsigned nblk(long n, int thr, long cap = 152L * 16) {
  return (unsigned)std::max<long>(1, std::min<long>((n + thr - 1) / thr, cap));
}

// ---- block reduction helper (fixed order) ----------------------------------
template <int NS>
__device__ __forceinline__ void block_sums(double (&v)[NS], double* part) {
  __shared__ double sh[NS][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int s = 0; s < NS; ++s) {
    double x = v[s];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[s][warp] = x;
  }
  __syncthreads();
  if (threadIdx.x < NS) {
    const int nw = blockDim.x >> 5;
    double t = 0.0;
    for (int w = 0; w < nw; ++w) t += sh[threadIdx.x][w];
    part[blockIdx.x * NS + threadIdx.x] = t;
  }
}

__global__ void k_finalize(const double* __restrict__ part, int nblocks, int ns, double* __restrict__ out) {
  const int s = threadIdx.x;
  if (s >= ns) return;
  double t = 0.0;
  for (int b = 0; b < nblocks; ++b) t += part[b * ns + s];
  out[s] = t;
}

// ---- density ------------------------------------------------------------------
__global__ void k_density(const double2* __restrict__ psi_r, long N, int ne, double* __restrict__ rho) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < N; r += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < ne; ++k) {
      const double2 v = psi_r[(long)k * N + r];
      s += v.x * v.x + v.y * v.y;
    }
    rho[r] = 2.0 * s;
  }
}

cudaError_t density(const double2* psi_r, long N, int ne, double* rho, cudaStream_t s) {
  k_density<<<nblk(N, 256, 152L * 64), 256, 0, s>>>(psi_r, N, ne, rho); launched();
  return cudaGetLastError();
}

// FP32 squares summed in FP32 over groups of 16 bands (eight loads in flight
// per thread), the group sums accumulated in FP64: FP64 work drops 16-fold.
__global__ void k_density32(const float2* __restrict__ psi_r, long N, int ne, double* __restrict__ rho) {
  constexpr int G = 16;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < N; r += (long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k0 = 0; k0 < ne; k0 += G) {
      const int kn = min(G, ne - k0);
      float g = 0.f;
#pragma unroll 8
      for (int k = 0; k < kn; ++k) {
        const float2 v = __ldg(psi_r + (long)(k0 + k) * N + r);
        g = fmaf(v.x, v.x, fmaf(v.y, v.y, g));
      }
      s += (double)g;
    }
    rho[r] = 2.0 * s;
  }
}

cudaError_t density32(const float2* psi_r, long N, int ne, double* rho, cudaStream_t s) {
  k_density32<<<nblk(N, 256, 152L * 64), 256, 0, s>>>(psi_r, N, ne, rho); launched();
  return cudaGetLastError();
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) b[t] = (float)a[t];
}

cudaError_t to_float(const double* a, float* b, long n, cudaStream_t s) {
  k_to_float<<<nblk(n, 256), 256, 0, s>>>(a, b, n); launched();
  return cudaGetLastError();
}

// ---- local potential -----------------------------------------------------------
__global__ void k_rho_to_complex(const double* __restrict__ rho, double2* __restrict__ buf, long N) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < N; r += (long)gridDim.x * blockDim.x)
    buf[r] = make_double2(rho[r], 0.0);
}

__global__ void k_vloc(const double* __restrict__ vion, const double2* __restrict__ vh_c, const double* __restrict__ rho,
                       long N, int use_h, double w_lda, double* __restrict__ vh, double* __restrict__ vloc) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < N; r += (long)gridDim.x * blockDim.x) {
    double v = vion[r];
    if (use_h) {
      const double h = vh_c[r].x;
      vh[r] = h;
      v += h;
    }
    if (w_lda != 0.0) v += w_lda * (-cbrt(3.0 * rho[r] / M_PI));
    vloc[r] = v;
  }
}

cudaError_t rho_to_complex(const double* rho, double2* buf, long N, cudaStream_t s) {
  k_rho_to_complex<<<nblk(N, 256), 256, 0, s>>>(rho, buf, N); launched();
  return cudaGetLastError();
}

cudaError_t assemble_vloc(const double* vion, const double2* vh_c, const double* rho, long N, int use_h, double w_lda,
                          double* vh, double* vloc, cudaStream_t s) {
  k_vloc<<<nblk(N, 256), 256, 0, s>>>(vion, vh_c, rho, N, use_h, w_lda, vh, vloc); launched();
  return cudaGetLastError();
}

// Gaussian wells summed over atoms and periodic images in real space.
__global__ void k_vion(double* __restrict__ v, int n0, int n1, int n2, double a0, double a1, double a2,
                       const double* __restrict__ atoms, int na, double depth, double sigma, double rcut) {
  const long N = (long)n0 * n1 * n2;
  const double inv2s2 = 1.0 / (2.0 * sigma * sigma);
  const int m0 = (int)ceil(rcut / a0), m1 = (int)ceil(rcut / a1), m2 = (int)ceil(rcut / a2);
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    const int i2 = (int)(t % n2);
    const int i1 = (int)((t / n2) % n1);
    const int i0 = (int)(t / ((long)n1 * n2));
    const double x = a0 * i0 / n0, y = a1 * i1 / n1, z = a2 * i2 / n2;
    double s = 0.0;
    for (int a = 0; a < na; ++a) {
      const double ax = atoms[3 * a] * a0, ay = atoms[3 * a + 1] * a1, az = atoms[3 * a + 2] * a2;
      for (int p = -m0; p <= m0; ++p) {
        const double dx = x - ax - p * a0;
        if (fabs(dx) > rcut) continue;
        for (int q = -m1; q <= m1; ++q) {
          const double dy = y - ay - q * a1;
          if (fabs(dy) > rcut) continue;
          for (int w = -m2; w <= m2; ++w) {
            const double dz = z - az - w * a2;
            const double d2 = dx * dx + dy * dy + dz * dz;
            if (d2 <= rcut * rcut) s += exp(-d2 * inv2s2);
          }
        }
      }
    }
    v[t] = -depth * s;
  }
}

cudaError_t ion_potential(double* v, Grid3 g, const double* cell, const double* d_atoms, int na, double depth,
                          double sigma, cudaStream_t s) {
  // exp(-d^2 / (2 sigma^2)) < 1e-20 beyond rcut
  const double rcut = sigma * std::sqrt(2.0 * 46.0);
  k_vion<<<nblk(g.N(), 128, 152L * 64), 128, 0, s>>>(v, g.n0, g.n1, g.n2, cell[0], cell[1], cell[2], d_atoms, na,
                                                     depth, sigma, rcut); launched();
  return cudaGetLastError();
}

// ---- PT residual (Alg. 1 and Alg. 3) ---------------------------------------------
// psi_half = psi - i dt/2 R
__global__ void k_half_step(const double2* __restrict__ psi, const double2* __restrict__ R, double hdt,
                            double2* __restrict__ out, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double2 p = psi[t], r = R[t];
    // -i hdt (rx + i ry) = hdt ry - i hdt rx
    out[t] = make_double2(p.x + hdt * r.y, p.y - hdt * r.x);
  }
}

cudaError_t half_step(const double2* psi, const double2* R, double hdt, double2* out, long n, cudaStream_t s) {
  k_half_step<<<nblk(n, 256), 256, 0, s>>>(psi, R, hdt, out, n); launched();
  return cudaGetLastError();
}

// r = -(psi_f + i dt/2 T - psi_half); block partials of |r|^2
__global__ void k_resid(const double2* __restrict__ psi_f, const double2* __restrict__ T, const double2* __restrict__ ph,
                        double hdt, double2* __restrict__ r, long n, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double2 p = psi_f[t], q = T[t], h = ph[t];
    // i hdt (qx + i qy) = -hdt qy + i hdt qx
    const double2 R = make_double2(p.x - hdt * q.y - h.x, p.y + hdt * q.x - h.y);
    r[t] = make_double2(-R.x, -R.y);
    acc[0] += R.x * R.x + R.y * R.y;
  }
  block_sums<1>(acc, part);
}

cudaError_t pt_residual(const double2* psi_f, const double2* T, const double2* ph, double hdt, double2* r, long n,
                        double* part, double* out_norm2, cudaStream_t s) {
  const unsigned b = nblk(n, 256, 1024);
  k_resid<<<b, 256, 0, s>>>(psi_f, T, ph, hdt, r, n, part); launched();
  k_finalize<<<1, 32, 0, s>>>(part, b, 1, out_norm2); launched();
  return cudaGetLastError();
}

// y = x - tau * P * R, P = 1 / (1 + kin) per basis vector (start-state relaxation)
__global__ void k_precond_step(double2* __restrict__ x, const double2* __restrict__ R, const double* __restrict__ kin,
                               int npw, long n, double tau) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double p = tau / (1.0 + kin[t % npw]);
    const double2 r = R[t];
    double2 v = x[t];
    v.x -= p * r.x;
    v.y -= p * r.y;
    x[t] = v;
  }
}

cudaError_t precond_step(double2* x, const double2* R, const double* kin, int npw, long n, double tau, cudaStream_t s) {
  k_precond_step<<<nblk(n, 256), 256, 0, s>>>(x, R, kin, npw, n, tau); launched();
  return cudaGetLastError();
}

// ---- Anderson mixing (Sec. 3.4), per band -------------------------------------------
// push: dX[slot] = x - x_prev, dR[slot] = r - r_prev (when have_prev), then x_prev = x, r_prev = r
// History entries are stored as H: complex128, or complex64 in mixed precision
// (the differences of successive iterates and residuals, whose rounding to FP32
// only perturbs the least-squares extrapolation, not the fixed point).
template <typename H>
__global__ void k_anderson_push(const double2* __restrict__ x, const double2* __restrict__ r, double2* __restrict__ xp,
                                double2* __restrict__ rp, H* __restrict__ dx, H* __restrict__ dr, long n,
                                int have_prev) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double2 a = x[t], b = r[t];
    if (have_prev) {
      const double2 c = xp[t], d = rp[t];
      dx[t] = {(decltype(H::x))(a.x - c.x), (decltype(H::x))(a.y - c.y)};
      dr[t] = {(decltype(H::x))(b.x - d.x), (decltype(H::x))(b.y - d.y)};
    }
    xp[t] = a;
    rp[t] = b;
  }
}

cudaError_t anderson_push(const double2* x, const double2* r, double2* xp, double2* rp, void* dx, void* dr, long n,
                          int have_prev, int f32, cudaStream_t s) {
  if (f32)
    k_anderson_push<float2><<<nblk(n, 256), 256, 0, s>>>(x, r, xp, rp, (float2*)dx, (float2*)dr, n, have_prev);
  else
    k_anderson_push<double2><<<nblk(n, 256), 256, 0, s>>>(x, r, xp, rp, (double2*)dx, (double2*)dr, n, have_prev);
  launched();
  return cudaGetLastError();
}

// For each band b: gram[b][slot_q][new] = <dR_{slot_q}, dR_new>_b (and its
// conjugate at [new][slot_q]) and rhs[b][q] = <dR_{slot_q}, r>_b for the
// history slots in order (oldest first). One block per band; the slots are
// processed four at a time to bound registers.
// Complex64 history (mixed precision): the products are formed in FP32 and
// summed in FP32 over each thread's share of the basis (about npw / 256 terms);
// the per-thread sums are reduced in FP64. FP64 otherwise. The Gram matrix and
// right-hand side feed the FP64 solve either way.
template <typename H>
__global__ void k_anderson_dots(const H* __restrict__ dR, long slot_stride, SlotList sl, int newslot,
                                const double2* __restrict__ r, int npw, int mdim, double2* __restrict__ gram,
                                double2* __restrict__ rhs) {
  using A = decltype(H::x);
  const int b = blockIdx.x;
  const int k = sl.k;
  const long boff = (long)b * npw;
  const H* dn = dR + (long)newslot * slot_stride + boff;
  const double2* rb = r + boff;
  __shared__ double sh[16][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int q0 = 0; q0 < k; q0 += 4) {
    A acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = (A)0;
    for (int g = threadIdx.x; g < npw; g += blockDim.x) {
      const H vnd = dn[g];
      const double2 vrd = rb[g];
      const A vnx = vnd.x, vny = vnd.y, vrx = (A)vrd.x, vry = (A)vrd.y;
#pragma unroll
      for (int qq = 0; qq < 4; ++qq) {
        if (q0 + qq < k) {
          const H ud = dR[(long)sl.s[q0 + qq] * slot_stride + boff + g];
          const A ux = ud.x, uy = ud.y;
          acc[4 * qq + 0] += ux * vnx + uy * vny;
          acc[4 * qq + 1] += ux * vny - uy * vnx;
          acc[4 * qq + 2] += ux * vrx + uy * vry;
          acc[4 * qq + 3] += ux * vry - uy * vrx;
        }
      }
    }
#pragma unroll
    for (int c = 0; c < 16; ++c) {
      double x = (double)acc[c];
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) sh[c][warp] = x;
    }
    __syncthreads();
    if (threadIdx.x < 4 && q0 + (int)threadIdx.x < k) {
      const int qq = threadIdx.x, q = q0 + qq;
      double v[4];
      for (int c = 0; c < 4; ++c) {
        double t = 0.0;
        for (int w = 0; w < nw; ++w) t += sh[4 * qq + c][w];
        v[c] = t;
      }
      const long gb = (long)b * mdim * mdim;
      const int sq = sl.s[q];
      if (sq == newslot) {
        gram[gb + (long)sq * mdim + sq] = make_double2(v[0], 0.0);
      } else {
        gram[gb + (long)sq * mdim + newslot] = make_double2(v[0], v[1]);
        gram[gb + (long)newslot * mdim + sq] = make_double2(v[0], -v[1]);
      }
      rhs[(long)b * mdim + q] = make_double2(v[2], v[3]);
    }
    __syncthreads();
  }
}

cudaError_t anderson_dots(const void* dR, long slot_stride, const SlotList& sl, int newslot, const double2* r,
                          int npw, int ne, int mdim, double2* gram, double2* rhs, int f32, cudaStream_t s) {
  if (sl.k > kSlotMax) return cudaErrorInvalidValue;
  if (f32)
    k_anderson_dots<float2><<<ne, 256, 0, s>>>((const float2*)dR, slot_stride, sl, newslot, r, npw, mdim, gram, rhs);
  else
    k_anderson_dots<double2><<<ne, 256, 0, s>>>((const double2*)dR, slot_stride, sl, newslot, r, npw, mdim, gram, rhs);
  launched();
  return cudaGetLastError();
}

// Solve (G + 1e-14 tr(G) I) gamma = rhs per band by Cholesky; gamma = 0 when
// the trace is zero or a pivot is not positive. One thread per band.
__global__ void k_anderson_solve(const double2* __restrict__ gram, const double2* __restrict__ rhs, SlotList sl,
                                 int mdim, int ne, double2* __restrict__ gamma) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= ne) return;
  const int k = sl.k;
  double2 L[kSlotMax][kSlotMax];
  double2 y[kSlotMax];
  const long gb = (long)b * mdim * mdim;
  double tr = 0.0;
  for (int q = 0; q < k; ++q) tr += gram[gb + (long)sl.s[q] * mdim + sl.s[q]].x;
  bool ok = tr > 0.0;
  const double shift = 1e-14 * tr;
  // L L^H = A with A[i][j] = G[s_i][s_j]  (G[s][t] = <dR_s, dR_t>)
  for (int j = 0; j < k && ok; ++j) {
    double d = gram[gb + (long)sl.s[j] * mdim + sl.s[j]].x + shift;
    for (int p = 0; p < j; ++p) d -= L[j][p].x * L[j][p].x + L[j][p].y * L[j][p].y;
    if (!(d > 0.0)) { ok = false; break; }
    const double ljj = sqrt(d);
    L[j][j] = make_double2(ljj, 0.0);
    for (int i = j + 1; i < k; ++i) {
      double2 a = gram[gb + (long)sl.s[i] * mdim + sl.s[j]];
      for (int p = 0; p < j; ++p) {
        // a -= L[i][p] * conj(L[j][p])
        a.x -= L[i][p].x * L[j][p].x + L[i][p].y * L[j][p].y;
        a.y -= L[i][p].y * L[j][p].x - L[i][p].x * L[j][p].y;
      }
      L[i][j] = make_double2(a.x / ljj, a.y / ljj);
    }
  }
  if (!ok) {
    for (int q = 0; q < k; ++q) gamma[(long)b * mdim + q] = make_double2(0.0, 0.0);
    return;
  }
  for (int i = 0; i < k; ++i) {   // L y = rhs
    double2 a = rhs[(long)b * mdim + i];
    for (int p = 0; p < i; ++p) {
      a.x -= L[i][p].x * y[p].x - L[i][p].y * y[p].y;
      a.y -= L[i][p].x * y[p].y + L[i][p].y * y[p].x;
    }
    y[i] = make_double2(a.x / L[i][i].x, a.y / L[i][i].x);
  }
  for (int i = k - 1; i >= 0; --i) {   // L^H g = y
    double2 a = y[i];
    for (int p = i + 1; p < k; ++p) {
      const double2 gp = y[p];
      a.x -= L[p][i].x * gp.x + L[p][i].y * gp.y;
      a.y -= L[p][i].x * gp.y - L[p][i].y * gp.x;
    }
    y[i] = make_double2(a.x / L[i][i].x, a.y / L[i][i].x);
  }
  for (int q = 0; q < k; ++q) gamma[(long)b * mdim + q] = y[q];
}

cudaError_t anderson_solve(const double2* gram, const double2* rhs, const SlotList& sl, int mdim, int ne,
                           double2* gamma, cudaStream_t s) {
  k_anderson_solve<<<(ne + 63) / 64, 64, 0, s>>>(gram, rhs, sl, mdim, ne, gamma); launched();
  return cudaGetLastError();
}

// x <- x + beta r - sum_q (dX_q + beta dR_q) gamma_q  (per band)
// x += beta r - sum_q gamma_q (dX_q + beta dR_q). One block row per band (no
// division per element). With complex64 history the correction sum is formed
// in FP32 and added to the FP64 iterate once.
template <typename H>
__global__ void k_anderson_update(double2* __restrict__ x, const double2* __restrict__ r, const H* __restrict__ dX,
                                  const H* __restrict__ dR, long slot_stride, SlotList sl,
                                  const double2* __restrict__ gamma, int mdim, int npw, double beta) {
  using A = decltype(H::x);
  const int k = sl.k;
  const int b = blockIdx.y;
  const long boff = (long)b * npw;
  __shared__ A gs[2 * kSlotMax];
  if (threadIdx.x < k) {
    const double2 g = gamma[(long)b * mdim + threadIdx.x];
    gs[2 * threadIdx.x] = (A)g.x;
    gs[2 * threadIdx.x + 1] = (A)g.y;
  }
  __syncthreads();
  const A bt = (A)beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < npw; i += gridDim.x * blockDim.x) {
    const long t = boff + i;
    A cx = 0, cy = 0;
    for (int q = 0; q < k; ++q) {
      const long sq = (long)sl.s[q] * slot_stride + t;
      const H a = dX[sq], c = dR[sq];
      const A ux = a.x + bt * c.x, uy = a.y + bt * c.y;
      const A gx = gs[2 * q], gy = gs[2 * q + 1];
      cx += ux * gx - uy * gy;
      cy += ux * gy + uy * gx;
    }
    double2 v = x[t];
    const double2 rr = r[t];
    v.x += beta * rr.x - (double)cx;
    v.y += beta * rr.y - (double)cy;
    x[t] = v;
  }
}

cudaError_t anderson_update(double2* x, const double2* r, const void* dX, const void* dR, long slot_stride,
                            const SlotList& sl, const double2* gamma, int mdim, int npw, long n, double beta, int f32,
                            cudaStream_t s) {
  if (sl.k > kSlotMax) return cudaErrorInvalidValue;
  const int ne = npw > 0 ? (int)(n / npw) : 0;
  if (ne == 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min(32, (npw + 255) / 256), (unsigned)ne);
  if (f32)
    k_anderson_update<float2><<<grid, 256, 0, s>>>(x, r, (const float2*)dX, (const float2*)dR, slot_stride, sl, gamma,
                                                   mdim, npw, beta);
  else
    k_anderson_update<double2><<<grid, 256, 0, s>>>(x, r, (const double2*)dX, (const double2*)dR, slot_stride, sl,
                                                    gamma, mdim, npw, beta);
  launched();
  return cudaGetLastError();
}

// kin[k] = |gk[k] + a|^2 / 2 with gk the basis vectors G + kick (three arrays of npw)
__global__ void k_kinetic_shifted(const double* __restrict__ gk3, int npw, double ax, double ay, double az,
                                  double* __restrict__ kin) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < npw; k += gridDim.x * blockDim.x) {
    const double x = gk3[k] + ax, y = gk3[npw + k] + ay, z = gk3[2 * (long)npw + k] + az;
    kin[k] = 0.5 * (x * x + y * y + z * z);
  }
}

cudaError_t kinetic_shifted(const double* gk3, int npw, double ax, double ay, double az, double* kin, cudaStream_t s) {
  k_kinetic_shifted<<<nblk(npw, 256), 256, 0, s>>>(gk3, npw, ax, ay, az, kin); launched();
  return cudaGetLastError();
}

// ---- density change, energy, dipole ---------------------------------------------------
__global__ void k_drho(const double* __restrict__ a, const double* __restrict__ b, long N, double* __restrict__ part) {
  double acc[1] = {0.0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x)
    acc[0] += fabs(a[t] - b[t]);
  block_sums<1>(acc, part);
}

cudaError_t rho_change(const double* a, const double* b, long N, double* part, double* out, cudaStream_t s) {
  const unsigned nb = nblk(N, 256, 1024);
  k_drho<<<nb, 256, 0, s>>>(a, b, N, part); launched();
  k_finalize<<<1, 32, 0, s>>>(part, nb, 1, out); launched();
  return cudaGetLastError();
}

// grid sums: [0] vion*rho, [1] vh*rho, [2] rho^{4/3}, [3..5] r*rho
__global__ void k_grid_sums(const double* __restrict__ rho, const double* __restrict__ vion,
                            const double* __restrict__ vh, int use_h, int n0, int n1, int n2, double a0, double a1,
                            double a2, double* __restrict__ part) {
  const long N = (long)n0 * n1 * n2;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    const int i2 = (int)(t % n2);
    const int i1 = (int)((t / n2) % n1);
    const int i0 = (int)(t / ((long)n1 * n2));
    const double p = rho[t];
    acc[0] += vion[t] * p;
    if (use_h) acc[1] += vh[t] * p;
    acc[2] += cbrt(p) * p;
    acc[3] += (a0 * i0 / n0) * p;
    acc[4] += (a1 * i1 / n1) * p;
    acc[5] += (a2 * i2 / n2) * p;
  }
  block_sums<6>(acc, part);
}

// [0] sum kin |c|^2
__global__ void k_kin_sum(const double2* __restrict__ c, const double* __restrict__ kin, int npw, long n,
                          double* __restrict__ part) {
  double acc[1] = {0.0};
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double2 v = c[t];
    acc[0] += kin[t % npw] * (v.x * v.x + v.y * v.y);
  }
  block_sums<1>(acc, part);
}

__global__ void k_trace_real(const double2* __restrict__ M, int n, double* __restrict__ out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += M[i + (long)i * n].x;
    *out = t;
  }
}

cudaError_t energy_sums(const double* rho, const double* vion, const double* vh, int use_h, Grid3 g, const double* cell,
                        const double2* c, const double* kin, int npw, int ne, const double2* negM, double* part,
                        double* out8, cudaStream_t s) {
  const unsigned nb = nblk(g.N(), 256, 1024);
  k_grid_sums<<<nb, 256, 0, s>>>(rho, vion, vh, use_h, g.n0, g.n1, g.n2, cell[0], cell[1], cell[2], part); launched();
  k_finalize<<<1, 32, 0, s>>>(part, nb, 6, out8); launched();
  const long n = (long)npw * ne;
  const unsigned nb2 = nblk(n, 256, 1024);
  k_kin_sum<<<nb2, 256, 0, s>>>(c, kin, npw, n, part + 6 * 1024); launched();
  k_finalize<<<1, 32, 0, s>>>(part + 6 * 1024, nb2, 1, out8 + 6); launched();
  if (negM != nullptr) { k_trace_real<<<1, 32, 0, s>>>(negM, ne, out8 + 7); launched(); }
  return cudaGetLastError();
}

__global__ void k_hartree_factor(double* __restrict__ f, int n0, int n1, int n2, double a0, double a1, double a2) {
  const long N = (long)n0 * n1 * n2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    const int i2 = (int)(t % n2);
    const int i1 = (int)((t / n2) % n1);
    const int i0 = (int)(t / ((long)n1 * n2));
    const int m0 = i0 < (n0 + 1) / 2 ? i0 : i0 - n0;
    const int m1 = i1 < (n1 + 1) / 2 ? i1 : i1 - n1;
    const int m2 = i2 < (n2 + 1) / 2 ? i2 : i2 - n2;
    const double g0 = 2.0 * M_PI * m0 / a0, g1 = 2.0 * M_PI * m1 / a1, g2 = 2.0 * M_PI * m2 / a2;
    const double gg = g0 * g0 + g1 * g1 + g2 * g2;
    f[t] = gg > 0.0 ? 4.0 * M_PI / (gg * (double)N) : 0.0;
  }
}

cudaError_t hartree_factor(double* f, Grid3 g, const double* cell, cudaStream_t s) {
  k_hartree_factor<<<nblk(g.N(), 256), 256, 0, s>>>(f, g.n0, g.n1, g.n2, cell[0], cell[1], cell[2]); launched();
  return cudaGetLastError();
}

}  // namespace pt

namespace pt {

__global__ void k_axpy(double2 a, const double2* __restrict__ x, double2* __restrict__ y, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    const double2 v = x[t];
    double2 w = y[t];
    w.x += a.x * v.x - a.y * v.y;
    w.y += a.x * v.y + a.y * v.x;
    y[t] = w;
  }
}

cudaError_t axpy(double2 a, const double2* x, double2* y, long n, cudaStream_t s) {
  k_axpy<<<nblk(n, 256), 256, 0, s>>>(a, x, y, n); launched();
  return cudaGetLastError();
}

}  // namespace pt

namespace pt {

__global__ void k_diff_to_complex(const double* __restrict__ a, const double* __restrict__ b, double2* __restrict__ buf,
                                  long N) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x)
    buf[t] = make_double2(a[t] - b[t], 0.0);
}

__global__ void k_add_real(const double2* __restrict__ buf, double* __restrict__ a, long N) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x)
    a[t] += buf[t].x;
}

cudaError_t diff_to_complex(const double* a, const double* b, double2* buf, long N, cudaStream_t s) {
  k_diff_to_complex<<<nblk(N, 256), 256, 0, s>>>(a, b, buf, N); launched();
  return cudaGetLastError();
}

cudaError_t add_real(const double2* buf, double* a, long N, cudaStream_t s) {
  k_add_real<<<nblk(N, 256), 256, 0, s>>>(buf, a, N); launched();
  return cudaGetLastError();
}

// b |G|^2 / (|G|^2 + q0^2) / N  (Kerker weight with the inverse-FFT normalisation)
__global__ void k_kerker_factor(double* __restrict__ f, int n0, int n1, int n2, double a0, double a1, double a2,
                                double b, double q2) {
  const long N = (long)n0 * n1 * n2;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    const int i2 = (int)(t % n2);
    const int i1 = (int)((t / n2) % n1);
    const int i0 = (int)(t / ((long)n1 * n2));
    const int m0 = i0 < (n0 + 1) / 2 ? i0 : i0 - n0;
    const int m1 = i1 < (n1 + 1) / 2 ? i1 : i1 - n1;
    const int m2 = i2 < (n2 + 1) / 2 ? i2 : i2 - n2;
    const double g0 = 2.0 * M_PI * m0 / a0, g1 = 2.0 * M_PI * m1 / a1, g2 = 2.0 * M_PI * m2 / a2;
    const double gg = g0 * g0 + g1 * g1 + g2 * g2;
    f[t] = b * gg / (gg + q2) / (double)N;
  }
}

cudaError_t kerker_factor(double* f, Grid3 g, const double* cell, double b, double q0, cudaStream_t s) {
  k_kerker_factor<<<nblk(g.N(), 256), 256, 0, s>>>(f, g.n0, g.n1, g.n2, cell[0], cell[1], cell[2], b, q0 * q0);
  launched();
  return cudaGetLastError();
}

}  // namespace pt
