// Transforms (FP32 or FP64) between the planewave sphere and the real-space grid for
// cubic grids of 32, 48, 64 or 96 points (the orbital transforms of the SCF loop,
// Sec. 3.2 and 3.4: real-space orbitals for the density and exchange, and the
// local-potential product of Eq. 2).
//
// The basis is the sphere |G|^2/2 <= ecut, a small part of the grid's
// frequency cube (about 6% at the workloads' cutoff). A 3D transform from the
// sphere therefore starts with few nonzero lines and only the last axis is
// full, and a transform to the sphere needs few outputs after its first axis:
//   to real space:  rows (axis 2) only for the live (i0, i1) rows, the basis
//                   coefficients scattered straight into them; axis 1 only on
//                   the live i0 planes, reading only their live rows; axis 0
//                   on every line, reading only the live planes.
//   to the sphere:  axis 0 on every line (the real-space product with the
//                   local potential fused into the load), storing only the
//                   live planes; axis 1 on the live planes, storing only the
//                   live rows; axis 2 on the live rows, gathering the basis
//                   coefficients straight from them.
// Rows and planes that no basis vector reaches are never read or written, so
// a pass never depends on what they hold. The transforms are exact: the
// skipped inputs are zero and the skipped outputs are not needed.
#include "common.cuh"
#include "fft_ct.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr int SNT = 64;   // threads per block
constexpr int SC = 16;    // lines (rows, or i2 columns) per block
constexpr int SW = SC + 1;

template <int L> constexpr int RW = L + 1;   // row stride of the row kernels

// Row kernels: SC live rows per block, rows of length L at stride L + 1.
template <typename C, int L> constexpr size_t smem_rows() { return sizeof(C) * (size_t)(L + SC * RW<L>); }
// Column kernels: an L x SC block (element e of column c at e * (SC + 1) + c).
template <typename C, int L> constexpr size_t smem_cols() { return sizeof(C) * (size_t)(L + L * SW); }

template <typename C> __device__ __forceinline__ C scaled(double2 a, double s) { return cvt<C>(make_double2(a.x * s, a.y * s)); }

// Inverse along axis 2 of SC live rows, the row's basis coefficients scattered in.
template <typename C, int L>
__global__ void __launch_bounds__(SNT) k_sph_rows_inv(const double2* __restrict__ coef, long ldc,
                                                      C* __restrict__ vol, const SphereTables st,
                                                      const int* __restrict__ basis, double scale,
                                                      const C* __restrict__ tw_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * SC;
  const int nr = min(SC, st.nrows - r0);
  const long v = blockIdx.y;
  for (int t = tid; t < L; t += SNT) tw[t] = tw_g[t];
  for (int e = tid; e < SC * RW<L>; e += SNT) buf[e] = C{};
  __syncthreads();
  const int k0 = st.row_kbeg[r0], k1 = st.row_kbeg[r0 + nr];
  const double2* cv = coef + v * ldc;
  for (int k = k0 + tid; k < k1; k += SNT)
    buf[(st.krow[k] - r0) * RW<L> + basis[k] % L] = scaled<C>(cv[k], scale);
  __syncthreads();
  ct_inverse<C, L, SC, SNT, RW<L>, 1>(buf, nr, tw, tid);
  C* vv = vol + v * (long)L * L * L;
  for (int e = tid; e < nr * L; e += SNT) {
    const int rr = e / L, i2 = e % L;
    vv[(long)st.row_idx[r0 + rr] * L + i2] = buf[rr * RW<L> + i2];
  }
}

// Axis-1 transform of one live plane i0 over SC columns i2. INV: reads only the
// plane's live rows (others are zero), writes the whole plane block. Forward:
// reads the whole plane block, writes only the live rows.
template <typename C, int L, bool INV>
__global__ void __launch_bounds__(SNT) k_sph_axis1(C* __restrict__ vol, const SphereTables st,
                                                   const C* __restrict__ tw_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x;
  const int i2s = blockIdx.x * SC;
  const int i0 = st.planes[blockIdx.y];
  const long v = blockIdx.z;
  for (int t = tid; t < L; t += SNT) tw[t] = tw_g[t];
  C* base = vol + v * (long)L * L * L + (long)i0 * L * L + i2s;
  const unsigned char* live = st.rowlive + i0 * L;
  for (int idx = tid; idx < L * SC; idx += SNT) {
    const int i1 = idx / SC, c = idx % SC;
    buf[i1 * SW + c] = (!INV || live[i1]) ? base[(long)i1 * L + c] : C{};
  }
  __syncthreads();
  if (INV) ct_inverse<C, L, SC, SNT, 1, SW>(buf, SC, tw, tid);
  else ct_forward<C, L, SC, SNT, 1, SW>(buf, SC, tw, tid);
  for (int idx = tid; idx < L * SC; idx += SNT) {
    const int i1 = idx / SC, c = idx % SC;
    if (INV || live[i1]) base[(long)i1 * L + c] = buf[i1 * SW + c];
  }
}

// Axis-0 transform of the lines (i1, i2s..i2s+SC). INV: reads only the live
// planes, writes every plane. Forward: reads every plane (times the real field
// `mul` when given), writes only the live planes. `dst` may be `src`: a block
// reads all of its lines before it writes them.
template <typename C, int L, bool INV>
__global__ void __launch_bounds__(SNT) k_sph_axis0(const C* src, C* dst, const typename real_of<C>::type* __restrict__ mul,
                                                   const SphereTables st, const C* __restrict__ tw_g) {
  using R = typename real_of<C>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x;
  const int i2s = blockIdx.x * SC;
  const int i1 = blockIdx.y;
  const long v = blockIdx.z;
  for (int t = tid; t < L; t += SNT) tw[t] = tw_g[t];
  const long off = (long)i1 * L + i2s;
  const C* sb = src + v * (long)L * L * L + off;
  C* db = dst + v * (long)L * L * L + off;
  for (int idx = tid; idx < L * SC; idx += SNT) {
    const int i0 = idx / SC, c = idx % SC;
    C x{};
    if (!INV || st.planelive[i0]) {
      x = sb[(long)i0 * L * L + c];
      if (!INV && mul != nullptr) x = cscale(x, (R)__ldg(mul + (long)i0 * L * L + off + c));
    }
    buf[i0 * SW + c] = x;
  }
  __syncthreads();
  if (INV) ct_inverse<C, L, SC, SNT, 1, SW>(buf, SC, tw, tid);
  else ct_forward<C, L, SC, SNT, 1, SW>(buf, SC, tw, tid);
  for (int idx = tid; idx < L * SC; idx += SNT) {
    const int i0 = idx / SC, c = idx % SC;
    if (INV || st.planelive[i0]) db[(long)i0 * L * L + c] = buf[i0 * SW + c];
  }
}

// Forward along axis 2 of SC live rows, then out[k] = scale * F[k]
// (+ kin[k] x[k]) (+ out[k]) for the rows' basis vectors.
template <typename C, int L>
__global__ void __launch_bounds__(SNT) k_sph_rows_fwd(const C* __restrict__ vol, const SphereTables st,
                                                      const int* __restrict__ basis, double scale,
                                                      const double* __restrict__ kin, const double2* __restrict__ x,
                                                      long ldx, double2* __restrict__ out, long ldo, int accumulate,
                                                      const C* __restrict__ tw_g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* buf = tw + L;
  const int tid = threadIdx.x;
  const int r0 = blockIdx.x * SC;
  const int nr = min(SC, st.nrows - r0);
  const long v = blockIdx.y;
  for (int t = tid; t < L; t += SNT) tw[t] = tw_g[t];
  const C* vv = vol + v * (long)L * L * L;
  for (int e = tid; e < nr * L; e += SNT) {
    const int rr = e / L, i2 = e % L;
    buf[rr * RW<L> + i2] = vv[(long)st.row_idx[r0 + rr] * L + i2];
  }
  __syncthreads();
  ct_forward<C, L, SC, SNT, RW<L>, 1>(buf, nr, tw, tid);
  const int k0 = st.row_kbeg[r0], k1 = st.row_kbeg[r0 + nr];
  double2* ov = out + v * ldo;
  const double2* xv = x != nullptr ? x + v * ldx : nullptr;
  for (int k = k0 + tid; k < k1; k += SNT) {
    const double2 f = to_d(buf[(st.krow[k] - r0) * RW<L> + basis[k] % L]);
    double2 r = make_double2(f.x * scale, f.y * scale);
    if (kin != nullptr) {
      const double2 c = xv[k];
      r.x += kin[k] * c.x;
      r.y += kin[k] * c.y;
    }
    if (accumulate) {
      const double2 o = ov[k];
      r.x += o.x;
      r.y += o.y;
    }
    ov[k] = r;
  }
}

template <typename C, int L>
cudaError_t to_real_t(const double2* coef, long ldc, C* vol, long nvol, const SphereTables& st, const int* basis,
                      double scale, const C* tw, cudaStream_t s) {
  if (st.nrows == 0) return cudaMemsetAsync(vol, 0, sizeof(C) * (size_t)L * L * L * nvol, s);
  const dim3 gr((unsigned)((st.nrows + SC - 1) / SC), (unsigned)nvol);
  k_sph_rows_inv<C, L><<<gr, SNT, smem_rows<C, L>(), s>>>(coef, ldc, vol, st, basis, scale, tw);
  const dim3 g1((unsigned)(L / SC), (unsigned)st.nplanes, (unsigned)nvol);
  k_sph_axis1<C, L, true><<<g1, SNT, smem_cols<C, L>(), s>>>(vol, st, tw);
  const dim3 g0((unsigned)(L / SC), (unsigned)L, (unsigned)nvol);
  k_sph_axis0<C, L, true><<<g0, SNT, smem_cols<C, L>(), s>>>(vol, vol, nullptr, st, tw);
  launched(3);
  return cudaGetLastError();
}

template <typename C, int L>
cudaError_t to_sphere_t(const C* vol, const typename real_of<C>::type* mul, C* work, long nvol,
                        const SphereTables& st, const int* basis, double scale, const double* kin, const double2* x,
                        long ldx, double2* out, long ldo, int accumulate, const C* tw, cudaStream_t s) {
  if (st.nrows == 0) return cudaSuccess;
  const dim3 g0((unsigned)(L / SC), (unsigned)L, (unsigned)nvol);
  k_sph_axis0<C, L, false><<<g0, SNT, smem_cols<C, L>(), s>>>(vol, work, mul, st, tw);
  const dim3 g1((unsigned)(L / SC), (unsigned)st.nplanes, (unsigned)nvol);
  k_sph_axis1<C, L, false><<<g1, SNT, smem_cols<C, L>(), s>>>(work, st, tw);
  const dim3 gr((unsigned)((st.nrows + SC - 1) / SC), (unsigned)nvol);
  k_sph_rows_fwd<C, L><<<gr, SNT, smem_rows<C, L>(), s>>>(work, st, basis, scale, kin, x, ldx, out, ldo, accumulate,
                                                          tw);
  launched(3);
  return cudaGetLastError();
}

}  // namespace

bool sphere_fast_supported(Grid3 g) {
  return g.n0 == g.n1 && g.n1 == g.n2 && (g.n0 == 32 || g.n0 == 48 || g.n0 == 64 || g.n0 == 96);
}

template <typename C>
static cudaError_t to_real_any(const double2* coef, long ldc, C* vol, long nvol, Grid3 g, const SphereTables& st,
                               const int* basis, double scale, const C* tw_L, cudaStream_t s) {
  if (nvol <= 0) return cudaSuccess;
  if (nvol > 65535) return cudaErrorInvalidValue;
  switch (g.n0) {
    case 32: return to_real_t<C, 32>(coef, ldc, vol, nvol, st, basis, scale, tw_L, s);
    case 48: return to_real_t<C, 48>(coef, ldc, vol, nvol, st, basis, scale, tw_L, s);
    case 64: return to_real_t<C, 64>(coef, ldc, vol, nvol, st, basis, scale, tw_L, s);
    case 96: return to_real_t<C, 96>(coef, ldc, vol, nvol, st, basis, scale, tw_L, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename C>
static cudaError_t from_real_any(const C* vol, const typename real_of<C>::type* mul, C* work, long nvol, Grid3 g,
                                 const SphereTables& st, const int* basis, double scale, const double* kin,
                                 const double2* x, long ldx, double2* out, long ldo, int accumulate, const C* tw_L,
                                 cudaStream_t s) {
  if (nvol <= 0) return cudaSuccess;
  if (nvol > 65535) return cudaErrorInvalidValue;
  switch (g.n0) {
    case 32: return to_sphere_t<C, 32>(vol, mul, work, nvol, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
    case 48: return to_sphere_t<C, 48>(vol, mul, work, nvol, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
    case 64: return to_sphere_t<C, 64>(vol, mul, work, nvol, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
    case 96: return to_sphere_t<C, 96>(vol, mul, work, nvol, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t sphere_to_real(const double2* coef, long ldc, float2* vol, long nvol, Grid3 g, const SphereTables& st,
                           const int* basis, double scale, const float2* tw_L, cudaStream_t s) {
  return to_real_any(coef, ldc, vol, nvol, g, st, basis, scale, tw_L, s);
}
cudaError_t sphere_to_real(const double2* coef, long ldc, double2* vol, long nvol, Grid3 g, const SphereTables& st,
                           const int* basis, double scale, const double2* tw_L, cudaStream_t s) {
  return to_real_any(coef, ldc, vol, nvol, g, st, basis, scale, tw_L, s);
}
cudaError_t sphere_from_real(const float2* vol, const float* mul, float2* work, long nvol, Grid3 g,
                             const SphereTables& st, const int* basis, double scale, const double* kin,
                             const double2* x, long ldx, double2* out, long ldo, int accumulate, const float2* tw_L,
                             cudaStream_t s) {
  return from_real_any(vol, mul, work, nvol, g, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
}
cudaError_t sphere_from_real(const double2* vol, const double* mul, double2* work, long nvol, Grid3 g,
                             const SphereTables& st, const int* basis, double scale, const double* kin,
                             const double2* x, long ldx, double2* out, long ldo, int accumulate, const double2* tw_L,
                             cudaStream_t s) {
  return from_real_any(vol, mul, work, nvol, g, st, basis, scale, kin, x, ldx, out, ldo, accumulate, tw_L, s);
}

}  // namespace pt
