// Declarations shared by the library's translation units (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <cstddef>
#include <string>
#include <atomic>

namespace pt {

// Supported FFT lengths and the offset of each length's twiddle table.
constexpr int kNumLengths = 8;
constexpr int kLengths[kNumLengths] = {8, 12, 16, 24, 32, 48, 64, 96};
constexpr int kTwiddleTotal = 8 + 12 + 16 + 24 + 32 + 48 + 64 + 96;
int twiddle_offset(int L);   // -1 if unsupported
void twiddle_host(double2* out);   // all tables, exp(-2 pi i t / L)

struct Grid3 {
  int n0, n1, n2;
  long N() const { return (long)n0 * n1 * n2; }
};

// Twiddle tables resident on the device (per precision).
struct DevTwiddles {
  const double2* d64;
  const float2* d32;
  template <typename T> const void* base() const;
};

// ---- generic batched 3D transforms (fft3d.cu) -----------------------------
// Volumes are [v][i0][i1][i2] (axis 2 fastest), `nvol` of them, in place.
// dir: +1 inverse (exp(+i...)), -1 forward. Scale applied at the end of the pass.
template <typename T>
cudaError_t fft_rows(const void* in, void* out, long nvol, Grid3 g, int inverse, double scale,
                     const T* mul_real, const DevTwiddles& tw, cudaStream_t s);
// axis in {0, 1}. mode 0: one transform; mode 1 (axis 0 only): inverse, multiply
// by mul_real (natural layout), forward; mode 2 (axis 0 only): forward,
// multiply by mul_real, inverse.
template <typename T>
cudaError_t fft_cols(void* data, long nvol, Grid3 g, int axis, int inverse, int mode, double scale,
                     const T* mul_real, const DevTwiddles& tw, cudaStream_t s);
// out[v][basis[k]] = scale * in[v][k] (in: complex128 coefficients), zero elsewhere.
template <typename T>
cudaError_t scatter_basis(const double2* in, long in_ld, void* out, long nvol, Grid3 g, const int* basis,
                          int npw, double scale, cudaStream_t s);
// out[v][k] = kin_scale * kin[k] * x[v][k] + scale * in[v][basis[k]] (+ out if accumulate)
template <typename T>
cudaError_t gather_basis(const void* in, double2* out, long out_ld, long nvol, Grid3 g, const int* basis,
                         int npw, double scale, const double* kin, const double2* x, long x_ld, int accumulate,
                         cudaStream_t s);
cudaError_t convert_c128_to_c64(const double2* in, float2* out, long n, cudaStream_t s);

// ---- sphere-pruned FP32 transforms for cubic 32/64/96 grids (fft_sphere.cu) --
// Device tables of the basis sphere. Live rows are the (i0, i1) with at least
// one basis vector, in increasing flat order; their basis vectors are the
// contiguous range [row_kbeg[r], row_kbeg[r + 1]) of the basis listing.
struct SphereTables {
  int nrows;
  const int* row_idx;             // i0 * L + i1 of live row r
  const int* row_kbeg;            // nrows + 1 entries
  const int* krow;                // live-row ordinal of basis vector k
  const unsigned char* rowlive;   // L * L flags, (i0, i1)
  int nplanes;
  const int* planes;              // live i0 values
  const unsigned char* planelive; // L flags
};
bool sphere_fast_supported(Grid3 g);
// vol[v] = sum_k coef[v][k] * scale * exp(+i G_k r) on the grid (complex64 or complex128 volumes).
cudaError_t sphere_to_real(const double2* coef, long ldc, float2* vol, long nvol, Grid3 g, const SphereTables& st,
                           const int* basis, double scale, const float2* tw_L, cudaStream_t s);
cudaError_t sphere_to_real(const double2* coef, long ldc, double2* vol, long nvol, Grid3 g, const SphereTables& st,
                           const int* basis, double scale, const double2* tw_L, cudaStream_t s);
// out[v][k] = scale * F[mul * vol[v]](G_k) (+ kin[k] x[v][k]) (+ out[v][k] if accumulate),
// F the forward transform; mul may be null; `work` (nvol volumes) may be `vol`.
cudaError_t sphere_from_real(const float2* vol, const float* mul, float2* work, long nvol, Grid3 g,
                             const SphereTables& st, const int* basis, double scale, const double* kin,
                             const double2* x, long ldx, double2* out, long ldo, int accumulate, const float2* tw_L,
                             cudaStream_t s);
cudaError_t sphere_from_real(const double2* vol, const double* mul, double2* work, long nvol, Grid3 g,
                             const SphereTables& st, const int* basis, double scale, const double* kin,
                             const double2* x, long ldx, double2* out, long ldo, int accumulate, const double2* tw_L,
                             cudaStream_t s);

// ---- Fock exchange pair pipeline (fock.cu) ----------------------------------
constexpr int kTileMax = 4;
struct PairTile {
  // device addresses of the real-space rows of slot o (exchange precision) and of its
  // accumulator (when is_out[o]); set by fock_bind_tiles, so the tiles of one launch
  // group may belong to different systems
  const void* in[2 * kTileMax];
  void* out[2 * kTileMax];
  int n_orb;
  int n_pairs;
  int orb[2 * kTileMax];
  signed char src[2 * kTileMax];     // 0: occupied orbitals, 1: X columns
  signed char is_out[2 * kTileMax];  // accumulate into this orbital's W
  signed char pi[kTileMax * kTileMax];
  signed char pj[kTileMax * kTileMax];
  // contributions to each output orbital: pair index, the other orbital's
  // slot, and whether the pair potential enters conjugated (i side of a
  // symmetric pair). At most kTileMax per output.
  signed char out_n[2 * kTileMax];
  signed char out_pair[2 * kTileMax][kTileMax];
  signed char out_other[2 * kTileMax][kTileMax];
  signed char out_conj[2 * kTileMax][kTileMax];
};

struct FockPlan {
  int tile;               // orbitals per tile edge
  int tiles_per_launch;   // cap on tiles in one pass triple
  // launches: [first_tile, count) ranges into the device tile array
  int n_launch;
  int* launch_first;      // host arrays
  int* launch_count;
  PairTile* d_tiles;      // device
  int n_tiles;
  // Largest |G2| (frequency index along axis 2) a pair product can reach: twice
  // the largest |g2| of the basis. Products of band-limited orbitals vanish
  // exactly beyond it on an alias-free grid, so the fast path skips those
  // axis-2 slabs. A value >= n2 / 2 disables the skip.
  int g2_reach;
};

// The pair kernels of `plan` (tiles bound to their orbitals and accumulators).
template <typename T>
cudaError_t fock_pairs(const FockPlan& plan, int sym, Grid3 g, const T* khat_t, void* scratch, const DevTwiddles& tw,
                       cudaStream_t s);
// FP32 cubic fast path (fock_fast.cu): n0 == n1 == n2 in {32, 48, 64, 96}.
bool fock_fast_supported(Grid3 g);
cudaError_t fock_pairs_fast(const FockPlan& plan, Grid3 g, const float* khat_t, void* scratch, const float2* tw_L,
                            cudaStream_t s);
// Sets in[] / out[] of host tiles from their orbital slots: slot o reads
// (src 0 ? psi_r : x_r) + orb * N and accumulates into (src 0 ? w_occ : w_x) + orb * N,
// N complex values of `cs` bytes per orbital.
void fock_bind_tiles(PairTile* tiles, int n, const void* psi_r, const void* x_r, void* w_occ, void* w_x, long N,
                     size_t cs);
// Host tile schedules. sym: pairs i <= j of n_occ orbitals; otherwise n_occ x n_x pairs.
int fock_build_tiles(int n_occ, int n_x, int tile, int sym, int tiles_per_launch, PairTile** tiles_out,
                     int** launch_first, int** launch_count, int* n_launch);

// ---- dense linear algebra (linalg.cu) -------------------------------------
// C(M x N) = alpha * op(A) op(B) + beta * C, complex, column-major, batched by strides.
// A element (i, k) of op(A) == N: A[i + k * lda]; == H: conj(A[k + i * lda]).
// Inputs stored as complex128; Tc is the compute / accumulate precision.
// structure: GEMM_HERM for C = A^H A (only the lower half is computed, the upper
// half is its conjugate mirror); GEMM_TRI_B when op(B) is upper triangular.
enum { OP_N = 0, OP_H = 1 };
enum { GEMM_GENERAL = 0, GEMM_HERM = 1, GEMM_TRI_B = 2 };
template <typename Tc>
cudaError_t gemm(int opA, int opB, int M, int N, int K, double2 alpha, const double2* A, long lda, long strideA,
                 const double2* B, long ldb, long strideB, double2 beta, double2* C, long ldc, long strideC,
                 int batch, double2* splitk_ws, size_t splitk_ws_elems, cudaStream_t s,
                 int structure = GEMM_GENERAL);
// The same product from complex64 copies of A and B on the tensor cores (gemm_tc.cu):
// 3xTF32 with FP32 accumulation, C complex128; GEMM_GENERAL or GEMM_TRI_B. `d_err`
// (device int) gets bit 0 set when a bounded wait inside the kernel expires.
cudaError_t gemm_tc(int opA, int opB, int M, int N, int K, double2 alpha, const float2* A, long lda, const float2* B,
                    long ldb, double2 beta, double2* C, long ldc, double2* splitk_ws, size_t splitk_ws_elems,
                    int* d_err, cudaStream_t s, int structure = GEMM_GENERAL);
// C = alpha sum_kz part[kz] + beta C over ksplit partials part[(kz N + j) M + i], fixed order.
cudaError_t splitk_reduce(int M, int N, int ksplit, double2 alpha, const double2* part, double2 beta, double2* C,
                          long ldc, cudaStream_t s);
// In-place lower Cholesky of an n x n Hermitian matrix (column-major, lower
// triangle used and overwritten, upper set to 0). *d_status = 1 on a
// non-positive pivot.
cudaError_t cholesky(double2* A, int n, int* d_status, cudaStream_t s);
// Linv = L^{-1} for lower-triangular L (n x n, column-major).
cudaError_t tri_inverse(const double2* L, double2* Linv, int n, cudaStream_t s);

std::string cuda_msg(cudaError_t e);

// One-time per-device setup (kernel attributes, occupancy queries): bit d of `mask`
// records that device d (d < 64) is done. Returns the current device's bit, or 0
// when the setup is already done for it.
inline unsigned long long device_bit_todo(const std::atomic<unsigned long long>& mask) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const unsigned long long bit = 1ull << (dev & 63);
  return (mask.load(std::memory_order_acquire) & bit) ? 0ull : bit;
}

// Count of kernels this library has launched (all systems, this process).
void launched(int n = 1);
unsigned long long launch_count();

}  // namespace pt
