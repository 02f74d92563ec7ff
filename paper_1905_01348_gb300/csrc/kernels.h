// Host launchers of the elementwise / reduction kernels (kernels.cu).
#pragma once

#include <cuda_runtime.h>
#include "internal.h"

namespace pt {

constexpr int kSlotMax = 24;   // Anderson history slots a kernel accepts
struct SlotList {
  int k;                       // valid entries
  int s[kSlotMax];             // history slots, oldest first
};

cudaError_t density(const double2* psi_r, long N, int ne, double* rho, cudaStream_t s);
cudaError_t density32(const float2* psi_r, long N, int ne, double* rho, cudaStream_t s);
cudaError_t to_float(const double* a, float* b, long n, cudaStream_t s);
cudaError_t rho_to_complex(const double* rho, double2* buf, long N, cudaStream_t s);
cudaError_t assemble_vloc(const double* vion, const double2* vh_c, const double* rho, long N, int use_h, double w_lda,
                          double* vh, double* vloc, cudaStream_t s);
cudaError_t ion_potential(double* v, Grid3 g, const double* cell, const double* d_atoms, int na, double depth,
                          double sigma, cudaStream_t s);
cudaError_t hartree_factor(double* f, Grid3 g, const double* cell, cudaStream_t s);
cudaError_t half_step(const double2* psi, const double2* R, double hdt, double2* out, long n, cudaStream_t s);
cudaError_t pt_residual(const double2* psi_f, const double2* T, const double2* ph, double hdt, double2* r, long n,
                        double* part, double* out_norm2, cudaStream_t s);
cudaError_t precond_step(double2* x, const double2* R, const double* kin, int npw, long n, double tau, cudaStream_t s);
cudaError_t anderson_push(const double2* x, const double2* r, double2* xp, double2* rp, void* dx, void* dr, long n,
                          int have_prev, int f32, cudaStream_t s);
cudaError_t anderson_dots(const void* dR, long slot_stride, const SlotList& sl, int newslot, const double2* r,
                          int npw, int ne, int mdim, double2* gram, double2* rhs, int f32, cudaStream_t s);
cudaError_t anderson_solve(const double2* gram, const double2* rhs, const SlotList& sl, int mdim, int ne,
                           double2* gamma, cudaStream_t s);
cudaError_t anderson_update(double2* x, const double2* r, const void* dX, const void* dR, long slot_stride,
                            const SlotList& sl, const double2* gamma, int mdim, int npw, long n, double beta, int f32,
                            cudaStream_t s);
cudaError_t kinetic_shifted(const double* gk3, int npw, double ax, double ay, double az, double* kin, cudaStream_t s);
cudaError_t rho_change(const double* a, const double* b, long N, double* part, double* out, cudaStream_t s);
// out8: [0] sum vion rho, [1] sum vh rho, [2] sum rho^{4/3}, [3..5] sum r rho,
//       [6] sum kin |c|^2, [7] Re tr(negM)   (grid sums without the dV factor)
cudaError_t energy_sums(const double* rho, const double* vion, const double* vh, int use_h, Grid3 g, const double* cell,
                        const double2* c, const double* kin, int npw, int ne, const double2* negM, double* part,
                        double* out8, cudaStream_t s);
cudaError_t axpy(double2 a, const double2* x, double2* y, long n, cudaStream_t s);
cudaError_t diff_to_complex(const double* a, const double* b, double2* buf, long N, cudaStream_t s);
cudaError_t add_real(const double2* buf, double* a, long N, cudaStream_t s);
cudaError_t kerker_factor(double* f, Grid3 g, const double* cell, double b, double q0, cudaStream_t s);

}  // namespace pt
