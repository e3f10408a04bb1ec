// Launchers of the element, node and vector kernels (all asynchronous on stream s).
#pragma once
#include <cuda_runtime.h>
#include "lh_internal.h"

namespace lh {

// element + assembly launchers (lh_kernels.cu); vectors use the layout of include/lh.h
cudaError_t launch_residual(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                            double* ev, double* blockmin, double* r);
cudaError_t launch_jvp_f64(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const double* dk, double* ev, double* out);
cudaError_t launch_jvp_f32(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const float* dk, float* ev, float* out);
cudaError_t launch_jtvp(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                        const double* y, double* ev, double* out);
cudaError_t launch_mass_h1(const ElemParams& P, cudaStream_t s, const double* f, double* ev, double* out);
cudaError_t launch_mass_l2(const ElemParams& P, cudaStream_t s, const double* g, double* out);
cudaError_t launch_dt_estimate(const ElemParams& P, cudaStream_t s, const double* u, double* blockmin);
cudaError_t launch_setup(const ElemParams& P, cudaStream_t s, double* ev, double* diag_mv, double* inv_me);
cudaError_t launch_initial_nodes(const ElemParams& P, cudaStream_t s, double* x0);
unsigned elem_grid(const ElemParams& P);

// vector kernels (lh_vec.cu).  Reductions are deterministic: a fixed partition of the
// index range (a function of n only) and fixed-order sums.
constexpr int kRedBlocks = 592;     // 4 x 148 SMs
constexpr int kRedThreads = 256;
// out_dev[j] = sum_i V[j*ld + i] * w[i] for j < m (w == NULL: plain sums);
// partials: kRedBlocks * m doubles
cudaError_t launch_mdot(cudaStream_t s, const double* V, int m, long long ld, const double* w, long long n,
                        double* partials, double* out_dev);
// out_dev[0] = min(v[0..n))
cudaError_t launch_min(cudaStream_t s, const double* v, long long n, double* out_dev);
// w -= sum_j h[j] V[j*ld + .]  (h on the device, m <= 64)
cudaError_t launch_gemv_sub(cudaStream_t s, const double* V, int m, long long ld, const double* h, double* w,
                            long long n);
// y = sum_j h[j] V[j*ld + .] + beta y  (h on the device)
cudaError_t launch_gemv(cudaStream_t s, const double* V, int m, long long ld, const double* h, double beta,
                        double* y, long long n);
cudaError_t launch_axpby(cudaStream_t s, double a, const double* x, double b, double* y, long long n);
cudaError_t launch_scale_copy(cudaStream_t s, const double* x, const double* scale_dev, double* y, long long n);
cudaError_t launch_to_f32(cudaStream_t s, const double* x, float* y, long long n);
cudaError_t launch_to_f64(cudaStream_t s, const float* x, double* y, long long n);
// block-diagonal preconditioner z = diag(I, diag(M_V)^-1 (identity on fixed rows), M_E^-1) r
cudaError_t launch_precond(cudaStream_t s, const ElemParams& P, const double* diag_mv, const double* inv_me,
                           const double* r, double* z);
// z = r / diag (component-wise H1 Jacobi, dim*NV entries, diag has NV entries)
cudaError_t launch_jacobi_h1(cudaStream_t s, long long nv, int dim, const double* diag, const double* r, double* z);
cudaError_t launch_mul(cudaStream_t s, const double* a, const double* b, double* y, long long n);
cudaError_t launch_probe_fma(int prec, double* tflops);

}  // namespace lh
