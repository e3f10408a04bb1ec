// Launchers of the element, node and vector kernels (all asynchronous on stream s).
#pragma once
#include <cuda_runtime.h>
#include "lh_internal.h"

namespace lh {

// kernels launched so far (all launchers add to it)
void count_launches(int n);
long long launches();
// write the constant-memory basis tables of the element kernels on the current device
// (once per device; the launchers also do it before their first launch there)
cudaError_t init_const_tables();
cudaError_t init_const_tables_explicit();

// element + assembly launchers (lh_kernels.cu); vectors use the layout of include/lh.h.
// ev2, if not NULL, is an event pair recorded around the element kernel only.
// rec, if not NULL, receives the linearisation record [NE][rec_len(dim)][NQ] (float)
cudaError_t launch_residual(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                            double* ev, double* blockmin, double* r, cudaEvent_t* ev2 = nullptr,
                            float* rec = nullptr);
// FP32 J.w from the linearisation record (float or double output).  err (device int, may be
// NULL): the pipelined form (elements of 64 points) ORs in kWaitErrPipe when a bounded wait
// on its record copy runs out (the element rows of that warp are then NaN).
constexpr int kWaitErrTc = 1, kWaitErrPipe = 2;
cudaError_t launch_jvp_rec_f32(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* dk,
                               float* ev, float* out, cudaEvent_t* ev2 = nullptr, int* err = nullptr);
cudaError_t launch_jvp_rec_f64out(const ElemParams& P, cudaStream_t s, const float* rec, double tau,
                                  const float* dk, float* ev, double* out, cudaEvent_t* ev2 = nullptr,
                                  int* err = nullptr);
// node-centric assembly of a float J.w from its element scratch (x rows from dk)
template <class TO>
cudaError_t launch_assemble_jvp(const ElemParams& P, cudaStream_t s, const float* dk, double tau, const float* ev,
                                TO* out);
// Tensor-core J.w from the linearisation record (lh_tc_jvp.cu): element contractions as
// tcgen05 MMAs, kind 0 = TF32, 1 = BF16 operands, FP32 accumulation; quadrature-point
// arithmetic in FP32.  err (device int) is set non-zero if a tensor-core wait timed out.
// Returns cudaErrorNotSupported for orders whose dense element operator does not fit in
// shared memory (3D k >= 3).
template <class TO>
cudaError_t launch_jvp_tc(const ElemParams& P, cudaStream_t s, int kind, const float* rec, double tau,
                          const float* dk, float* ev, TO* out, int* err, cudaEvent_t* ev2 = nullptr);
bool jvp_tc_supported(int dim, int k);
// process-wide poll limit of the tensor-core waits; returns the previous limit
unsigned set_tc_wait_polls(unsigned polls);
// halo of a box face (lh_halo.cu): mode 0 packs the dim velocity rows of the face nodes
// into dst[dim][face nodes]; mode 1 adds src into the free velocity rows of dst
long long halo_len(const ElemParams& P, int axis);
template <class T>
cudaError_t launch_halo(const ElemParams& P, cudaStream_t s, int face, int mode, const T* src, T* dst);
// diagonal of the velocity block dR_v/dk_v = M_V + tau dF.1/dw_v from the linearisation
// record [dim NV] (1 on fixed rows); ev: float element scratch of NE * dim * ND.  floor > 0
// clamps each free entry to at least floor * diag(M_V) (the preconditioner's use: the
// viscous tangent is not sign-definite); floor = 0 returns the diagonal itself
cudaError_t launch_jvv_diag(const ElemParams& P, cudaStream_t s, const float* rec, double tau, float* ev,
                            const double* dmv, double* out, double floor = 0.0);
// Taylor-Green L1 velocity error terms (2D), one per (element, quadrature point) (lh_diag.cu)
long long tg_error_terms(const ElemParams& P);
cudaError_t launch_tg_error(const ElemParams& P, cudaStream_t s, const double* u, double* out);
cudaError_t launch_jvp_f64(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const double* dk, double* ev, double* out, cudaEvent_t* ev2 = nullptr);
cudaError_t launch_jvp_f32(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                           const float* dk, float* ev, float* out, cudaEvent_t* ev2 = nullptr);
// FP32 transpose action from the linearisation record (float y and out)
cudaError_t launch_jtvp_rec_f32(const ElemParams& P, cudaStream_t s, const float* rec, double tau, const float* y,
                               float* ev, float* out, cudaEvent_t* ev2 = nullptr);
cudaError_t launch_jtvp(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                        const double* y, double* ev, double* out, cudaEvent_t* ev2 = nullptr);
cudaError_t launch_mass_h1(const ElemParams& P, cudaStream_t s, const double* f, double* ev, double* out,
                           cudaEvent_t* ev2 = nullptr);
cudaError_t launch_mass_l2(const ElemParams& P, cudaStream_t s, const double* g, double* out);
cudaError_t launch_dt_estimate(const ElemParams& P, cudaStream_t s, const double* u, double* blockmin);
cudaError_t launch_setup(const ElemParams& P, cudaStream_t s, double* ev, double* diag_mv, double* inv_me);
cudaError_t launch_initial_nodes(const ElemParams& P, cudaStream_t s, double* x0);
unsigned elem_grid(const ElemParams& P);

// vector kernels (lh_vec.cu).  Reductions are deterministic: a fixed partition of the
// index range (a function of n only) and fixed-order sums.
constexpr int kRedBlocks = 592;     // 4 x 148 SMs
constexpr int kRedThreads = 256;
// out_dev[j] = sum_i V[j*ld + i] * w[i] for j < m (w == NULL: plain sums of V_j), and
// out_dev[m] = w . w when with_self; one launch, deterministic.  partials: kRedBlocks *
// (m + 1) doubles (m + with_self <= 72); counter: a device unsigned that is 0 between calls.
// T = double or float (float: per-thread and warp sums in float, the rest in double).
template <class T>
cudaError_t launch_mdot(cudaStream_t s, const T* V, int m, long long ld, const T* w, long long n, int with_self,
                        double* partials, unsigned* counter, double* out_dev);
// out_dev[0] = min(v[0..n))
cudaError_t launch_min(cudaStream_t s, const double* v, long long n, double* out_dev);
// w -= sum_j h[j] V[j*ld + .]  (h: device doubles, m <= 64)
template <class T>
cudaError_t launch_gemv_sub(cudaStream_t s, const T* V, int m, long long ld, const double* h, T* w, long long n);
// second Gram-Schmidt pass fused with the normalisation: y = (w - V h) / hn, with
// hn^2 = h[m] - sum_{q<m} h[q]^2 (h[m] = w.w of the same multi-dot); y = 0 if hn^2 <= 0
template <class T>
cudaError_t launch_gemv_norm(cudaStream_t s, const T* V, int m, long long ld, const double* h, const T* w, T* y,
                             long long n);
// y = sum_j h[j] V[j*ld + .] + beta y  (h: device doubles, m <= 64)
template <class T>
cudaError_t launch_gemv(cudaStream_t s, const T* V, int m, long long ld, const double* h, double beta, T* y,
                        long long n);
// ---- device-side Arnoldi of the FP32-basis GMRES (one restart cycle per CUDA graph) ----
// State of one restart cycle in device memory.  The host writes the header and g[0] before
// the cycle and reads the whole struct after it.  H is the Hessenberg matrix after the
// Givens rotations, row-major with row stride kArnMax.
constexpr int kArnMax = 64;
struct ArnState {
  int j;             // columns built so far in this cycle (the next column to build)
  int stop;          // 0 running; 1 converged or breakdown; 3 restart length reached;
                     // 4 iteration budget reached; 5 non-finite Krylov vector
  int fix;           // this iteration needs the exact norm (the second pass still cancelled)
  int mres;          // restart length of the cycle (<= kArnMax)
  int maxit;         // iterations this cycle may take (the budget left)
  int pad_;
  double tol;        // stop when |g[j+1]| <= tol
  double hn2;        // squared norm of the projected vector (Pythagoras, or exact if fix)
  double g[kArnMax + 1], cs[kArnMax], sn[kArnMax];
  double H[(kArnMax + 1) * kArnMax];
};
// the multi-dot and updates above with the column count taken from the device (m = *jdev + 1)
// and an optional device gate (the launch does nothing unless *gate != 0); float4 forms only
// (n, ld multiples of 4, 16-byte aligned vectors)
cudaError_t launch_mdot_dev(cudaStream_t s, const float* V, const int* jdev, long long ld, const float* w, long long n,
                            int with_self, const int* gate, double* partials, unsigned* counter, double* out_dev);
cudaError_t launch_gemv_sub_dev(cudaStream_t s, const float* V, const int* jdev, long long ld, const double* h,
                                float* w, long long n, const int* gate);
// the first Gram-Schmidt update fused in front of the second multi-dot (float4 form):
// wout = w - V hsub (m columns, or *jdev + 1 when jdev is given), out_dev[q] = V_q . wout for
// q < m and out_dev[m] = wout . wout
cudaError_t launch_mdot_sub(cudaStream_t s, const float* V, int m, const int* jdev, long long ld, const float* w,
                            const double* hsub, float* wout, long long n, double* partials, unsigned* counter,
                            double* out_dev);
// v_{j+1} = V[(j+1) ld + .] = (w - V h) / hn as launch_gemv_norm (j = st->j), also copied to
// vin; stores hn^2 by Pythagoras (h: j + 1 coefficients and w.w at h[j + 1]) in st->hn2 and
// st->fix = 1 if it kept no more than 1e-4 of w.w (the exact norm is then taken), which it
// also sets as the conditional `fix` of the enclosing graph
cudaError_t launch_gemv_norm_dev(cudaStream_t s, float* V, ArnState* st, long long ld, const double* h,
                                 const float* w, float* vin, long long n, cudaGraphConditionalHandle fix);
// if st->fix: v_{j+1} = vin = w / sqrt(st->hn2) (st->hn2 then holds the exact w.w)
cudaError_t launch_arn_scale(cudaStream_t s, const ArnState* st, const float* w, float* V, long long ld, float* vin,
                             long long n);
// column j of H from the two passes' coefficients, the Givens rotations, the residual
// estimate |g[j+1]| and the stopping test; sets the WHILE condition of the enclosing graph
cudaError_t launch_arn_givens(cudaStream_t s, const double* h1, const double* h2, ArnState* st,
                              cudaGraphConditionalHandle cond);

// y = a x + b z  (z float, may be NULL)
template <class TX, class TY>
cudaError_t launch_scale(cudaStream_t s, double a, const TX* x, double b, const float* z, TY* y, long long n);
cudaError_t launch_axpby(cudaStream_t s, double a, const double* x, double b, double* y, long long n);
cudaError_t launch_scale_copy(cudaStream_t s, const double* x, const double* scale_dev, double* y, long long n);
// y = w * x elementwise (x may alias y)
template <class T>
cudaError_t launch_row_mul(cudaStream_t s, const double* w, const T* x, T* y, long long n);
// row weights of the scaled residual norm: 1 on x rows and fixed v rows, 1 / (M_V)_ii on
// free v rows, (M_E^-1)_ii on e rows
cudaError_t launch_row_weights(const ElemParams& P, cudaStream_t s, const double* diagMv, const double* invMe,
                               double* w);
cudaError_t launch_to_f32(cudaStream_t s, const double* x, float* y, long long n);
cudaError_t launch_to_f64(cudaStream_t s, const float* x, double* y, long long n);
// block upper-triangular preconditioner [I, tau M_V^-1, 0; 0, M_V^-1, 0; 0, 0, M_E^-1] with
// M_V^-1 = diagonal (kind 0) or exact Kronecker inverse (kind 1, lh_prec.cu), or the
// inverse of a per-dof velocity diagonal passed as diag_mv (kind 2: the diagonal of
// dR_v/dk_v, launch_jvv_diag); fixed velocity rows identity.  Instantiated for (double, double), (double, float), (float, float),
// (float, double) input/output types.
template <class TR, class TZ>
cudaError_t launch_prec(int kind, cudaStream_t s, const ElemParams& P, const KronPrec& K, const double* diag_mv,
                        const double* inv_me, const TR* r, TZ* z, double tau);
// Chebyshev pieces of preconditioner kind 3 (lh_prec.cu); state-shaped float vectors whose
// velocity rows [n1, 2 n1) are used; dv the per-dof velocity diagonal [n1]
template <class TR>
cudaError_t launch_cheb_init(cudaStream_t s, long long n1, const double* dv, const TR* r, float* res, float* d,
                             float* z, double inv_theta);
cudaError_t launch_cheb_dir(cudaStream_t s, long long n1, long long n, const float* d, float* w, double tau);
cudaError_t launch_cheb_step(cudaStream_t s, long long n1, const double* dv, const float* jw, float* res, float* d,
                             float* z, double c1, double c2);
template <class TR, class TZ>
cudaError_t launch_cheb_out(cudaStream_t s, long long n1, long long n, const double* ime, const TR* r, const float* z,
                            TZ* out, double tau);
cudaError_t launch_cheb_scale(cudaStream_t s, long long n1, const double* dv, const float* x, float* y);
// J.w with float arithmetic, float input and double output (inside the FP64 Krylov solver)
cudaError_t launch_jvp_f32_to_f64(const ElemParams& P, cudaStream_t s, const double* u, const double* k, double tau,
                                  const float* dk, float* ev, double* out, cudaEvent_t* ev2 = nullptr);
// z = r / diag (component-wise H1 Jacobi, dim*NV entries, diag has NV entries)
cudaError_t launch_jacobi_h1(cudaStream_t s, long long nv, int dim, const double* diag, const double* r, double* z);
cudaError_t launch_mul(cudaStream_t s, const double* a, const double* b, double* y, long long n);
cudaError_t launch_probe_fma(int prec, double* tflops);
// explicit path (lh_explicit.cu): F's point data S = alpha detJ sigma J^-T at state u
// ([NE][dim^2][NQ]), F.1 assembled into f1 [dim NV] (ev: element scratch NE dim ND),
// the Taylor-Green source rows into bsrc [NEd] (2D, if P.tg and bsrc), the per-block
// minimum of the explicit time-step estimate into blockmin (if not NULL); vm 0 = mu_imp,
// 1 = mu_exp.  launch_force_t: out [NEd] = F^T w (+ bsrc if not NULL) from the stored S.
cudaError_t launch_force(const ElemParams& P, cudaStream_t s, int vm, const ExpC& X, const double* u, double* Sq,
                         double* ev, double* f1, double* bsrc, double* blockmin);
cudaError_t launch_force_t(const ElemParams& P, cudaStream_t s, const double* Sq, const double* w, const double* bsrc,
                           double* out);
// dst = src (or 0 if src is NULL) on the fixed rows of a velocity array [dim NV]
cudaError_t launch_copy_fixed(const ElemParams& P, cudaStream_t s, const double* src, double* dst);

}  // namespace lh
