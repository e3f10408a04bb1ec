// Host-side internals shared by the C-ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>
#include "../../include/lh.h"

namespace lh {

// Everything an element or node kernel needs to know about the mesh, by value.
struct ElemParams {
  int dim, K;
  int n0, n1, n2;          // elements per direction (n2 = 1 in 2D)
  int N0, N1, N2;          // H1 lattice extents (N2 = 1 in 2D)
  long long NE, NV, NEd;   // elements, H1 nodes, L2 unknowns
  double lo[3], h[3];
  double detJ0;            // element Jacobian determinant of the undeformed box
  const double* rho0;      // device [NE]
  const double* gamma;     // device [NE]
  const double* tab;       // device 1D tables, layout in lh_kernels.cu (TabLayout)
  double h0, inv_hc, q1, q2, scoef, eps2;
  int visc, tg;
  unsigned bc;
  // float copies for the FP32 tangent kernels (no conversions on the FP64 pipe there)
  float fh0, finv_hc, fq1, fq2, fscoef, feps2, finv_detJ0;
  // double-word (hi, lo float pairs) copies of the mesh constants for the residual's point
  // kernel on the FP32 pipe: 1 / detJ0, h0, 1 / h_coarse, q1, q2, scoef, eps_e^2
  float dw_inv_detJ0[2], dw_h0[2], dw_inv_hc[2], dw_q1[2], dw_q2[2], dw_scoef[2], dw_eps2[2];
  const float* fmq0;       // device [NE]: rho0 detJ0
  const float* fgm1;       // device [NE]: gamma - 1
  const float* fggm1;      // device [NE]: gamma (gamma - 1)
};

// parameters of the original tensor viscosity mu_exp of the explicit path (lh_qp_exp.cuh);
// J0^-1 of the undeformed box is diag(1 / h_c)
struct ExpC {
  double l0, q1, q2;
  double inv_h[3];
  int vorticity;
};

// shared set-up helpers (lh_api.cu)
bool check_desc(const lh_mesh_desc* d, std::string* why);
void fill_params(const lh_mesh_desc& d, ElemParams* out);
std::vector<double> host_tables(int K);   // [B | G | Bl | w | zh | zl] for order K
lh_status set_global_error(lh_status st, const std::string& msg);   // for lh_last_error(NULL)

// floats per quadrature point in the linearisation record (lh_qp.cuh, lin_record): J^-1,
// grad v, 7 scalars of the stress and linearised viscosity chain (and the Taylor-Green
// source in 2D)
inline int rec_len(int dim) { return dim == 3 ? 25 : 18; }

// Device-driven Arnoldi of the FP32-basis GMRES (lh_api.cu): the CUDA graph of one restart
// cycle (a WHILE conditional node around one Arnoldi iteration) and what its recorded
// kernels depend on; it is recorded again when any of that changes.
struct ArnState;
struct ArnGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t cap = nullptr;      // private streams, used only to record the body and the
  cudaStream_t cap2 = nullptr;     // body of its IF node
  long long per_it = 0;            // kernel launches per iteration (for the launch counter)
  long long per_fix = 0;           // ... in the IF body of the exact-norm fallback
  bool off = false;                // a graph call failed once: the host loop from then on
  const void* V = nullptr;
  const void* w = nullptr;
  const void* z = nullptr;
  const void* wsc = nullptr;
  long long ld = 0, len = 0, n = 0;
  int pk = -9, tck = -9, mres = 0, cheb_degree = 0;
  double tau = 0.0, cheb_b = 0.0, cheb_ratio = 0.0;
  // operator kinds whose kernels have run once outside a recording (one-time set-up done)
  unsigned long long warm = 0;
};

// Kronecker factors of the H1 mass inverse (lh_prec.cu); device pointers owned by the mesh
struct KronPrec {
  float* At_free[3] = {nullptr, nullptr, nullptr};    // transposed 1D inverses, N_d x N_d
  float* At_fixed[3] = {nullptr, nullptr, nullptr};   // ... with the masked end rows removed
  double* scale = nullptr;                            // nodal rho0^(-1/2) [NV]
  float* work = nullptr;                              // 2 x dim x NV floats
};

// event-pair profiler of element-kernel launches (opt-in)
struct Prof {
  static constexpr int kMax = 2048;
  bool on = false;
  cudaEvent_t ev[2 * kMax] = {};
  int kind[kMax] = {};
  int n = 0;
  double ms[8] = {};
  long long cnt[8] = {};
};

}  // namespace lh

struct lh_mesh {
  lh_mesh_desc desc;
  lh::ElemParams P;
  cudaStream_t stream = nullptr;
  long long n = 0;           // unknowns
  long long NQ = 0;          // quadrature points
  // device buffers owned by the mesh
  double* d_rho0 = nullptr;
  double* d_gamma = nullptr;
  double* d_tab = nullptr;
  double* d_ev = nullptr;          // element scratch: NE * 2*dim * ND doubles
  double* d_part = nullptr;        // reduction partials
  unsigned* d_counter = nullptr;   // ticket counter of the fused reductions (0 between calls)
  double* d_scalar = nullptr;      // small device scalars
  double* d_diagMv = nullptr;      // diagonal of M_V [NV]
  double* d_invMe = nullptr;       // inverse of the (diagonal) L2 mass [NEd]
  double* d_blockmin = nullptr;    // per-block min detJ of the last residual
  long long nblocks_elem = 0;
  // Newton / GMRES workspace (allocated on first lh_newton_step)
  double* d_work = nullptr;
  long long work_len = 0;
  float* d_fwork = nullptr;        // FP32 Krylov basis and work vectors, leading dimension ldf
  long long ldf = 0;               // n rounded up to 64 floats (16-byte aligned, zero tails)
  float* d_fconst = nullptr;       // [3 NE] float rho0 detJ0, gamma - 1, gamma (gamma - 1)
  float* d_rec = nullptr;          // linearisation record [NE][rec_len][NQ] (lazily allocated)
  double* d_stage = nullptr;       // SDIRK stage increments k_1..k_3 and stage base state [4 n] (lazily)
  double* d_xwork = nullptr;       // explicit path work arrays (lazily, lh_api.cu XWork)
  double* d_adv = nullptr;         // lh_advance trial state u, k and the internal increment [3 n] (lazily)
  double* d_wscale = nullptr;      // row weights of the scaled Newton norm [n] (lazily)
  float* d_cheb = nullptr;         // Chebyshev work vectors of preconditioner kind 3 [5 ldf] (lazily)
  double cheb_b = 1.0, cheb_ratio = 20.0;   // Chebyshev interval [b / ratio, b] at the current iterate
  int cheb_degree = 3;
  double* d_jdiag = nullptr;       // diagonal of dR_v/dk_v for preconditioner kind 2 [dim NV] (lazily)
  const double* rec_u = nullptr;   // arguments of the last lh_linearize (for the LH_FP32_LIN check)
  const double* rec_k = nullptr;
  double rec_tau = 0.0;
  bool rec_valid = false;
  int restart_alloc = 0;
  lh::KronPrec kron;
  // device-driven Arnoldi: cycle state (device) and its pinned host copy, the operator
  // input v_j (FP32 [ldf]), and the recorded graph
  lh::ArnState* d_arn = nullptr;
  lh::ArnState* h_arn = nullptr;
  float* d_vin = nullptr;
  lh::ArnGraph arn;
  double* h_small = nullptr;       // pinned host scratch for the Newton loop's read-backs
  lh::Prof prof;
  std::string err;
};
