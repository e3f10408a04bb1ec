// Host-side internals shared by the C-ABI layer and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <string>
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
  double* d_scalar = nullptr;      // small device scalars
  double* d_diagMv = nullptr;      // diagonal of M_V [NV]
  double* d_invMe = nullptr;       // inverse of the (diagonal) L2 mass [NEd]
  double* d_blockmin = nullptr;    // per-block min detJ of the last residual
  long long nblocks_elem = 0;
  // Newton / GMRES workspace (allocated on first lh_newton_step)
  double* d_work = nullptr;
  long long work_len = 0;
  float* d_fwork = nullptr;        // FP32 J.w in/out buffers
  int restart_alloc = 0;
  std::string err;
};
