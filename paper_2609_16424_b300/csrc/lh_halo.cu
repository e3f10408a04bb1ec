// Halo exchange of a box decomposition (paper Sec. 2.2, Eq. (8) with the parallel
// prolongation P != I): the H1 rows of nodes on a shared face hold partial sums of the
// element contributions of each side, and the operator's value there is their sum (the
// P^T of the paper).  x rows (R_x = k_x - w_v), fixed rows (R_v = k_v) and the element-local
// L2 rows are complete on each side and are not exchanged.
#include "lh_internal.h"
#include "lh_kernels.h"

namespace lh {

namespace {

template <class T>
__global__ void k_halo(ElemParams P, int axis, int side, int mode, const T* __restrict__ src, T* __restrict__ dst) {
  const long long Nx[3] = {P.N0, P.N1, P.N2};
  const int dim = P.dim;
  const int a1 = axis == 0 ? 1 : 0;
  const int a2 = dim == 3 ? (axis == 2 ? 1 : 2) : -1;
  const long long nf = Nx[a1] * (a2 >= 0 ? Nx[a2] : 1);
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= dim * nf) return;
  const int c = (int)(t / nf);
  const long long i = t % nf;
  long long ic[3] = {0, 0, 0};
  ic[axis] = side ? Nx[axis] - 1 : 0;
  ic[a1] = i % Nx[a1];
  if (a2 >= 0) ic[a2] = i / Nx[a1];
  const long long nd = ic[0] + P.N0 * (ic[1] + P.N1 * ic[2]);
  const long long row = (long long)(dim + c) * P.NV + nd;
  if (mode == 0) {
    dst[t] = src[row];
    return;
  }
  // v_c fixed on a masked face of this mesh: the row is R_v = k_v on both sides
  const bool lo = ((P.bc >> (2 * c)) & 1u) && ic[c] == 0;
  const bool hi = ((P.bc >> (2 * c + 1)) & 1u) && ic[c] == Nx[c] - 1;
  if (!(lo || hi)) dst[row] += src[t];
}

}  // namespace

long long halo_len(const ElemParams& P, int axis) {
  const long long Nx[3] = {P.N0, P.N1, P.N2};
  long long nf = 1;
  for (int a = 0; a < P.dim; ++a)
    if (a != axis) nf *= Nx[a];
  return P.dim * nf;
}

template <class T>
cudaError_t launch_halo(const ElemParams& P, cudaStream_t s, int face, int mode, const T* src, T* dst) {
  const int axis = face / 2, side = face % 2;
  const long long n = halo_len(P, axis);
  count_launches(1);
  k_halo<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, axis, side, mode, src, dst);
  return cudaGetLastError();
}

template cudaError_t launch_halo<double>(const ElemParams&, cudaStream_t, int, int, const double*, double*);
template cudaError_t launch_halo<float>(const ElemParams&, cudaStream_t, int, int, const float*, float*);

}  // namespace lh
