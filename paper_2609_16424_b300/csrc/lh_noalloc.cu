// Stage residual that allocates no device memory.
//
// For callers that must not allocate device memory when they call the library: for
// example code embedded in a host application that owns all device memory through its
// own pool and forbids other allocations, or latency-critical loops that cannot accept
// the implicit synchronisation of cudaMalloc.  Such a caller passes every input and
// output; the element scratch the residual needs lives in file-scope __device__ arrays
// of fixed size that every GPU loading this library holds until the process exits.
#include <mutex>
#include <string>
#include "lh_internal.h"
#include "lh_kernels.h"

namespace {

constexpr long long kEvMax = 2LL * 1024 * 1024;   // element scratch, doubles (16 MiB)
constexpr long long kBlocksMax = 64LL * 1024;     // per-block det J minima, doubles (512 KiB)
constexpr int kTabMax = 256;                      // 1D bases and weights of one order (order 4 needs 129)
constexpr int kOrders = 4;                        // orders 1..4, one table row each

__device__ __align__(256) double g_ev[kEvMax];
__device__ __align__(256) double g_blockmin[kBlocksMax];
__device__ __align__(256) double g_tab[kOrders * kTabMax];

// device addresses of the arrays above, looked up once per device
struct DevAddr {
  bool ready = false;
  double* ev = nullptr;
  double* blockmin = nullptr;
  double* tab = nullptr;   // kOrders rows of kTabMax entries, filled at set-up
};
constexpr int kMaxDevices = 64;
DevAddr g_addr[kMaxDevices];
std::mutex g_mu;

lh_status device_addresses(DevAddr* out, std::string* why) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    *why = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return LH_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    *why = "lh_residual_noalloc: device index out of range";
    return LH_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  DevAddr& a = g_addr[dev];
  if (!a.ready) {
    // the names g_ev, ... are host-side stand-ins; their device addresses come from here
    e = cudaGetSymbolAddress(reinterpret_cast<void**>(&a.ev), g_ev);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&a.blockmin), g_blockmin);
    if (e == cudaSuccess) e = cudaGetSymbolAddress(reinterpret_cast<void**>(&a.tab), g_tab);
    if (e != cudaSuccess) {
      *why = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return LH_ECUDA;
    }
    // the 1D tables of every order, written once per device (synchronous copies, made
    // before any call of this device launches work), so that a call copies nothing
    for (int K = 1; K <= kOrders; ++K) {
      const std::vector<double> tab = lh::host_tables(K);
      if ((int)tab.size() > kTabMax) {
        *why = "lh_residual_noalloc: table too large";
        return LH_EINVAL;
      }
      e = cudaMemcpy(a.tab + (size_t)(K - 1) * kTabMax, tab.data(), sizeof(double) * tab.size(),
                     cudaMemcpyHostToDevice);
      if (e != cudaSuccess) {
        *why = std::string("lh_residual_noalloc: table upload: ") + cudaGetErrorString(e);
        return LH_ECUDA;
      }
    }
    a.ready = true;
  }
  *out = a;
  return LH_OK;
}

}  // namespace

extern "C" lh_status lh_residual_noalloc(const lh_mesh_desc* desc, const double* rho0, const double* gamma,
                                         const double* u, const double* k, double tau, double* r) {
  std::string why;
  if (!lh::check_desc(desc, &why)) return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: " + why);
  if (!rho0 || !gamma || !u || !k || !r)
    return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: NULL array argument");
  if (r == u || r == k) return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: r must not alias u or k");
  lh::ElemParams P;
  lh::fill_params(*desc, &P);
  long long nd = 1;
  for (int c = 0; c < P.dim; ++c) nd *= P.K + 1;
  const long long ev_need = P.NE * P.dim * nd;
  if (ev_need > kEvMax)
    return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: mesh too large for the static scratch (NE*dim*(k+1)^dim = " +
                                               std::to_string(ev_need) + " > " + std::to_string(kEvMax) + ")");
  if ((long long)lh::elem_grid(P) > kBlocksMax)
    return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: too many element blocks for the static scratch");
  if (P.K < 1 || P.K > kOrders) return lh::set_global_error(LH_EINVAL, "lh_residual_noalloc: order out of range");
  DevAddr a;
  lh_status st = device_addresses(&a, &why);
  if (st != LH_OK) return lh::set_global_error(st, why);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(desc->stream);
  // the tables are constant per order; the element scratch and the block minima are fully
  // written before they are read, so nothing needs clearing
  P.tab = a.tab + (size_t)(P.K - 1) * kTabMax;
  P.rho0 = rho0;
  P.gamma = gamma;
  cudaError_t e = lh::launch_residual(P, s, u, k, tau, a.ev, a.blockmin, r, nullptr, nullptr);
  if (e != cudaSuccess)
    return lh::set_global_error(LH_ECUDA, std::string("lh_residual_noalloc: ") + cudaGetErrorString(e));
  return LH_OK;
}
