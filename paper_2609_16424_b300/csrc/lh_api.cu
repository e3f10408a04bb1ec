// C ABI of the library (include/lh.h): mesh set-up, operator calls, mass solves and the
// Newton-GMRES implicit midpoint step (paper Sec. 3.5 and Sec. 4.1).
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>
#include "lh_internal.h"
#include "lh_kernels.h"

using namespace lh;

namespace {

std::string g_err;   // message for failures that have no mesh

// precond 2 keeps each free velocity entry at >= this fraction of diag(M_V): the viscous part
// tau dF.1/dv of the diagonal comes from the FP32 record and is not sign-definite
constexpr double kJvvFloor = 0.5;

lh_status fail(lh_mesh* m, lh_status st, const std::string& msg) {
  if (m) m->err = msg; else g_err = msg;
  return st;
}

#define LH_CK(m, call)                                                                     \
  do {                                                                                     \
    cudaError_t e__ = (call);                                                              \
    if (e__ != cudaSuccess)                                                                \
      return fail(m, LH_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__));      \
  } while (0)

// ---- 1D rules and bases on [0, 1] (host, double) -------------------------------------
// Legendre P_n and P_n' at x in [-1, 1] by the three-term recurrence.
void legendre(int n, double x, double& p, double& dp) {
  double p0 = 1.0, p1 = x;
  if (n == 0) { p = 1.0; dp = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    const double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  p = p1;
  dp = n * (x * p1 - p0) / (x * x - 1.0);
}

// n-point Gauss-Legendre on [0, 1]: roots of P_n by Newton from Chebyshev-like guesses
void gauss(int n, std::vector<double>& z, std::vector<double>& w) {
  z.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double x = -std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(n, x, p, dp);
      const double dx = p / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    double p, dp;
    legendre(n, x, p, dp);
    z[i] = 0.5 * (x + 1.0);
    w[i] = 1.0 / ((1.0 - x * x) * dp * dp);     // 2 / ((1-x^2) P'^2) scaled by 1/2
  }
}

// n-point Gauss-Lobatto on [0, 1]: end points and the roots of P'_{n-1}, found by Newton
// on P'_{n-1} with P''_{n-1} from Legendre's equation
void lobatto(int n, std::vector<double>& z) {
  z.assign(n, 0.0);
  const int m = n - 1;
  z[0] = 0.0;
  z[n - 1] = 1.0;
  for (int i = 1; i < n - 1; ++i) {
    double x = -std::cos(M_PI * i / m);
    for (int it = 0; it < 100; ++it) {
      double p, dp;
      legendre(m, x, p, dp);
      const double ddp = (2.0 * x * dp - m * (m + 1.0) * p) / (1.0 - x * x);
      const double dx = dp / ddp;
      x -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    z[i] = 0.5 * (x + 1.0);
  }
}

double lagr(const std::vector<double>& z, int j, double t) {
  double v = 1.0;
  for (size_t l = 0; l < z.size(); ++l)
    if ((int)l != j) v *= (t - z[l]) / (z[j] - z[l]);
  return v;
}

double lagr_d(const std::vector<double>& z, int j, double t) {
  double s = 0.0;
  for (size_t l = 0; l < z.size(); ++l) {
    if ((int)l == j) continue;
    double v = 1.0 / (z[j] - z[l]);
    for (size_t i = 0; i < z.size(); ++i)
      if ((int)i != j && i != l) v *= (t - z[i]) / (z[j] - z[i]);
    s += v;
  }
  return s;
}

// device table: [B (QxD) | G (QxD) | Bl (QxL) | w (Q) | zh (D) | zl (L)]
std::vector<double> build_tables(int K) {
  const int D = K + 1, L = K, Q = 2 * K;
  std::vector<double> zq, wq, zh, zl, wl;
  gauss(Q, zq, wq);
  lobatto(D, zh);
  gauss(L, zl, wl);
  std::vector<double> t;
  for (int q = 0; q < Q; ++q)
    for (int a = 0; a < D; ++a) t.push_back(lagr(zh, a, zq[q]));
  for (int q = 0; q < Q; ++q)
    for (int a = 0; a < D; ++a) t.push_back(lagr_d(zh, a, zq[q]));
  for (int q = 0; q < Q; ++q)
    for (int j = 0; j < L; ++j) t.push_back(lagr(zl, j, zq[q]));
  for (int q = 0; q < Q; ++q) t.push_back(wq[q]);
  for (int a = 0; a < D; ++a) t.push_back(zh[a]);
  for (int j = 0; j < L; ++j) t.push_back(zl[j]);
  return t;
}

// dense inverse by Gauss-Jordan elimination with partial pivoting (row-major, n x n)
bool invert(std::vector<double>& a, int n) {
  std::vector<double> inv((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) inv[(size_t)i * n + i] = 1.0;
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(a[(size_t)r * n + c]) > std::fabs(a[(size_t)piv * n + c])) piv = r;
    if (a[(size_t)piv * n + c] == 0.0) return false;
    if (piv != c)
      for (int j = 0; j < n; ++j) {
        std::swap(a[(size_t)c * n + j], a[(size_t)piv * n + j]);
        std::swap(inv[(size_t)c * n + j], inv[(size_t)piv * n + j]);
      }
    const double d = 1.0 / a[(size_t)c * n + c];
    for (int j = 0; j < n; ++j) {
      a[(size_t)c * n + j] *= d;
      inv[(size_t)c * n + j] *= d;
    }
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * n + c];
      if (f == 0.0) continue;
      for (int j = 0; j < n; ++j) {
        a[(size_t)r * n + j] -= f * a[(size_t)c * n + j];
        inv[(size_t)r * n + j] -= f * inv[(size_t)c * n + j];
      }
    }
  }
  a.swap(inv);
  return true;
}

// transposed inverse (float) of the assembled 1D mass matrix along one axis; with
// drop_lo / drop_hi the end rows and columns are removed first and identity rows put back
bool kron_factor(const std::vector<double>& tab, int K, int nel, double h, bool drop_lo, bool drop_hi,
                 std::vector<float>& out) {
  const int D = K + 1, Q = 2 * K, N = K * nel + 1;
  const double* B = tab.data();
  const double* w = tab.data() + 2 * Q * D + Q * K;
  std::vector<double> M((size_t)N * N, 0.0);
  for (int e = 0; e < nel; ++e)
    for (int a = 0; a < D; ++a)
      for (int b = 0; b < D; ++b) {
        double s = 0.0;
        for (int q = 0; q < Q; ++q) s += w[q] * B[q * D + a] * B[q * D + b];
        M[(size_t)(e * K + a) * N + e * K + b] += h * s;
      }
  const int lo = drop_lo ? 1 : 0, hi = drop_hi ? N - 1 : N;
  const int n = hi - lo;
  std::vector<double> R((size_t)n * n);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) R[(size_t)i * n + j] = M[(size_t)(i + lo) * N + j + lo];
  if (!invert(R, n)) return false;
  out.assign((size_t)N * N, 0.f);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double v;
      if (i >= lo && i < hi && j >= lo && j < hi) v = R[(size_t)(i - lo) * n + (j - lo)];
      else v = (i == j) ? 1.0 : 0.0;
      out[(size_t)j * N + i] = (float)v;    // transposed: entry [j][i]
    }
  return true;
}

lh_status ensure_work(lh_mesh* m, int restart) {
  const long long n = m->n;
  const long long need = (long long)(restart + 1) * n + 8 * n;
  if (m->d_work && m->work_len >= need) return LH_OK;
  if (m->d_work) cudaFree(m->d_work);
  if (m->d_fwork) cudaFree(m->d_fwork);
  m->d_work = nullptr;
  m->d_fwork = nullptr;
  if (cudaMalloc(&m->d_work, sizeof(double) * need) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate Newton-GMRES workspace");
  m->ldf = (n + 63) / 64 * 64;
  if (cudaMalloc(&m->d_fwork, sizeof(float) * ((long long)(restart + 4) * m->ldf)) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate FP32 workspace");
  // the tails [n, ldf) stay zero: kernels write n entries, the float4 reductions read n4
  if (cudaMemset(m->d_fwork, 0, sizeof(float) * ((long long)(restart + 4) * m->ldf)) != cudaSuccess)
    return fail(m, LH_ECUDA, "cannot clear FP32 workspace");
  m->work_len = need;
  m->restart_alloc = restart;
  return LH_OK;
}

// ---- opt-in event profiler of element kernels
cudaError_t prof_flush(lh_mesh* m) {
  Prof& p = m->prof;
  if (p.n == 0) return cudaSuccess;
  cudaError_t e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < p.n; ++i) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]);
    if (e != cudaSuccess) return e;
    p.ms[p.kind[i]] += ms;
    p.cnt[p.kind[i]] += 1;
  }
  p.n = 0;
  return cudaSuccess;
}

// event pair for the next element-kernel launch of the given kind, or NULL when off
// device int set by the tensor-core J.w when one of its bounded waits gives up
int* tc_err(lh_mesh* m) { return reinterpret_cast<int*>(m->d_scalar + 255); }

cudaEvent_t* prof_pair(lh_mesh* m, int kind) {
  Prof& p = m->prof;
  if (!p.on) return nullptr;
  if (p.n == Prof::kMax && prof_flush(m) != cudaSuccess) return nullptr;
  p.kind[p.n] = kind;
  return &p.ev[2 * p.n++];
}

// pinned host scratch for the small read-backs of the Newton loop and the GMRES coefficients
// y (entries 16..16 + kArnMax); NULL if it cannot be allocated (pageable memory then)
constexpr int kSmallHost = 16 + kArnMax;
double* host_small(lh_mesh* m) {
  if (!m->h_small && cudaMallocHost(&m->h_small, sizeof(double) * kSmallHost) != cudaSuccess) {
    m->h_small = nullptr;
    (void)cudaGetLastError();
  }
  return m->h_small;
}

// a . b into a host double (synchronises)
lh_status dot_host(lh_mesh* m, const double* a, const double* b, long long n, double* out) {
  LH_CK(m, launch_mdot<double>(m->stream, a, 1, 0, b, n, 0, m->d_part, m->d_counter, m->d_scalar));
  double* h = host_small(m);
  LH_CK(m, cudaMemcpyAsync(h ? h : out, m->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  if (h) *out = h[0];
  return LH_OK;
}

// Krylov operator of one Newton iteration, y = J P^-1 x, for a basis of type T:
//   T = double: FP64 preconditioner and FP64 J.w (state re-gathered and re-contracted);
//   T = float : FP32 preconditioner and FP32 J.w from the linearisation record written by
//               the last residual evaluation (at the current Newton iterate).
// velocity diagonal of the preconditioner kind: diag(M_V) per node, or (kind 2) the per-dof
// diagonal of dR_v/dk_v at the current Newton iterate
const double* prec_diag(const lh_mesh* m, int pk) { return pk == 2 ? m->d_jdiag : m->d_diagMv; }

template <class T>
struct KrylovOp {
  lh_mesh* m;
  int pk;             // preconditioner kind
  int tck;            // float J.w: -1 FP32 CUDA cores, 0 TF32 tensor cores, 1 BF16 tensor cores
  const double* u;
  const double* k;
  double tau;
  T* z;               // scratch [n]
  const double* wsc = nullptr;   // row weights W of the scaled norm: the operator is W J P^-1

  lh_status apply(const T* x, T* y) {
    if (pk == 3) {
      lh_status st = cheb(x, z);
      if (st != LH_OK) return st;
    } else {
      LH_CK(m, (launch_prec<T, T>(pk, m->stream, m->P, m->kron, prec_diag(m, pk), m->d_invMe, x, z, tau)));
    }
    if constexpr (sizeof(T) == sizeof(double)) {
      LH_CK(m, launch_jvp_f64(m->P, m->stream, u, k, tau, z, m->d_ev, y, prof_pair(m, LH_PROF_JVP64)));
    } else {
      LH_CK(m, jvp_f32(z, y));
    }
    if (wsc) LH_CK(m, launch_row_mul<T>(m->stream, wsc, y, y, m->n));
    return LH_OK;
  }
  cudaError_t jvp_f32(const float* x, float* y) {
    if (tck < 0)
      return launch_jvp_rec_f32(m->P, m->stream, m->d_rec, tau, x, reinterpret_cast<float*>(m->d_ev), y,
                                prof_pair(m, LH_PROF_JVP32), tc_err(m));
    return launch_jvp_tc<float>(m->P, m->stream, tck, m->d_rec, tau, x, reinterpret_cast<float*>(m->d_ev), y,
                                tc_err(m), prof_pair(m, LH_PROF_JVPTC));
  }
  // z = P^-1 x with the Chebyshev velocity block (kind 3, FP32 record J.w); float input
  template <class TZ>
  lh_status cheb(const T* x, TZ* out) {
    if constexpr (sizeof(T) != sizeof(float)) {
      return fail(m, LH_EINVAL, "precond 3 needs the FP32 Krylov basis");
    } else {
      cudaStream_t s = m->stream;
      const long long n = m->n, n1 = (long long)m->P.dim * m->P.NV, ld = m->ldf;
      float* res = m->d_cheb;
      float* d = res + ld;
      float* zc = d + ld;
      float* wdir = zc + ld;
      float* jw = wdir + ld;
      const double a = m->cheb_b / m->cheb_ratio, b = m->cheb_b;
      const double theta = 0.5 * (b + a), delta = 0.5 * (b - a), sigma = theta / delta;
      LH_CK(m, launch_cheb_init<float>(s, n1, m->d_jdiag, x, res, d, zc, 1.0 / theta));
      double rho_old = 1.0 / sigma;
      for (int it = 1; it < m->cheb_degree; ++it) {
        LH_CK(m, launch_cheb_dir(s, n1, n, d, wdir, tau));
        LH_CK(m, jvp_f32(wdir, jw));
        const double rho = 1.0 / (2.0 * sigma - rho_old);
        LH_CK(m, launch_cheb_step(s, n1, m->d_jdiag, jw, res, d, zc, rho * rho_old, 2.0 * rho / delta));
        rho_old = rho;
      }
      LH_CK(m, (launch_cheb_out<float, TZ>(s, n1, n, m->d_invMe, x, zc, out, tau)));
      return LH_OK;
    }
  }
  // y = J d for a double vector d (restarts)
  lh_status jac(const double* d, T* y) {
    if constexpr (sizeof(T) == sizeof(double)) {
      LH_CK(m, launch_jvp_f64(m->P, m->stream, u, k, tau, d, m->d_ev, y, prof_pair(m, LH_PROF_JVP64)));
    } else {
      LH_CK(m, (launch_scale<double, float>(m->stream, 1.0, d, 0.0, nullptr, z, m->n)));
      LH_CK(m, jvp_f32(z, y));
    }
    if (wsc) LH_CK(m, launch_row_mul<T>(m->stream, wsc, y, y, m->n));
    return LH_OK;
  }
};

// Upper end of the spectrum of D^-1 S for the Chebyshev interval of preconditioner kind 3:
// five power steps from the diagonal itself, S applied by the record J.w; b = 1.1 x the
// estimate (tmp: double scratch of dim NV)
lh_status cheb_bounds(lh_mesh* m, const lh_newton_opts& o, double tau, int tck, double* tmp) {
  cudaStream_t s = m->stream;
  const long long n = m->n, n1 = (long long)m->P.dim * m->P.NV, ld = m->ldf;
  float* v = m->d_cheb;
  float* y = v + ld;
  float* wdir = v + 3 * ld;
  float* jw = v + 4 * ld;
  KrylovOp<float> op{m, 3, tck, nullptr, nullptr, tau, nullptr};
  lh_status st;
  LH_CK(m, launch_to_f32(s, m->d_jdiag, v + n1, n1));
  double nv2 = 0.0, lam = 0.0;
  LH_CK(m, launch_to_f64(s, v + n1, tmp, n1));
  if ((st = dot_host(m, tmp, tmp, n1, &nv2)) != LH_OK) return st;
  LH_CK(m, (launch_scale<float, float>(s, 1.0 / std::sqrt(nv2), v + n1, 0.0, nullptr, v + n1, n1)));
  for (int it = 0; it < 5; ++it) {
    LH_CK(m, launch_cheb_dir(s, n1, n, v, wdir, tau));
    LH_CK(m, op.jvp_f32(wdir, jw));
    LH_CK(m, launch_cheb_scale(s, n1, m->d_jdiag, jw, y));
    LH_CK(m, launch_to_f64(s, y + n1, tmp, n1));
    double ny2 = 0.0;
    if ((st = dot_host(m, tmp, tmp, n1, &ny2)) != LH_OK) return st;
    if (!(ny2 > 0.0) || !std::isfinite(ny2)) return fail(m, LH_ENONFINITE, "precond 3: power iteration failed");
    lam = std::sqrt(ny2);
    LH_CK(m, (launch_scale<float, float>(s, 1.0 / lam, y + n1, 0.0, nullptr, v + n1, n1)));
  }
  m->cheb_b = 1.1 * lam;
  m->cheb_ratio = o.cheb_ratio;
  m->cheb_degree = o.cheb_degree;
  return LH_OK;
}

// ---- device-driven Arnoldi (FP32 basis) ----
// bit of the operator kind (preconditioner, J.w form, row weights) in ArnGraph::warm
unsigned long long arn_kind(const KrylovOp<float>& op) {
  return 1ull << (((op.pk * 3) + (op.tck + 1)) * 2 + (op.wsc ? 1 : 0));
}

// gives up on the device-driven Arnoldi for this mesh (the host loop runs from then on)
bool arn_off(lh_mesh* m) {
  ArnGraph& G = m->arn;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
  G.off = true;
  (void)cudaGetLastError();
  return false;
}

// zero-initialised graph-node parameters (cudaGraphNodeParams has no default constructor:
// its union holds dim3s)
union ZeroNodeParams {
  cudaGraphNodeParams p;
  unsigned char raw[sizeof(cudaGraphNodeParams)];
  ZeroNodeParams() { std::memset(raw, 0, sizeof(raw)); }
};

// One Arnoldi iteration, recorded into the WHILE body: y = J P^-1 v_j (v_j in d_vin), both
// Gram-Schmidt passes with the column count read from the cycle state, v_{j+1} by the
// Pythagorean norm, an IF node with the exact-norm fallback (run only when the second pass
// still cancelled; its body is recorded on the second private stream), then the Givens
// update that ends the loop.
lh_status arn_body(lh_mesh* m, KrylovOp<float>& op, float* V, float* w, long long ld, long long len,
                   cudaGraphConditionalHandle cond) {
  cudaStream_t s = m->stream;
  double* dh = m->d_scalar + 8;
  double* dh2 = dh + 72;
  ArnState* st = m->d_arn;
  const int* jd = &st->j;
  lh_status e = op.apply(m->d_vin, w);
  if (e != LH_OK) return e;
  float* wp = op.z;   // the projected vector w' = w - V h1 (the operator's scratch is free again)
  LH_CK(m, launch_mdot_dev(s, V, jd, ld, w, len, 1, nullptr, m->d_part, m->d_counter, dh));
  LH_CK(m, launch_mdot_sub(s, V, 0, jd, ld, w, dh, wp, len, m->d_part, m->d_counter, dh2));
  // the IF node after the second update, then its body
  cudaStreamCaptureStatus cs;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  LH_CK(m, cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, nullptr, nullptr, nullptr));   // the WHILE body
  cudaGraphConditionalHandle fix;
  LH_CK(m, cudaGraphConditionalHandleCreate(&fix, capg, 0u, 0u));
  LH_CK(m, launch_gemv_norm_dev(s, V, st, ld, dh2, wp, m->d_vin, len, fix));
  LH_CK(m, cudaStreamGetCaptureInfo(s, &cs, nullptr, &capg, &deps, nullptr, &nd));
  ZeroNodeParams zp;
  cudaGraphNodeParams& np = zp.p;
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = fix;
  np.conditional.type = cudaGraphCondTypeIf;
  np.conditional.size = 1;
  cudaGraphNode_t ifn;
  LH_CK(m, cudaGraphAddNode(&ifn, capg, deps, nullptr, nd, &np));
  LH_CK(m, cudaStreamUpdateCaptureDependencies(s, &ifn, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaStream_t s2 = m->arn.cap2;
  LH_CK(m, cudaStreamBeginCaptureToGraph(s2, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal));
  const long long l0 = launches();
  const cudaError_t e1 = launch_gemv_sub_dev(s2, V, jd, ld, dh2, wp, len, nullptr);
  const cudaError_t e2 = launch_mdot_dev(s2, wp, nullptr, 0, wp, len, 0, nullptr, m->d_part, m->d_counter, &st->hn2);
  const cudaError_t e3 = launch_arn_scale(s2, st, wp, V, ld, m->d_vin, len);
  m->arn.per_fix = launches() - l0;   // the IF body runs only when the second pass cancelled
  cudaGraph_t got = nullptr;
  const cudaError_t e4 = cudaStreamEndCapture(s2, &got);
  LH_CK(m, e1 != cudaSuccess ? e1 : e2 != cudaSuccess ? e2 : e3 != cudaSuccess ? e3 : e4);
  LH_CK(m, launch_arn_givens(s, dh, dh2, st, cond));
  return LH_OK;
}

// Records the cycle graph: a WHILE conditional node (condition 1 at every launch) whose body
// is one Arnoldi iteration, captured on a private stream.  False (and the host loop from then
// on) if any step is refused.
bool arn_record(lh_mesh* m, KrylovOp<float>& op, float* V, float* w, long long ld, long long len) {
  ArnGraph& G = m->arn;
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.graph) cudaGraphDestroy(G.graph);
  G.exec = nullptr;
  G.graph = nullptr;
  if (!G.cap && cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking) != cudaSuccess) {
    G.cap = nullptr;
    return arn_off(m);
  }
  if (!G.cap2 && cudaStreamCreateWithFlags(&G.cap2, cudaStreamNonBlocking) != cudaSuccess) {
    G.cap2 = nullptr;
    return arn_off(m);
  }
  if (cudaGraphCreate(&G.graph, 0) != cudaSuccess) {
    G.graph = nullptr;
    return arn_off(m);
  }
  cudaGraphConditionalHandle cond;
  if (cudaGraphConditionalHandleCreate(&cond, G.graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess)
    return arn_off(m);
  ZeroNodeParams zp;
  cudaGraphNodeParams& np = zp.p;
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = cond;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  if (cudaGraphAddNode(&node, G.graph, nullptr, nullptr, 0, &np) != cudaSuccess) return arn_off(m);
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamBeginCaptureToGraph(G.cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
      cudaSuccess)
    return arn_off(m);
  cudaStream_t keep = m->stream;
  const long long l0 = launches();
  m->stream = G.cap;
  const lh_status st = arn_body(m, op, V, w, ld, len, cond);
  m->stream = keep;
  cudaGraph_t got = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(G.cap, &got);
  G.per_it = launches() - l0;
  count_launches((int)-G.per_it);   // recorded, not run
  G.per_it -= G.per_fix;            // kernels of every iteration (the IF body's are rare)
  if (st != LH_OK || ce != cudaSuccess) return arn_off(m);
  if (cudaGraphInstantiate(&G.exec, G.graph, 0) != cudaSuccess) {
    G.exec = nullptr;
    return arn_off(m);
  }
  G.V = V;
  G.w = w;
  G.z = op.z;
  G.wsc = op.wsc;
  G.ld = ld;
  G.len = len;
  G.n = m->n;
  G.pk = op.pk;
  G.tck = op.tck;
  G.tau = op.tau;
  G.cheb_b = m->cheb_b;
  G.cheb_ratio = m->cheb_ratio;
  G.cheb_degree = m->cheb_degree;
  return true;
}

// GMRES of the header comment below with the Arnoldi iterations of each restart cycle in one
// graph launch; *used = false (nothing done) when this path does not apply.
lh_status gmres_dev(lh_mesh* m, const lh_newton_opts& o, KrylovOp<float>& op, const double* r, double nr,
                    double* dk, float* V, float* w, float* ulin, double* zd, double* wd, lh_step_stats& S,
                    bool* used) {
  *used = false;
  ArnGraph& G = m->arn;
  if (o.arnoldi != 1 || G.off || m->prof.on || o.restart < 1 || o.restart > kArnMax || !(G.warm & arn_kind(op)))
    return LH_OK;
  const long long n = m->n, ld = m->ldf, len = (n + 3) / 4 * 4;
  const int mres = o.restart;
  cudaStream_t s = m->stream;
  if (!m->d_arn && cudaMalloc(&m->d_arn, sizeof(ArnState)) != cudaSuccess) {
    m->d_arn = nullptr;
    arn_off(m);
    return LH_OK;
  }
  if (!m->h_arn && cudaMallocHost(&m->h_arn, sizeof(ArnState)) != cudaSuccess) {
    m->h_arn = nullptr;
    arn_off(m);
    return LH_OK;
  }
  if (!m->d_vin) {
    if (cudaMalloc(&m->d_vin, sizeof(float) * ld) != cudaSuccess) {
      m->d_vin = nullptr;
      arn_off(m);
      return LH_OK;
    }
    LH_CK(m, cudaMemsetAsync(m->d_vin, 0, sizeof(float) * ld, s));
  }
  const bool same = G.exec && G.V == V && G.w == w && G.z == op.z && G.wsc == op.wsc && G.ld == ld &&
                    G.len == len && G.n == n && G.pk == op.pk && G.tck == op.tck && G.tau == op.tau &&
                    (op.pk != 3 || (G.cheb_b == m->cheb_b && G.cheb_ratio == m->cheb_ratio &&
                                    G.cheb_degree == m->cheb_degree));
  if (!same && !arn_record(m, op, V, w, ld, len)) return LH_OK;
  *used = true;
  double* dh = m->d_scalar + 8;
  ArnState* h = m->h_arn;
  LH_CK(m, cudaMemsetAsync(dk, 0, sizeof(double) * n, s));
  double beta = nr;
  const double beta0 = nr;
  LH_CK(m, (launch_scale<double, float>(s, -1.0 / beta, r, 0.0, nullptr, V, n)));
  int total = 0;
  lh_status st;
  while (total < o.gmres_maxit) {
    LH_CK(m, cudaMemcpyAsync(m->d_vin, V, sizeof(float) * len, cudaMemcpyDeviceToDevice, s));
    h->j = 0;
    h->stop = 0;
    h->fix = 0;
    h->mres = mres;
    h->maxit = o.gmres_maxit - total;
    h->pad_ = 0;
    h->tol = o.gmres_rtol * beta0;
    h->hn2 = 0.0;
    for (int i = 0; i <= kArnMax; ++i) h->g[i] = 0.0;
    h->g[0] = beta;
    LH_CK(m, cudaMemcpyAsync(m->d_arn, h, offsetof(ArnState, cs), cudaMemcpyHostToDevice, s));
    LH_CK(m, cudaGraphLaunch(G.exec, s));
    LH_CK(m, cudaMemcpyAsync(h, m->d_arn, sizeof(ArnState), cudaMemcpyDeviceToHost, s));
    LH_CK(m, cudaStreamSynchronize(s));
    const int j = h->j;
    count_launches((int)(j * G.per_it));
    total += j;
    S.jvp_evals += j;
    S.reorth += j;
    if (h->stop == 5) return fail(m, LH_ENONFINITE, "lh_newton_step: non-finite Krylov vector");
    if (j < 1 || j > mres) return fail(m, LH_ECUDA, "device Arnoldi: inconsistent cycle state");
    const bool done = h->stop == 1;
    // y = H^-1 g (upper triangular j x j), dk += P^-1 V y
    std::vector<double> yv(j);
    double* hs = host_small(m);
    double* y = hs ? hs + 16 : yv.data();   // pinned: the copy below does not stage
    for (int i = j - 1; i >= 0; --i) {
      double sum = h->g[i];
      for (int l = i + 1; l < j; ++l) sum -= h->H[i * kArnMax + l] * y[l];
      y[i] = sum / h->H[i * kArnMax + i];
    }
    LH_CK(m, cudaMemcpyAsync(dh, y, sizeof(double) * j, cudaMemcpyHostToDevice, s));
    LH_CK(m, launch_gemv<float>(s, V, j, ld, dh, 0.0, ulin, len));
    if (op.pk == 3) {
      if ((st = op.template cheb<double>(ulin, zd)) != LH_OK) return st;
    } else {
      LH_CK(m, (launch_prec<float, double>(op.pk, s, m->P, m->kron, prec_diag(m, op.pk), m->d_invMe, ulin, zd,
                                           op.tau)));
    }
    LH_CK(m, launch_axpby(s, 1.0, zd, 1.0, dk, n));
    if (done || total >= o.gmres_maxit) break;
    // restart from the true linear residual -r - J dk
    if ((st = op.jac(dk, w)) != LH_OK) return st;
    ++S.jvp_evals;
    LH_CK(m, (launch_scale<double, double>(s, -1.0, r, -1.0, w, wd, n)));
    double b2;
    if ((st = dot_host(m, wd, wd, n, &b2)) != LH_OK) return st;
    beta = std::sqrt(b2);
    if (beta <= o.gmres_rtol * beta0) break;
    LH_CK(m, (launch_scale<double, float>(s, 1.0 / beta, wd, 0.0, nullptr, V, n)));
  }
  S.gmres_its_total += total;
  return LH_OK;
}

// Restarted, right-preconditioned GMRES on J dk = -r from dk = 0 (paper Sec. 3.5, Eq. (22)).
// Classical Gram-Schmidt applied twice (CGS2), each pass one fused reduction (V^T w and
// w.w); the norm of the projected vector by Pythagoras from the second pass, computed on
// the device by the update that writes v_{j+1}, so an iteration reads back one column of
// coefficients; an exact norm only if the second pass still cancelled.  (Skipping the
// second pass for the FP32 basis unless 63/64 of the norm cancelled was tried: GMRES then
// needed 2.4x the iterations on the point-blast workload.)
// Basis V and work vectors w, ulin of type T; zd, wd double scratch; Givens on the host.
template <class T>
lh_status gmres(lh_mesh* m, const lh_newton_opts& o, KrylovOp<T>& op, const double* r, double nr, double* dk,
                T* V, T* w, T* ulin, double* zd, double* wd, lh_step_stats& S) {
  if constexpr (sizeof(T) == sizeof(float)) {
    bool used = false;
    const lh_status sd = gmres_dev(m, o, op, r, nr, dk, V, w, ulin, zd, wd, S, &used);
    if (used || sd != LH_OK) return sd;
  }
  const long long n = m->n;
  // FP32 basis: leading dimension ldf, reductions over n rounded up to 4 (zero tails);
  // FP64 basis: contiguous
  const long long ld = sizeof(T) == sizeof(float) ? m->ldf : n;
  const long long len = sizeof(T) == sizeof(float) ? (n + 3) / 4 * 4 : n;
  const int mres = o.restart;
  cudaStream_t s = m->stream;
  double* dh = m->d_scalar + 8;   // device coefficients: first pass [0, 72), second [72, 144); y
  lh_status st;
  std::vector<double> H((size_t)(mres + 1) * mres), cs(mres), sn(mres), g(mres + 1), hcol(144);
  LH_CK(m, cudaMemsetAsync(dk, 0, sizeof(double) * n, s));
  double beta = nr;
  const double beta0 = nr;
  LH_CK(m, (launch_scale<double, T>(s, -1.0 / beta, r, 0.0, nullptr, V, n)));
  int total = 0;
  bool done = false;
  while (!done) {
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int j = 0;
    for (; j < mres && total < o.gmres_maxit; ++j) {
      T* vj = V + (long long)j * ld;
      if ((st = op.apply(vj, w)) != LH_OK) return st;
      ++S.jvp_evals;
      // CGS2: both passes and the normalisation on the device, one read-back per iteration
      double* dh2 = dh + 72;   // the first pass writes up to 66 values at dh
      T* vn = V + (long long)(j + 1) * ld;
      LH_CK(m, launch_mdot<T>(s, V, j + 1, ld, w, len, 1, m->d_part, m->d_counter, dh));
      T* wp = w;   // the projected vector w' = w - V h1
      if constexpr (sizeof(T) == sizeof(float)) {   // update fused into the second multi-dot, w' in z
        wp = op.z;
        LH_CK(m, launch_mdot_sub(s, V, j + 1, nullptr, ld, w, dh, wp, len, m->d_part, m->d_counter, dh2));
      } else {
        LH_CK(m, launch_gemv_sub<T>(s, V, j + 1, ld, dh, w, len));
        LH_CK(m, launch_mdot<T>(s, V, j + 1, ld, w, len, 1, m->d_part, m->d_counter, dh2));
      }
      LH_CK(m, launch_gemv_norm<T>(s, V, j + 1, ld, dh2, wp, vn, len));
      LH_CK(m, cudaMemcpyAsync(hcol.data(), dh, sizeof(double) * (72 + j + 2), cudaMemcpyDeviceToHost, s));
      LH_CK(m, cudaStreamSynchronize(s));
      ++S.reorth;
      double hh2 = 0.0;
      for (int i = 0; i <= j; ++i) {
        H[(size_t)i * mres + j] = hcol[i] + hcol[72 + i];
        hh2 += hcol[72 + i] * hcol[72 + i];
      }
      const double ww2 = hcol[72 + j + 1];
      double hn2 = ww2 - hh2;
      if (!(hn2 > 1e-4 * ww2)) {   // the second pass still cancelled: take the exact norm
        LH_CK(m, launch_gemv_sub<T>(s, V, j + 1, ld, dh2, wp, len));
        LH_CK(m, launch_mdot<T>(s, wp, 1, 0, wp, len, 0, m->d_part, m->d_counter, dh));
        LH_CK(m, cudaMemcpyAsync(hcol.data(), dh, sizeof(double), cudaMemcpyDeviceToHost, s));
        LH_CK(m, cudaStreamSynchronize(s));
        hn2 = hcol[0];
        if (hn2 > 0.0) LH_CK(m, (launch_scale<T, T>(s, 1.0 / std::sqrt(hn2), wp, 0.0, nullptr, vn, n)));
      }
      if (!std::isfinite(hn2)) return fail(m, LH_ENONFINITE, "lh_newton_step: non-finite Krylov vector");
      const double hn = std::sqrt(std::fmax(hn2, 0.0));
      H[(size_t)(j + 1) * mres + j] = hn;
      for (int i = 0; i < j; ++i) {   // previous Givens rotations
        const double a = H[(size_t)i * mres + j], b = H[(size_t)(i + 1) * mres + j];
        H[(size_t)i * mres + j] = cs[i] * a + sn[i] * b;
        H[(size_t)(i + 1) * mres + j] = -sn[i] * a + cs[i] * b;
      }
      const double a = H[(size_t)j * mres + j], b = H[(size_t)(j + 1) * mres + j];
      const double rad = std::hypot(a, b);
      cs[j] = rad > 0 ? a / rad : 1.0;
      sn[j] = rad > 0 ? b / rad : 0.0;
      H[(size_t)j * mres + j] = rad;
      H[(size_t)(j + 1) * mres + j] = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      if (std::fabs(g[j + 1]) <= o.gmres_rtol * beta0 || hn == 0.0) {
        ++j;
        done = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular j x j), dk += P^-1 V y
    std::vector<double> y(j);
    for (int i = j - 1; i >= 0; --i) {
      double sum = g[i];
      for (int l = i + 1; l < j; ++l) sum -= H[(size_t)i * mres + l] * y[l];
      y[i] = sum / H[(size_t)i * mres + i];
    }
    LH_CK(m, cudaMemcpyAsync(dh, y.data(), sizeof(double) * j, cudaMemcpyHostToDevice, s));
    LH_CK(m, launch_gemv<T>(s, V, j, ld, dh, 0.0, ulin, len));
    if (op.pk == 3) {
      if ((st = op.template cheb<double>(ulin, zd)) != LH_OK) return st;
    } else {
      LH_CK(m, (launch_prec<T, double>(op.pk, s, m->P, m->kron, prec_diag(m, op.pk), m->d_invMe, ulin, zd,
                                       op.tau)));
    }
    LH_CK(m, launch_axpby(s, 1.0, zd, 1.0, dk, n));
    if (done || total >= o.gmres_maxit) break;
    // restart from the true linear residual -r - J dk
    if ((st = op.jac(dk, w)) != LH_OK) return st;
    ++S.jvp_evals;
    if constexpr (sizeof(T) == sizeof(double)) {
      LH_CK(m, launch_axpby(s, -1.0, r, -1.0, w, n));
      if (static_cast<void*>(w) != static_cast<void*>(wd))
        LH_CK(m, cudaMemcpyAsync(wd, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
    } else {
      LH_CK(m, (launch_scale<double, double>(s, -1.0, r, -1.0, w, wd, n)));
    }
    double b2;
    if ((st = dot_host(m, wd, wd, n, &b2)) != LH_OK) return st;
    beta = std::sqrt(b2);
    if (beta <= o.gmres_rtol * beta0) break;
    LH_CK(m, (launch_scale<double, T>(s, 1.0 / beta, wd, 0.0, nullptr, V, n)));
  }
  S.gmres_its_total += total;
  if constexpr (sizeof(T) == sizeof(float)) m->arn.warm |= arn_kind(op);   // its kernels have run once
  return LH_OK;
}

lh_status ensure_rec(lh_mesh* m) {
  if (m->d_rec) return LH_OK;
  if (cudaMalloc(&m->d_rec, sizeof(float) * (size_t)m->NQ * rec_len(m->P.dim)) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate the linearisation record");
  return LH_OK;
}

// residual + min detJ (host) in one call; rec (optional) receives the linearisation record
// the residual, its min det J and ||x||_2^2 with x = r (or W r in rs when wsc is given),
// read back together (one synchronisation)
lh_status residual_min_norm(lh_mesh* m, const double* u, const double* k, double tau, double* r, double* mindet,
                            double* nr2, float* rec, const double* wsc, double* rs) {
  cudaStream_t s = m->stream;
  LH_CK(m, launch_residual(m->P, s, u, k, tau, m->d_ev, m->d_blockmin, r, prof_pair(m, LH_PROF_RESIDUAL), rec));
  LH_CK(m, launch_min(s, m->d_blockmin, m->nblocks_elem, m->d_scalar + 1));
  const double* x = r;
  if (wsc) {
    LH_CK(m, launch_row_mul<double>(s, wsc, r, rs, m->n));
    x = rs;
  }
  LH_CK(m, launch_mdot<double>(s, x, 1, 0, x, m->n, 0, m->d_part, m->d_counter, m->d_scalar + 2));
  double* h = host_small(m);
  double tmp[2];
  LH_CK(m, cudaMemcpyAsync(h ? h : tmp, m->d_scalar + 1, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  LH_CK(m, cudaStreamSynchronize(s));
  *mindet = (h ? h : tmp)[0];
  *nr2 = (h ? h : tmp)[1];
  return LH_OK;
}

lh_status residual_min(lh_mesh* m, const double* u, const double* k, double tau, double* r, double* mindet,
                       float* rec = nullptr) {
  LH_CK(m, launch_residual(m->P, m->stream, u, k, tau, m->d_ev, m->d_blockmin, r, prof_pair(m, LH_PROF_RESIDUAL),
                           rec));
  LH_CK(m, launch_min(m->stream, m->d_blockmin, m->nblocks_elem, m->d_scalar + 1));
  LH_CK(m, cudaMemcpyAsync(mindet, m->d_scalar + 1, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return LH_OK;
}

}  // namespace

namespace lh {

bool check_desc(const lh_mesh_desc* d, std::string* why) {
  if (!d) { *why = "desc is NULL"; return false; }
  if (d->dim != 2 && d->dim != 3) { *why = "dim must be 2 or 3"; return false; }
  if (d->order < 1 || d->order > 4) { *why = "order must be in 1..4"; return false; }
  if (d->quad_1d != 0 && d->quad_1d != 2 * d->order) {
    *why = "only 2k Gauss points per direction are supported";
    return false;
  }
  for (int c = 0; c < d->dim; ++c) {
    if (d->n[c] < 1) { *why = "element counts must be >= 1"; return false; }
    if (!(d->hi[c] > d->lo[c])) { *why = "box must have hi > lo"; return false; }
  }
  {
    long long nv = 1;
    for (int c = 0; c < d->dim; ++c) nv *= (long long)d->order * d->n[c] + 1;
    if (d->dim * nv >= (1LL << 31)) {   // node-centric kernels index the lattice in 32 bits
      *why = "mesh too large: dim * H1 nodes must stay below 2^31";
      return false;
    }
  }
  if (d->visc && !(d->psi0 > 0.0 && d->psi0 < 1.0)) { *why = "psi0 must be in (0, 1)"; return false; }
  if (!(d->eps_e > 0.0)) { *why = "eps_e must be > 0"; return false; }
  if (d->tg_source && d->dim != 2) { *why = "the Taylor-Green source is 2D"; return false; }
  return true;
}

void fill_params(const lh_mesh_desc& d, ElemParams* out) {
  ElemParams& P = *out;
  P = ElemParams();
  const int dim = d.dim, K = d.order;
  P.dim = dim;
  P.K = K;
  P.n0 = d.n[0];
  P.n1 = d.n[1];
  P.n2 = dim == 3 ? d.n[2] : 1;
  P.N0 = K * P.n0 + 1;
  P.N1 = K * P.n1 + 1;
  P.N2 = dim == 3 ? K * P.n2 + 1 : 1;
  P.NE = (long long)P.n0 * P.n1 * P.n2;
  P.NV = (long long)P.N0 * P.N1 * P.N2;
  long long nl = 1;
  for (int c = 0; c < dim; ++c) nl *= K;
  P.NEd = P.NE * nl;
  double vol = 1.0;
  P.detJ0 = 1.0;
  for (int c = 0; c < 3; ++c) {
    P.lo[c] = c < dim ? d.lo[c] : 0.0;
    P.h[c] = c < dim ? (d.hi[c] - d.lo[c]) / d.n[c] : 1.0;
    if (c < dim) {
      vol *= d.hi[c] - d.lo[c];
      P.detJ0 *= P.h[c];
    }
  }
  P.h0 = d.h0 > 0 ? d.h0 : std::pow(vol / (double)P.NE, 1.0 / dim);
  P.inv_hc = 1.0 / (d.h_coarse > 0 ? d.h_coarse : P.h0);
  P.q1 = d.q1;
  P.q2 = d.q2;
  P.scoef = 2.0 * std::atanh(1.0 - 2.0 * d.psi0);
  P.eps2 = d.eps_e * d.eps_e;
  P.visc = d.visc;
  P.tg = d.tg_source;
  P.bc = d.bc_mask;
  auto split = [](double x, float (&w)[2]) {
    w[0] = (float)x;
    w[1] = (float)(x - (double)w[0]);
  };
  split(1.0 / P.detJ0, P.dw_inv_detJ0);
  split(P.h0, P.dw_h0);
  split(P.inv_hc, P.dw_inv_hc);
  split(P.q1, P.dw_q1);
  split(P.q2, P.dw_q2);
  split(P.scoef, P.dw_scoef);
  split(P.eps2, P.dw_eps2);
}

std::vector<double> host_tables(int K) { return build_tables(K); }

lh_status set_global_error(lh_status st, const std::string& msg) { return fail(nullptr, st, msg); }

}  // namespace lh

extern "C" {

void lh_mesh_desc_init(lh_mesh_desc* d) {
  if (!d) return;
  std::memset(d, 0, sizeof(*d));
  d->dim = 3;
  d->n[0] = d->n[1] = d->n[2] = 4;
  d->hi[0] = d->hi[1] = d->hi[2] = 1.0;
  d->order = 2;
  d->rho0_value = 1.0;
  d->gamma_value = 1.4;
  d->bc_mask = 0x3f;
  d->visc = 1;
  d->q1 = 0.5;
  d->q2 = 1.0;
  d->psi0 = 0.5;
  d->eps_e = 1e-6;
}

void lh_newton_opts_init(lh_newton_opts* o) {
  if (!o) return;
  o->newton_rtol = 1e-10;
  o->newton_atol = 0.0;
  o->gmres_rtol = 1e-12;
  o->newton_maxit = 20;
  o->gmres_maxit = 60;
  o->restart = 30;
  o->max_halvings = 10;
  o->jvp_prec = LH_FP64;
  o->precond = 1;
  o->forcing = 0;
  o->eta_max = 0.1;
  o->scaled_norm = 0;
  o->cheb_degree = 3;
  o->cheb_ratio = 20.0;
  o->arnoldi = 1;
}

lh_status lh_mesh_create(const lh_mesh_desc* d, lh_mesh** out) {
  if (!out) return fail(nullptr, LH_EINVAL, "out is NULL");
  *out = nullptr;
  std::string why;
  if (!lh::check_desc(d, &why)) return fail(nullptr, LH_EINVAL, why);
  lh_mesh* m = new (std::nothrow) lh_mesh();
  if (!m) return fail(nullptr, LH_ENOMEM, "host allocation failed");
  m->desc = *d;
  m->stream = reinterpret_cast<cudaStream_t>(d->stream);
  ElemParams& P = m->P;
  lh::fill_params(*d, &P);
  const int dim = d->dim, K = d->order;
  long long nd = 1, nq = 1;
  for (int c = 0; c < dim; ++c) {
    nd *= K + 1;
    nq *= 2 * K;
  }
  m->n = 2LL * dim * P.NV + P.NEd;
  m->NQ = P.NE * nq;

  std::vector<double> rho(P.NE), gam(P.NE);
  for (long long e = 0; e < P.NE; ++e) {
    rho[e] = d->rho0 ? d->rho0[e] : d->rho0_value;
    gam[e] = d->gamma ? d->gamma[e] : d->gamma_value;
    if (!(rho[e] > 0.0) || !(gam[e] > 1.0)) {
      delete m;
      return fail(nullptr, LH_EINVAL, "rho0 must be > 0 and gamma > 1");
    }
  }
  const std::vector<double> tab = build_tables(K);
  m->nblocks_elem = elem_grid(P);
  const long long evn = P.NE * 2 * dim * nd;
  bool ok = cudaMalloc(&m->d_rho0, sizeof(double) * P.NE) == cudaSuccess &&
            cudaMalloc(&m->d_gamma, sizeof(double) * P.NE) == cudaSuccess &&
            cudaMalloc(&m->d_tab, sizeof(double) * tab.size()) == cudaSuccess &&
            cudaMalloc(&m->d_ev, sizeof(double) * evn) == cudaSuccess &&
            cudaMalloc(&m->d_part, sizeof(double) * kRedBlocks * 72) == cudaSuccess &&
            cudaMalloc(&m->d_counter, sizeof(unsigned)) == cudaSuccess &&
            cudaMalloc(&m->d_scalar, sizeof(double) * 256) == cudaSuccess &&
            cudaMalloc(&m->d_diagMv, sizeof(double) * P.NV) == cudaSuccess &&
            cudaMalloc(&m->d_invMe, sizeof(double) * P.NEd) == cudaSuccess &&
            cudaMalloc(&m->d_blockmin, sizeof(double) * (m->nblocks_elem + 1)) == cudaSuccess;
  if (!ok) {
    lh_mesh_destroy(m);
    return fail(nullptr, LH_ENOMEM, "device allocation failed in lh_mesh_create");
  }
  if (lh::init_const_tables() != cudaSuccess) {
    lh_mesh_destroy(m);
    return fail(nullptr, LH_ECUDA, "writing the constant basis tables failed in lh_mesh_create");
  }
  P.rho0 = m->d_rho0;
  P.gamma = m->d_gamma;
  P.tab = m->d_tab;
  P.fh0 = (float)P.h0;
  P.finv_hc = (float)P.inv_hc;
  P.fq1 = (float)P.q1;
  P.fq2 = (float)P.q2;
  P.fscoef = (float)P.scoef;
  P.feps2 = (float)P.eps2;
  P.finv_detJ0 = (float)(1.0 / P.detJ0);
  std::vector<float> fc(3 * P.NE);
  for (long long i = 0; i < P.NE; ++i) {
    fc[i] = (float)(rho[i] * P.detJ0);
    fc[P.NE + i] = (float)(gam[i] - 1.0);
    fc[2 * P.NE + i] = (float)(gam[i] * (gam[i] - 1.0));
  }
  if (cudaMalloc(&m->d_fconst, sizeof(float) * 3 * P.NE) != cudaSuccess) {
    lh_mesh_destroy(m);
    return fail(nullptr, LH_ENOMEM, "device allocation failed in lh_mesh_create");
  }
  P.fmq0 = m->d_fconst;
  P.fgm1 = m->d_fconst + P.NE;
  P.fggm1 = m->d_fconst + 2 * P.NE;
  cudaError_t e = cudaMemcpyAsync(m->d_rho0, rho.data(), sizeof(double) * P.NE, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->d_gamma, gam.data(), sizeof(double) * P.NE, cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(m->d_fconst, fc.data(), sizeof(float) * fc.size(), cudaMemcpyHostToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_counter, 0, sizeof(unsigned), m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->d_scalar, 0, sizeof(double) * 256, m->stream);
  // Kronecker factors of the H1 mass inverse and the nodal rho0^(-1/2) scaling
  std::vector<std::vector<float>> kf(6);
  const int nel[3] = {P.n0, P.n1, P.n2};
  for (int a = 0; a < dim && e == cudaSuccess; ++a) {
    const bool lo = (P.bc >> (2 * a)) & 1u, hi = (P.bc >> (2 * a + 1)) & 1u;
    if (!kron_factor(tab, K, nel[a], P.h[a], false, false, kf[2 * a]) ||
        !kron_factor(tab, K, nel[a], P.h[a], lo, hi, kf[2 * a + 1])) {
      lh_mesh_destroy(m);
      return fail(nullptr, LH_EINVAL, "lh_mesh_create: singular 1D mass matrix");
    }
    const size_t bytes = sizeof(float) * kf[2 * a].size();
    if (cudaMalloc(&m->kron.At_free[a], bytes) != cudaSuccess || cudaMalloc(&m->kron.At_fixed[a], bytes) != cudaSuccess) {
      lh_mesh_destroy(m);
      return fail(nullptr, LH_ENOMEM, "device allocation failed in lh_mesh_create");
    }
    e = cudaMemcpy(m->kron.At_free[a], kf[2 * a].data(), bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(m->kron.At_fixed[a], kf[2 * a + 1].data(), bytes, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) {
    std::vector<double> sc(P.NV);
    for (long long i = 0; i < P.NV; ++i) {
      const int ic[3] = {(int)(i % P.N0), (int)((i / P.N0) % P.N1), (int)(i / ((long long)P.N0 * P.N1))};
      int lo3[3], hi3[3];
      for (int a = 0; a < 3; ++a) {
        if (a >= dim) { lo3[a] = hi3[a] = 0; continue; }
        const int q = ic[a] / K, r = ic[a] % K;
        lo3[a] = (r == 0 && q >= 1) ? q - 1 : (q < nel[a] ? q : nel[a] - 1);
        hi3[a] = (r == 0) ? (q < nel[a] ? q : nel[a] - 1) : q;
      }
      double sum = 0.0;
      int cnt = 0;
      for (int z = lo3[2]; z <= hi3[2]; ++z)
        for (int y = lo3[1]; y <= hi3[1]; ++y)
          for (int x = lo3[0]; x <= hi3[0]; ++x) {
            sum += rho[x + (long long)P.n0 * (y + (long long)P.n1 * z)];
            ++cnt;
          }
      sc[i] = 1.0 / std::sqrt(sum / cnt);
    }
    if (cudaMalloc(&m->kron.scale, sizeof(double) * P.NV) != cudaSuccess ||
        cudaMalloc(&m->kron.work, sizeof(float) * 2 * dim * P.NV) != cudaSuccess) {
      lh_mesh_destroy(m);
      return fail(nullptr, LH_ENOMEM, "device allocation failed in lh_mesh_create");
    }
    e = cudaMemcpy(m->kron.scale, sc.data(), sizeof(double) * P.NV, cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = launch_setup(P, m->stream, m->d_ev, m->d_diagMv, m->d_invMe);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    lh_mesh_destroy(m);
    return fail(nullptr, LH_ECUDA, std::string("lh_mesh_create: ") + cudaGetErrorString(e));
  }
  *out = m;
  return LH_OK;
}

lh_status lh_mesh_destroy(lh_mesh* m) {
  if (!m) return LH_OK;
  for (int i = 0; i < 2 * Prof::kMax; ++i)
    if (m->prof.ev[i]) cudaEventDestroy(m->prof.ev[i]);
  double* bufs[] = {m->d_rho0, m->d_gamma, m->d_tab, m->d_ev, m->d_part, m->d_scalar,
                    m->d_diagMv, m->d_invMe, m->d_blockmin, m->d_work};
  for (double* b : bufs)
    if (b) cudaFree(b);
  if (m->d_fwork) cudaFree(m->d_fwork);
  if (m->d_counter) cudaFree(m->d_counter);
  if (m->d_fconst) cudaFree(m->d_fconst);
  if (m->d_rec) cudaFree(m->d_rec);
  if (m->d_stage) cudaFree(m->d_stage);
  if (m->d_adv) cudaFree(m->d_adv);
  if (m->d_cheb) cudaFree(m->d_cheb);
  if (m->d_xwork) cudaFree(m->d_xwork);
  if (m->d_wscale) cudaFree(m->d_wscale);
  if (m->d_jdiag) cudaFree(m->d_jdiag);
  if (m->arn.exec) cudaGraphExecDestroy(m->arn.exec);
  if (m->arn.graph) cudaGraphDestroy(m->arn.graph);
  if (m->arn.cap) cudaStreamDestroy(m->arn.cap);
  if (m->arn.cap2) cudaStreamDestroy(m->arn.cap2);
  if (m->d_arn) cudaFree(m->d_arn);
  if (m->h_arn) cudaFreeHost(m->h_arn);
  if (m->d_vin) cudaFree(m->d_vin);
  if (m->h_small) cudaFreeHost(m->h_small);
  for (int a = 0; a < 3; ++a) {
    if (m->kron.At_free[a]) cudaFree(m->kron.At_free[a]);
    if (m->kron.At_fixed[a]) cudaFree(m->kron.At_fixed[a]);
  }
  if (m->kron.scale) cudaFree(m->kron.scale);
  if (m->kron.work) cudaFree(m->kron.work);
  delete m;
  return LH_OK;
}

lh_status lh_sizes(const lh_mesh* m, long long* out) {
  if (!m || !out) return fail(nullptr, LH_EINVAL, "NULL argument to lh_sizes");
  out[0] = m->P.NE;
  out[1] = m->P.NV;
  out[2] = m->P.NEd;
  out[3] = m->n;
  out[4] = m->NQ;
  out[5] = m->P.dim;
  return LH_OK;
}

lh_status lh_set_stream(lh_mesh* m, void* stream) {
  if (!m) return fail(nullptr, LH_EINVAL, "mesh is NULL");
  m->stream = reinterpret_cast<cudaStream_t>(stream);
  return LH_OK;
}

lh_status lh_initial_nodes(lh_mesh* m, double* x0) {
  if (!m || !x0) return fail(m, LH_EINVAL, "NULL argument to lh_initial_nodes");
  LH_CK(m, launch_initial_nodes(m->P, m->stream, x0));
  return LH_OK;
}

lh_status lh_residual(lh_mesh* m, const double* u, const double* k, double tau, double* r, double* min_detj) {
  if (!m || !u || !k || !r) return fail(m, LH_EINVAL, "NULL argument to lh_residual");
  if (r == u || r == k) return fail(m, LH_EINVAL, "r must not alias u or k");
  if (min_detj) return residual_min(m, u, k, tau, r, min_detj);
  LH_CK(m, launch_residual(m->P, m->stream, u, k, tau, m->d_ev, m->d_blockmin, r, prof_pair(m, LH_PROF_RESIDUAL)));
  return LH_OK;
}

lh_status lh_jvp(lh_mesh* m, const double* u, const double* k, double tau, const void* dk, void* out,
                 lh_prec prec) {
  if (!m || !u || !k || !dk || !out) return fail(m, LH_EINVAL, "NULL argument to lh_jvp");
  if (dk == out) return fail(m, LH_EINVAL, "out must not alias dk");
  if (prec == LH_FP64) {
    LH_CK(m, launch_jvp_f64(m->P, m->stream, u, k, tau, static_cast<const double*>(dk), m->d_ev,
                            static_cast<double*>(out), prof_pair(m, LH_PROF_JVP64)));
  } else if (prec == LH_FP32) {
    LH_CK(m, launch_jvp_f32(m->P, m->stream, u, k, tau, static_cast<const float*>(dk),
                            reinterpret_cast<float*>(m->d_ev), static_cast<float*>(out),
                            prof_pair(m, LH_PROF_JVP32)));
  } else if (prec == LH_FP32_LIN || prec == LH_TF32 || prec == LH_BF16) {
    if (!m->rec_valid || m->rec_u != u || m->rec_k != k || m->rec_tau != tau)
      return fail(m, LH_EINVAL, "lh_jvp(record precisions): call lh_linearize with the same u, k, tau first");
    if (prec == LH_FP32_LIN) {
      LH_CK(m, launch_jvp_rec_f32(m->P, m->stream, m->d_rec, tau, static_cast<const float*>(dk),
                                  reinterpret_cast<float*>(m->d_ev), static_cast<float*>(out),
                                  prof_pair(m, LH_PROF_JVP32), tc_err(m)));
    } else {
      if (!jvp_tc_supported(m->P.dim, m->P.K))
        return fail(m, LH_EINVAL, "lh_jvp: tensor-core J.w supports 2D orders 1-4 and 3D orders 1-2");
      LH_CK(m, launch_jvp_tc<float>(m->P, m->stream, prec == LH_TF32 ? 0 : 1, m->d_rec, tau,
                                    static_cast<const float*>(dk), reinterpret_cast<float*>(m->d_ev),
                                    static_cast<float*>(out), tc_err(m), prof_pair(m, LH_PROF_JVPTC)));
    }
  } else {
    return fail(m, LH_EINVAL, "lh_jvp: unsupported precision");
  }
  return LH_OK;
}

lh_status lh_linearize(lh_mesh* m, const double* u, const double* k, double tau) {
  if (!m || !u || !k) return fail(m, LH_EINVAL, "NULL argument to lh_linearize");
  lh_status st = ensure_rec(m);
  if (st != LH_OK) return st;
  if ((st = ensure_work(m, m->restart_alloc > 0 ? m->restart_alloc : 30)) != LH_OK) return st;
  double* r = m->d_work;   // residual written as a by-product
  LH_CK(m, launch_residual(m->P, m->stream, u, k, tau, m->d_ev, m->d_blockmin, r, nullptr, m->d_rec));
  m->rec_u = u;
  m->rec_k = k;
  m->rec_tau = tau;
  m->rec_valid = true;
  return LH_OK;
}

lh_status lh_jvv_diagonal(lh_mesh* m, const double* u, const double* k, double tau, double* out) {
  if (!m || !u || !k || !out) return fail(m, LH_EINVAL, "NULL argument to lh_jvv_diagonal");
  lh_status st = lh_linearize(m, u, k, tau);
  if (st != LH_OK) return st;
  LH_CK(m, launch_jvv_diag(m->P, m->stream, m->d_rec, tau, reinterpret_cast<float*>(m->d_ev), m->d_diagMv, out));
  return LH_OK;
}

lh_status lh_jtvp(lh_mesh* m, const double* u, const double* k, double tau, const void* y, void* out,
                  lh_prec prec) {
  if (!m || !u || !k || !y || !out) return fail(m, LH_EINVAL, "NULL argument to lh_jtvp");
  if (y == out) return fail(m, LH_EINVAL, "out must not alias y");
  if (prec == LH_FP32_LIN) {
    if (!m->rec_valid || m->rec_u != u || m->rec_k != k || m->rec_tau != tau)
      return fail(m, LH_EINVAL, "lh_jtvp(LH_FP32_LIN): call lh_linearize with the same u, k, tau first");
    LH_CK(m, launch_jtvp_rec_f32(m->P, m->stream, m->d_rec, tau, static_cast<const float*>(y),
                                 reinterpret_cast<float*>(m->d_ev), static_cast<float*>(out),
                                 prof_pair(m, LH_PROF_JTVP)));
    return LH_OK;
  }
  if (prec != LH_FP64) return fail(m, LH_EINVAL, "lh_jtvp supports LH_FP64 and LH_FP32_LIN");
  LH_CK(m, launch_jtvp(m->P, m->stream, u, k, tau, static_cast<const double*>(y), m->d_ev,
                       static_cast<double*>(out), prof_pair(m, LH_PROF_JTVP)));
  return LH_OK;
}

lh_status lh_mass_apply(lh_mesh* m, int which, const double* f, double* out) {
  if (!m || !f || !out) return fail(m, LH_EINVAL, "NULL argument to lh_mass_apply");
  if (which == 0) {
    LH_CK(m, launch_mass_h1(m->P, m->stream, f, m->d_ev, out, prof_pair(m, LH_PROF_MASS)));
  } else if (which == 1) {
    LH_CK(m, launch_mass_l2(m->P, m->stream, f, out));
  } else {
    return fail(m, LH_EINVAL, "which must be 0 (H1) or 1 (L2)");
  }
  return LH_OK;
}

lh_status lh_mass_solve(lh_mesh* m, int which, const double* rhs, double* sol, double rtol, int maxit,
                        int* iters) {
  if (!m || !rhs || !sol) return fail(m, LH_EINVAL, "NULL argument to lh_mass_solve");
  if (iters) *iters = 0;
  if (which == 1) {
    LH_CK(m, launch_mul(m->stream, rhs, m->d_invMe, sol, m->P.NEd));
    LH_CK(m, cudaStreamSynchronize(m->stream));
    return LH_OK;
  }
  if (which != 0) return fail(m, LH_EINVAL, "which must be 0 (H1) or 1 (L2)");
  lh_status st = ensure_work(m, m->restart_alloc > 0 ? m->restart_alloc : 30);
  if (st != LH_OK) return st;
  const long long n = (long long)m->P.dim * m->P.NV;
  double* r = m->d_work;
  double* z = r + n;
  double* p = z + n;
  double* Ap = p + n;
  LH_CK(m, cudaMemsetAsync(sol, 0, sizeof(double) * n, m->stream));
  LH_CK(m, cudaMemcpyAsync(r, rhs, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
  LH_CK(m, launch_jacobi_h1(m->stream, m->P.NV, m->P.dim, m->d_diagMv, r, z));
  LH_CK(m, cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, m->stream));
  double rz, bb, pAp, rr;
  if ((st = dot_host(m, r, z, n, &rz)) != LH_OK) return st;
  if ((st = dot_host(m, r, r, n, &bb)) != LH_OK) return st;
  if (bb == 0.0) return LH_OK;
  int it = 0;
  bool conv = false;
  for (; it < maxit; ++it) {
    LH_CK(m, launch_mass_h1(m->P, m->stream, p, m->d_ev, Ap, prof_pair(m, LH_PROF_MASS)));
    if ((st = dot_host(m, p, Ap, n, &pAp)) != LH_OK) return st;
    const double alpha = rz / pAp;
    LH_CK(m, launch_axpby(m->stream, alpha, p, 1.0, sol, n));
    LH_CK(m, launch_axpby(m->stream, -alpha, Ap, 1.0, r, n));
    if ((st = dot_host(m, r, r, n, &rr)) != LH_OK) return st;
    if (std::sqrt(rr) <= rtol * std::sqrt(bb)) {
      conv = true;
      ++it;
      break;
    }
    LH_CK(m, launch_jacobi_h1(m->stream, m->P.NV, m->P.dim, m->d_diagMv, r, z));
    double rz_new;
    if ((st = dot_host(m, r, z, n, &rz_new)) != LH_OK) return st;
    LH_CK(m, launch_axpby(m->stream, 1.0, z, rz_new / rz, p, n));
    rz = rz_new;
  }
  if (iters) *iters = it;
  return conv ? LH_OK : fail(m, LH_ENOCONV, "lh_mass_solve: CG reached maxit");
}

lh_status lh_precond(lh_mesh* m, int kind, double tau, const double* r, double* z) {
  if (!m || !r || !z) return fail(m, LH_EINVAL, "NULL argument to lh_precond");
  if (r == z) return fail(m, LH_EINVAL, "z must not alias r");
  if (kind != 0 && kind != 1) return fail(m, LH_EINVAL, "kind must be 0 or 1");
  LH_CK(m, (launch_prec<double, double>(kind, m->stream, m->P, m->kron, m->d_diagMv, m->d_invMe, r, z, tau)));
  return LH_OK;
}

lh_status lh_dt_estimate(lh_mesh* m, const double* u, double* dt) {
  if (!m || !u || !dt) return fail(m, LH_EINVAL, "NULL argument to lh_dt_estimate");
  LH_CK(m, launch_dt_estimate(m->P, m->stream, u, m->d_blockmin));
  LH_CK(m, launch_min(m->stream, m->d_blockmin, m->nblocks_elem, m->d_scalar + 2));
  LH_CK(m, cudaMemcpyAsync(dt, m->d_scalar + 2, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return LH_OK;
}

lh_status lh_energies(lh_mesh* m, const double* u, double* kinetic, double* internal) {
  if (!m || !u || !kinetic || !internal) return fail(m, LH_EINVAL, "NULL argument to lh_energies");
  lh_status st = ensure_work(m, m->restart_alloc > 0 ? m->restart_alloc : 30);
  if (st != LH_OK) return st;
  const long long n1 = (long long)m->P.dim * m->P.NV;
  double* t = m->d_work;
  LH_CK(m, launch_mass_h1(m->P, m->stream, u + n1, m->d_ev, t));
  double kv;
  if ((st = dot_host(m, u + n1, t, n1, &kv)) != LH_OK) return st;
  *kinetic = 0.5 * kv;
  LH_CK(m, launch_mass_l2(m->P, m->stream, u + 2 * n1, t));
  LH_CK(m, launch_mdot<double>(m->stream, t, 1, 0, nullptr, m->P.NEd, 0, m->d_part, m->d_counter, m->d_scalar));
  LH_CK(m, cudaMemcpyAsync(internal, m->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return LH_OK;
}

lh_status lh_tg_velocity_error(lh_mesh* m, const double* u, double* l1) {
  if (!m || !u || !l1) return fail(m, LH_EINVAL, "NULL argument to lh_tg_velocity_error");
  if (m->P.dim != 2) return fail(m, LH_EINVAL, "lh_tg_velocity_error: the Taylor-Green velocity is 2D");
  lh_status st = ensure_work(m, m->restart_alloc > 0 ? m->restart_alloc : 30);
  if (st != LH_OK) return st;
  double* t = m->d_work;   // NE (2k)^2 terms, fewer than the n = 4 NV + k^2 NE of the work buffer
  LH_CK(m, launch_tg_error(m->P, m->stream, u, t));
  LH_CK(m, launch_mdot<double>(m->stream, t, 1, 0, nullptr, tg_error_terms(m->P), 0, m->d_part, m->d_counter,
                               m->d_scalar));
  LH_CK(m, cudaMemcpyAsync(l1, m->d_scalar, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return LH_OK;
}

static lh_status check_newton_opts(lh_mesh* m, const lh_newton_opts& o) {
  if (o.restart < 1 || o.restart > 64) return fail(m, LH_EINVAL, "restart must be in 1..64");
  if (o.jvp_prec != LH_FP64 && o.jvp_prec != LH_FP32 && o.jvp_prec != LH_TF32 && o.jvp_prec != LH_BF16)
    return fail(m, LH_EINVAL, "unsupported jvp_prec");
  if ((o.jvp_prec == LH_TF32 || o.jvp_prec == LH_BF16) && !jvp_tc_supported(m->P.dim, m->P.K))
    return fail(m, LH_EINVAL, "tensor-core J.w supports 2D orders 1-4 and 3D orders 1-2");
  if (o.precond < 0 || o.precond > 3) return fail(m, LH_EINVAL, "precond must be 0, 1, 2 or 3");
  if (o.precond >= 2 && o.jvp_prec == LH_FP64)
    return fail(m, LH_EINVAL, "precond 2 and 3 (velocity block) need a reduced-precision J.w");
  if (o.precond == 3 && (o.cheb_degree < 1 || o.cheb_degree > 16 || !(o.cheb_ratio > 1.0)))
    return fail(m, LH_EINVAL, "precond 3: need 1 <= cheb_degree <= 16 and cheb_ratio > 1");
  if (o.arnoldi != 0 && o.arnoldi != 1) return fail(m, LH_EINVAL, "arnoldi must be 0 or 1");
  if (o.forcing != 0 && o.forcing != 1) return fail(m, LH_EINVAL, "forcing must be 0 or 1");
  if (o.forcing && !(o.eta_max >= o.gmres_rtol && o.eta_max < 1.0))
    return fail(m, LH_EINVAL, "eta_max must be in [gmres_rtol, 1)");
  if (o.scaled_norm != 0 && o.scaled_norm != 1) return fail(m, LH_EINVAL, "scaled_norm must be 0 or 1");
  return ensure_work(m, o.restart);
}

// Inexact Newton-GMRES on the stage system R(k; tau, u) = 0 (Eqs. (21)-(22), Sec. 3.5) from
// the initial guess k_init (device [n], or NULL for zero).  Fills S.  On LH_OK *k_out points
// at the converged k inside the mesh's work buffer (overwritten by the next solve); a solve
// that ends without convergence returns LH_ENOCONV with S filled.
static lh_status newton_solve(lh_mesh* m, const double* u, const double* k_init, double tau,
                              const lh_newton_opts& o, lh_step_stats& S, const double** k_out) {
  lh_status st;
  const bool f32 = o.jvp_prec != LH_FP64;
  const int tck = o.jvp_prec == LH_TF32 ? 0 : o.jvp_prec == LH_BF16 ? 1 : -1;
  float* rec = nullptr;
  if (f32) {
    if ((st = ensure_rec(m)) != LH_OK) return st;
    rec = m->d_rec;
  }
  m->rec_valid = false;   // the record will describe this solve's internal iterates
  // on a failure of a solve with the record J.w, a bounded wait of that kernel that ran out
  // (its rows are then NaN) is the cause to report
  auto wait_status = [&](lh_status failed) {
    if (f32 && tck < 0) {
      const lh_status t = lh_tc_status(m);
      if (t != LH_OK) return t;
    }
    return failed;
  };
  std::memset(&S, 0, sizeof(S));
  const long long n = m->n;
  const int mres = o.restart;
  cudaStream_t s = m->stream;
  double* V = m->d_work;                      // (mres + 1) x n FP64 Krylov basis
  double* k = V + (long long)(mres + 1) * n;  // Newton iterate
  double* r = k + n;                          // residual at k
  double* dk = r + n;                         // Newton correction
  double* zd = dk + n;                        // double scratch
  double* wd = zd + n;                        // double scratch
  double* kt = wd + n;                        // trial iterate
  double* rt = kt + n;                        // residual at the trial
  double* rs = rt + n;                        // row-weighted residual (scaled_norm)
  const long long ldf = m->ldf;
  float* Vf = m->d_fwork;                     // (mres + 1) x ldf FP32 Krylov basis
  float* wf = Vf + (long long)(mres + 1) * ldf;
  float* zf = wf + ldf;
  float* uf = zf + ldf;

  if (o.precond >= 2 && !m->d_jdiag &&
      cudaMalloc(&m->d_jdiag, sizeof(double) * (size_t)m->P.dim * m->P.NV) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate the velocity-block diagonal");
  if (o.precond == 3 && !m->d_cheb && cudaMalloc(&m->d_cheb, sizeof(float) * 5 * (size_t)ldf) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate the Chebyshev work vectors");
  const double* wsc = nullptr;
  if (o.scaled_norm) {
    if (!m->d_wscale) {
      if (cudaMalloc(&m->d_wscale, sizeof(double) * n) != cudaSuccess)
        return fail(m, LH_ENOMEM, "cannot allocate the residual row weights");
      LH_CK(m, launch_row_weights(m->P, s, m->d_diagMv, m->d_invMe, m->d_wscale));
    }
    wsc = m->d_wscale;
  }
  // squared norm of the stopping test: ||x||_2^2, or ||W x||_2^2 with scaled_norm (W x left in rs)

  if (k_init) {
    LH_CK(m, cudaMemcpyAsync(k, k_init, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  } else {
    LH_CK(m, cudaMemsetAsync(k, 0, sizeof(double) * n, s));
  }
  double mind, nr2;
  if ((st = residual_min_norm(m, u, k, tau, r, &mind, &nr2, rec, wsc, rs)) != LH_OK) return st;
  ++S.residual_evals;
  if (!(mind > 0.0) && k_init) {   // a tangled initial guess: restart from k = 0
    LH_CK(m, cudaMemsetAsync(k, 0, sizeof(double) * n, s));
    if ((st = residual_min_norm(m, u, k, tau, r, &mind, &nr2, rec, wsc, rs)) != LH_OK) return st;
    ++S.residual_evals;
  }
  if (!(mind > 0.0)) return fail(m, LH_ETANGLED, "Newton: det J <= 0 at the initial guess");
  double nr = std::sqrt(nr2);
  if (!std::isfinite(nr)) return fail(m, LH_ENONFINITE, "Newton: non-finite residual");
  S.r0 = nr;
  bool conv = nr <= std::fmax(o.newton_rtol * S.r0, o.newton_atol);
  double eta = o.forcing ? o.eta_max : o.gmres_rtol;   // relative tolerance of the next solve
  const double target = std::fmax(o.newton_rtol * S.r0, o.newton_atol);
  for (int it = 0; it < o.newton_maxit && !conv; ++it) {
    // ---- linear solve J dk = -r (Eq. (22)) at the current iterate k
    lh_newton_opts oi = o;
    oi.gmres_rtol = eta;
    if (o.precond >= 2)   // the record describes the current iterate k (its last residual)
      LH_CK(m, launch_jvv_diag(m->P, s, rec, tau, reinterpret_cast<float*>(m->d_ev), m->d_diagMv, m->d_jdiag,
                               kJvvFloor));
    if (o.precond == 3 && (st = cheb_bounds(m, o, tau, tck, zd)) != LH_OK) return wait_status(st);
    const double* rhs = r;   // with scaled_norm GMRES solves W J dk = -W r
    if (wsc) {
      LH_CK(m, launch_row_mul<double>(s, wsc, r, rs, n));
      rhs = rs;
    }
    if (f32) {
      KrylovOp<float> op{m, o.precond, tck, u, k, tau, zf};
      op.wsc = wsc;
      if ((st = gmres<float>(m, oi, op, rhs, nr, dk, Vf, wf, uf, zd, wd, S)) != LH_OK) return wait_status(st);
    } else {
      KrylovOp<double> op{m, o.precond, -1, u, k, tau, zd};
      op.wsc = wsc;
      if ((st = gmres<double>(m, oi, op, rhs, nr, dk, V, wd, wd, zd, wd, S)) != LH_OK) return st;
    }
    const double nr_prev = nr;
    // ---- backtracking line search on det J > 0 (Sec. 3.5)
    double lam = 1.0;
    bool accepted = false;
    for (int hlv = 0; hlv <= o.max_halvings; ++hlv) {
      LH_CK(m, cudaMemcpyAsync(kt, k, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      LH_CK(m, launch_axpby(s, lam, dk, 1.0, kt, n));
      if ((st = residual_min_norm(m, u, kt, tau, rt, &mind, &nr2, rec, wsc, rs)) != LH_OK) return st;
      ++S.residual_evals;
      if (mind > 0.0) {   // reject tangled trials (Sec. 3.5) and, as well, non-finite ones
        if (std::isfinite(nr2)) {
          accepted = true;
          break;
        }
      }
      lam *= 0.5;
      ++S.backtracks;
    }
    if (!accepted) return wait_status(fail(m, LH_ETANGLED, "Newton: line search found no trial with det J > 0 "
                                                           "and a finite residual"));
    std::swap(k, kt);
    std::swap(r, rt);
    nr = std::sqrt(nr2);
    S.min_detj = mind;
    ++S.newton_its;
    conv = nr <= target;
    if (o.forcing && !conv) {   // Eisenstat-Walker choice 2 with safeguards
      double e = 0.9 * (nr / nr_prev) * (nr / nr_prev);
      const double prev = 0.9 * eta * eta;
      if (prev > 0.1) e = std::fmax(e, prev);
      e = std::fmax(e, 0.5 * target / nr);
      eta = std::fmax(std::fmin(e, o.eta_max), o.gmres_rtol);
    }
  }
  S.rfinal = nr;
  S.newton_its_max = S.newton_its;
  if (S.min_detj == 0.0) S.min_detj = mind;
  if (tck >= 0 && (st = lh_tc_status(m)) != LH_OK) return st;
  *k_out = k;
  if (!conv) return wait_status(fail(m, LH_ENOCONV, "Newton did not converge"));
  return LH_OK;
}

lh_status lh_newton_step(lh_mesh* m, double* u, double* k_prev, double dt, const lh_newton_opts* opts_in,
                         lh_step_stats* stats) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_newton_step");
  lh_newton_opts o;
  if (opts_in) o = *opts_in; else lh_newton_opts_init(&o);
  if (!(dt > 0.0)) return fail(m, LH_EINVAL, "dt must be > 0");
  lh_status st = check_newton_opts(m, o);
  if (st != LH_OK) return st;
  lh_step_stats S;
  const double* k = nullptr;
  st = newton_solve(m, u, k_prev, 0.5 * dt, o, S, &k);
  if (st == LH_OK || st == LH_ENOCONV) {
    if (stats) *stats = S;
  }
  if (st != LH_OK) return st;
  cudaStream_t s = m->stream;
  LH_CK(m, launch_axpby(s, dt, k, 1.0, u, m->n));
  if (k_prev) LH_CK(m, cudaMemcpyAsync(k_prev, k, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, s));
  LH_CK(m, cudaStreamSynchronize(s));
  return LH_OK;
}

lh_status lh_stage_solve(lh_mesh* m, const double* u_base, double* k, double tau, const lh_newton_opts* opts_in,
                         lh_step_stats* stats) {
  if (!m || !u_base || !k) return fail(m, LH_EINVAL, "NULL argument to lh_stage_solve");
  if (k == u_base) return fail(m, LH_EINVAL, "lh_stage_solve: k must not alias u_base");
  if (!(tau > 0.0)) return fail(m, LH_EINVAL, "tau must be > 0");
  lh_newton_opts o;
  if (opts_in) o = *opts_in; else lh_newton_opts_init(&o);
  lh_status st = check_newton_opts(m, o);
  if (st != LH_OK) return st;
  lh_step_stats S;
  const double* kc = nullptr;
  st = newton_solve(m, u_base, k, tau, o, S, &kc);
  if (st == LH_OK || st == LH_ENOCONV) {
    if (stats) *stats = S;
  }
  if (st != LH_OK) return st;
  LH_CK(m, cudaMemcpyAsync(k, kc, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return LH_OK;
}

namespace {

// Butcher tableaux of the SDIRK schemes of Sec. 4 (SD2/SD3/SD4): A lower triangular with
// the common diagonal gamma, weights b.  SD3: Alexander's 3-stage L-stable, stiffly accurate
// method of order 3, gamma the root in (1/6, 1/2) of g^3 - 3 g^2 + 3/2 g - 1/6 = 0.  SD4:
// Crouzeix's 3-stage A-stable method of order 4, gamma = 1/2 + cos(pi/18)/sqrt(3).
struct Tableau {
  int s = 0;
  double a[3][3] = {};
  double b[3] = {};
};

bool sdirk_tableau(int scheme, Tableau* t) {
  *t = Tableau();
  if (scheme == 2) {
    t->s = 1;
    t->a[0][0] = 0.5;
    t->b[0] = 1.0;
    return true;
  }
  if (scheme == 3) {
    double g = 0.45;   // Newton on the cubic; the root is simple and 0.45 lies in its basin
    for (int it = 0; it < 50; ++it) {
      const double f = ((g - 3.0) * g + 1.5) * g - 1.0 / 6.0;
      const double df = (3.0 * g - 6.0) * g + 1.5;
      const double d = f / df;
      g -= d;
      if (std::fabs(d) < 1e-17) break;
    }
    t->s = 3;
    t->a[0][0] = t->a[1][1] = t->a[2][2] = g;
    t->a[1][0] = 0.5 * (1.0 - g);
    t->a[2][0] = t->b[0] = -0.25 * ((6.0 * g - 16.0) * g + 1.0);
    t->a[2][1] = t->b[1] = 0.25 * ((6.0 * g - 20.0) * g + 5.0);
    t->b[2] = g;
    return true;
  }
  if (scheme == 4) {
    const double pi = 3.14159265358979323846;
    const double g = 0.5 + std::cos(pi / 18.0) / std::sqrt(3.0);
    const double d = 1.0 / (6.0 * (2.0 * g - 1.0) * (2.0 * g - 1.0));
    t->s = 3;
    t->a[0][0] = t->a[1][1] = t->a[2][2] = g;
    t->a[1][0] = 0.5 - g;
    t->a[2][0] = 2.0 * g;
    t->a[2][1] = 1.0 - 4.0 * g;
    t->b[0] = t->b[2] = d;
    t->b[1] = 1.0 - 2.0 * d;
    return true;
  }
  return false;
}

void merge_stats(lh_step_stats& acc, const lh_step_stats& st, bool first) {
  acc.newton_its += st.newton_its;
  acc.gmres_its_total += st.gmres_its_total;
  acc.backtracks += st.backtracks;
  acc.residual_evals += st.residual_evals;
  acc.jvp_evals += st.jvp_evals;
  acc.reorth += st.reorth;
  acc.newton_its_max = std::max(acc.newton_its_max, st.newton_its);
  acc.r0 = first ? st.r0 : std::fmax(acc.r0, st.r0);
  acc.rfinal = first ? st.rfinal : std::fmax(acc.rfinal, st.rfinal);
  acc.min_detj = first ? st.min_detj : std::fmin(acc.min_detj, st.min_detj);
}

}  // namespace

lh_status lh_sdirk_tableau(int scheme, int* stages, double* A, double* b) {
  if (!stages || !A || !b) return set_global_error(LH_EINVAL, "NULL argument to lh_sdirk_tableau");
  Tableau T;
  if (!sdirk_tableau(scheme, &T)) return set_global_error(LH_EINVAL, "scheme must be 2, 3 or 4");
  *stages = T.s;
  for (int i = 0; i < 3; ++i) {
    b[i] = T.b[i];
    for (int j = 0; j < 3; ++j) A[3 * i + j] = T.a[i][j];
  }
  return LH_OK;
}

lh_status lh_sdirk_step(lh_mesh* m, int scheme, double* u, double* k_prev, double dt,
                        const lh_newton_opts* opts_in, lh_step_stats* stats) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_sdirk_step");
  Tableau T;
  if (!sdirk_tableau(scheme, &T)) return fail(m, LH_EINVAL, "scheme must be 2, 3 or 4");
  if (!(dt > 0.0)) return fail(m, LH_EINVAL, "dt must be > 0");
  lh_newton_opts o;
  if (opts_in) o = *opts_in; else lh_newton_opts_init(&o);
  lh_status st = check_newton_opts(m, o);
  if (st != LH_OK) return st;
  const long long n = m->n;
  if (!m->d_stage && cudaMalloc(&m->d_stage, sizeof(double) * 4 * (size_t)n) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate the SDIRK stage vectors");
  cudaStream_t s = m->stream;
  double* K[3] = {m->d_stage, m->d_stage + n, m->d_stage + 2 * n};
  double* base = m->d_stage + 3 * n;
  lh_step_stats acc;
  std::memset(&acc, 0, sizeof(acc));
  for (int i = 0; i < T.s; ++i) {
    // stage base state u + dt sum_{j<i} a_ij k_j; the first stage starts from u itself
    const double* ub = u;
    if (i > 0) {
      LH_CK(m, cudaMemcpyAsync(base, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      for (int j = 0; j < i; ++j) LH_CK(m, launch_axpby(s, dt * T.a[i][j], K[j], 1.0, base, n));
      ub = base;
    }
    const double* guess = i == 0 ? k_prev : K[i - 1];
    lh_step_stats Si;
    const double* kc = nullptr;
    st = newton_solve(m, ub, guess, dt * T.a[i][i], o, Si, &kc);
    if (st == LH_OK || st == LH_ENOCONV) merge_stats(acc, Si, i == 0);
    if (st != LH_OK) {
      if (st == LH_ENOCONV && stats) *stats = acc;
      return st;
    }
    LH_CK(m, cudaMemcpyAsync(K[i], kc, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  }
  for (int i = 0; i < T.s; ++i) LH_CK(m, launch_axpby(s, dt * T.b[i], K[i], 1.0, u, n));
  if (k_prev) LH_CK(m, cudaMemcpyAsync(k_prev, K[T.s - 1], sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  LH_CK(m, cudaStreamSynchronize(s));
  if (stats) *stats = acc;
  return LH_OK;
}

}  // extern "C"

// ---- explicit path ------------------------------------------------------------------------
namespace {

bool check_explicit_opts(const lh_explicit_opts& o, std::string* why) {
  if (o.scheme < 2 || o.scheme > 4) return *why = "scheme must be 2, 3 or 4", false;
  if (o.visc_model != 0 && o.visc_model != 1) return *why = "visc_model must be 0 or 1", false;
  if (!(o.q1_exp >= 0.0) || !(o.q2_exp >= 0.0) || !(o.l0_exp >= 0.0)) return *why = "negative mu_exp parameter", false;
  if (!(o.cfl > 0.0)) return *why = "cfl must be > 0", false;
  if (!(o.mass_rtol > 0.0) || o.mass_maxit < 1) return *why = "need mass_rtol > 0, mass_maxit >= 1", false;
  return true;
}

lh::ExpC exp_consts(const lh_mesh* m, const lh_explicit_opts& o) {
  lh::ExpC X;
  X.l0 = o.l0_exp > 0.0 ? o.l0_exp : m->P.h0 / m->P.K;
  X.q1 = o.q1_exp;
  X.q2 = o.q2_exp;
  for (int c = 0; c < 3; ++c) X.inv_h[c] = 1.0 / m->P.h[c];
  X.vorticity = o.vorticity;
  return X;
}

// explicit work arrays (lazily): S [NQ dim^2], f1, a, w1, w2, p, Ap [dim NV each],
// fe, de, b [NEd each], r_full, z_full, U_i, u_save, K_1..K_4 [n each]
struct XWork {
  double *Sq, *f1, *a, *w1, *w2, *p, *Ap, *fe, *de, *b, *rf, *zf, *Ui, *usave, *K[4];
};

lh_status xwork(lh_mesh* m, XWork* W) {
  const long long n = m->n, n1 = (long long)m->P.dim * m->P.NV, ne = m->P.NEd;
  const long long nsq = m->NQ * m->P.dim * m->P.dim;
  const long long need = nsq + 6 * n1 + 3 * ne + 8 * n;
  if (!m->d_xwork) {
    if (cudaMalloc(&m->d_xwork, sizeof(double) * (size_t)need) != cudaSuccess)
      return fail(m, LH_ENOMEM, "cannot allocate the explicit work arrays");
  }
  double* q = m->d_xwork;
  W->Sq = q; q += nsq;
  W->f1 = q; q += n1;
  W->a = q; q += n1;
  W->w1 = q; q += n1;
  W->w2 = q; q += n1;
  W->p = q; q += n1;
  W->Ap = q; q += n1;
  W->fe = q; q += ne;
  W->de = q; q += ne;
  W->b = q; q += ne;
  W->rf = q; q += n;
  W->zf = q; q += n;
  W->Ui = q; q += n;
  W->usave = q; q += n;
  for (int i = 0; i < 4; ++i) { W->K[i] = q; q += n; }
  return LH_OK;
}

// F's point data and F.1 at u (and b); with est non-NULL also the explicit estimate (sync)
lh_status x_force(lh_mesh* m, const lh_explicit_opts& o, const XWork& W, const double* u, double* est,
                  lh_explicit_stats* S) {
  const lh::ExpC X = exp_consts(m, o);
  LH_CK(m, launch_force(m->P, m->stream, o.visc_model, X, u, W.Sq, m->d_ev, W.f1, m->P.tg ? W.b : nullptr,
                        est ? m->d_blockmin : nullptr));
  if (S) ++S->force_evals;
  if (est) {
    LH_CK(m, launch_min(m->stream, m->d_blockmin, m->nblocks_elem, m->d_scalar + 2));
    LH_CK(m, cudaMemcpyAsync(est, m->d_scalar + 2, sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    LH_CK(m, cudaStreamSynchronize(m->stream));
  }
  return LH_OK;
}

// a = -M_V^-1 f1 on free rows (0 on fixed rows): CG preconditioned with the Kronecker
// inverse (lh_precond kind 1 applied to a state-shaped vector whose x and e rows are zero)
lh_status x_accel(lh_mesh* m, const lh_explicit_opts& o, const XWork& W, lh_explicit_stats* S) {
  cudaStream_t s = m->stream;
  const long long n = m->n, n1 = (long long)m->P.dim * m->P.NV;
  double* r = W.rf + n1;
  double* z = W.zf + n1;
  LH_CK(m, cudaMemsetAsync(W.rf, 0, sizeof(double) * n, s));
  LH_CK(m, launch_axpby(s, -1.0, W.f1, 0.0, r, n1));
  LH_CK(m, launch_copy_fixed(m->P, s, nullptr, r));
  LH_CK(m, cudaMemsetAsync(W.a, 0, sizeof(double) * n1, s));
  double bb, rz, pAp, rr;
  lh_status st;
  if ((st = dot_host(m, r, r, n1, &bb)) != LH_OK) return st;
  if (bb == 0.0) return LH_OK;
  LH_CK(m, (launch_prec<double, double>(1, s, m->P, m->kron, m->d_diagMv, m->d_invMe, W.rf, W.zf, 0.0)));
  LH_CK(m, cudaMemcpyAsync(W.p, z, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
  if ((st = dot_host(m, r, z, n1, &rz)) != LH_OK) return st;
  for (int it = 0; it < o.mass_maxit; ++it) {
    LH_CK(m, launch_mass_h1(m->P, s, W.p, m->d_ev, W.Ap));
    LH_CK(m, launch_copy_fixed(m->P, s, W.p, W.Ap));
    if ((st = dot_host(m, W.p, W.Ap, n1, &pAp)) != LH_OK) return st;
    const double alpha = rz / pAp;
    LH_CK(m, launch_axpby(s, alpha, W.p, 1.0, W.a, n1));
    LH_CK(m, launch_axpby(s, -alpha, W.Ap, 1.0, r, n1));
    if (S) ++S->mass_iters;
    if ((st = dot_host(m, r, r, n1, &rr)) != LH_OK) return st;
    if (std::sqrt(rr) <= o.mass_rtol * std::sqrt(bb)) return LH_OK;
    LH_CK(m, (launch_prec<double, double>(1, s, m->P, m->kron, m->d_diagMv, m->d_invMe, W.rf, W.zf, 0.0)));
    double rz2;
    if ((st = dot_host(m, r, z, n1, &rz2)) != LH_OK) return st;
    LH_CK(m, launch_axpby(s, 1.0, z, rz2 / rz, W.p, n1));
    rz = rz2;
  }
  return fail(m, LH_ENOCONV, "explicit step: the M_V solve did not reach mass_rtol");
}

// de = M_E^-1 (F^T w + b) from the stored point data
lh_status x_edot(lh_mesh* m, const XWork& W, const double* w, double* de) {
  LH_CK(m, launch_force_t(m->P, m->stream, W.Sq, w, m->P.tg ? W.b : nullptr, W.fe));
  LH_CK(m, launch_mul(m->stream, m->d_invMe, W.fe, de, m->P.NEd));
  return LH_OK;
}

// one explicit step in place on u; force_ready: F's data at u are already in W
lh_status x_step(lh_mesh* m, double* u, double dt, const lh_explicit_opts& o, const XWork& W, bool force_ready,
                 lh_explicit_stats* S) {
  cudaStream_t s = m->stream;
  const long long n = m->n, n1 = (long long)m->P.dim * m->P.NV, ne = m->P.NEd;
  lh_status st;
  if (o.scheme == 2) {   // RK2-average
    double* uh = W.Ui;
    if (!force_ready && (st = x_force(m, o, W, u, nullptr, S)) != LH_OK) return st;
    if ((st = x_accel(m, o, W, S)) != LH_OK) return st;
    double* vh = uh + n1;
    LH_CK(m, cudaMemcpyAsync(vh, u + n1, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
    LH_CK(m, launch_axpby(s, 0.5 * dt, W.a, 1.0, vh, n1));
    if ((st = x_edot(m, W, vh, W.de)) != LH_OK) return st;
    LH_CK(m, cudaMemcpyAsync(uh, u, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
    LH_CK(m, launch_axpby(s, 0.5 * dt, vh, 1.0, uh, n1));
    LH_CK(m, cudaMemcpyAsync(uh + 2 * n1, u + 2 * n1, sizeof(double) * ne, cudaMemcpyDeviceToDevice, s));
    LH_CK(m, launch_axpby(s, 0.5 * dt, W.de, 1.0, uh + 2 * n1, ne));
    if ((st = x_force(m, o, W, uh, nullptr, S)) != LH_OK) return st;
    if ((st = x_accel(m, o, W, S)) != LH_OK) return st;
    double* vbar = W.w1;
    LH_CK(m, cudaMemcpyAsync(vbar, u + n1, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
    LH_CK(m, launch_axpby(s, 0.5 * dt, W.a, 1.0, vbar, n1));
    if ((st = x_edot(m, W, vbar, W.de)) != LH_OK) return st;
    LH_CK(m, launch_axpby(s, dt, vbar, 1.0, u, n1));
    LH_CK(m, launch_axpby(s, dt, W.a, 1.0, u + n1, n1));
    LH_CK(m, launch_axpby(s, dt, W.de, 1.0, u + 2 * n1, ne));
    return LH_OK;
  }
  // RK3 SSP / RK4 on dU/dt = (v, a(U), g(U, v)); Butcher tableaux (explicit, lower triangular)
  static const double A3[3][3] = {{0, 0, 0}, {1, 0, 0}, {0.25, 0.25, 0}};
  static const double b3[3] = {1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0};
  static const double A4[4][4] = {{0, 0, 0, 0}, {0.5, 0, 0, 0}, {0, 0.5, 0, 0}, {0, 0, 1, 0}};
  static const double b4[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
  const int ns = o.scheme == 3 ? 3 : 4;
  for (int i = 0; i < ns; ++i) {
    const double* Ui = u;
    if (i > 0) {
      LH_CK(m, cudaMemcpyAsync(W.Ui, u, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
      for (int j = 0; j < i; ++j) {
        const double aij = o.scheme == 3 ? A3[i][j] : A4[i][j];
        if (aij != 0.0) LH_CK(m, launch_axpby(s, dt * aij, W.K[j], 1.0, W.Ui, n));
      }
      Ui = W.Ui;
    }
    if (!(i == 0 && force_ready) && (st = x_force(m, o, W, Ui, nullptr, S)) != LH_OK) return st;
    if ((st = x_accel(m, o, W, S)) != LH_OK) return st;
    LH_CK(m, cudaMemcpyAsync(W.K[i], Ui + n1, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
    LH_CK(m, cudaMemcpyAsync(W.K[i] + n1, W.a, sizeof(double) * n1, cudaMemcpyDeviceToDevice, s));
    if ((st = x_edot(m, W, Ui + n1, W.K[i] + 2 * n1)) != LH_OK) return st;
  }
  for (int i = 0; i < ns; ++i) LH_CK(m, launch_axpby(s, dt * (o.scheme == 3 ? b3[i] : b4[i]), W.K[i], 1.0, u, n));
  return LH_OK;
}

lh_status x_prepare(lh_mesh* m, const lh_explicit_opts* in, lh_explicit_opts* o, XWork* W) {
  if (in) *o = *in; else lh_explicit_opts_init(o);
  std::string why;
  if (!check_explicit_opts(*o, &why)) return fail(m, LH_EINVAL, "explicit path: " + why);
  lh_status st = ensure_work(m, m->restart_alloc > 0 ? m->restart_alloc : 30);
  if (st != LH_OK) return st;
  return xwork(m, W);
}

lh_status finite_or_restore(lh_mesh* m, double* u, const double* usave) {
  double nrm;
  lh_status st = dot_host(m, u, u, m->n, &nrm);
  if (st != LH_OK) return st;
  if (std::isfinite(nrm)) return LH_OK;
  LH_CK(m, cudaMemcpyAsync(u, usave, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  return fail(m, LH_ENONFINITE, "explicit step: the new state is not finite");
}

}  // namespace

extern "C" {

void lh_explicit_opts_init(lh_explicit_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->scheme = 2;
  o->visc_model = 1;
  o->q1_exp = 0.5;
  o->q2_exp = 2.0;
  o->cfl = 0.5;
  o->mass_rtol = 1e-13;
  o->mass_maxit = 200;
}

lh_status lh_force(lh_mesh* m, const double* u, const double* w, const lh_explicit_opts* opts, double* f1,
                   double* ftw, double* dt_est) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_force");
  lh_explicit_opts o;
  XWork W;
  lh_status st = x_prepare(m, opts, &o, &W);
  if (st != LH_OK) return st;
  if ((st = x_force(m, o, W, u, dt_est, nullptr)) != LH_OK) return st;
  const long long n1 = (long long)m->P.dim * m->P.NV;
  if (f1) LH_CK(m, cudaMemcpyAsync(f1, W.f1, sizeof(double) * n1, cudaMemcpyDeviceToDevice, m->stream));
  if (ftw) LH_CK(m, launch_force_t(m->P, m->stream, W.Sq, w ? w : u + n1, m->P.tg ? W.b : nullptr, ftw));
  return LH_OK;
}

lh_status lh_explicit_step(lh_mesh* m, double* u, double dt, const lh_explicit_opts* opts, lh_explicit_stats* stats) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_explicit_step");
  if (!(dt > 0.0)) return fail(m, LH_EINVAL, "dt must be > 0");
  lh_explicit_opts o;
  XWork W;
  lh_status st = x_prepare(m, opts, &o, &W);
  if (st != LH_OK) return st;
  lh_explicit_stats S;
  std::memset(&S, 0, sizeof(S));
  LH_CK(m, cudaMemcpyAsync(W.usave, u, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
  st = x_step(m, u, dt, o, W, false, &S);
  if (st == LH_ENOCONV) {
    LH_CK(m, cudaMemcpyAsync(u, W.usave, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
    LH_CK(m, cudaStreamSynchronize(m->stream));
  }
  if (st == LH_OK) st = finite_or_restore(m, u, W.usave);
  S.steps = st == LH_OK ? 1 : 0;
  S.t = st == LH_OK ? dt : 0.0;
  S.dt_last = dt;
  if (stats) *stats = S;
  return st;
}

lh_status lh_explicit_advance(lh_mesh* m, double* u, double t_end, int max_steps, const lh_explicit_opts* opts,
                              lh_explicit_stats* stats) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_explicit_advance");
  if (!(t_end >= 0.0) || max_steps < 1) return fail(m, LH_EINVAL, "need t_end >= 0 and max_steps >= 1");
  lh_explicit_opts o;
  XWork W;
  lh_status st = x_prepare(m, opts, &o, &W);
  if (st != LH_OK) return st;
  lh_explicit_stats S;
  std::memset(&S, 0, sizeof(S));
  double est = 0.0;
  if ((st = x_force(m, o, W, u, &est, &S)) != LH_OK) return st;
  bool ready = true;   // W holds F's data at u
  double dt = o.cfl * est;
  const double t_tol = 1e-14 * std::fmax(1.0, t_end);
  while (S.t < t_end - t_tol && S.steps < max_steps) {
    if (!(dt > 0.0) || !std::isfinite(dt)) {
      st = fail(m, LH_ENONFINITE, "explicit advance: the time-step estimate is not positive");
      break;
    }
    const double h = std::fmin(dt, t_end - S.t);
    LH_CK(m, cudaMemcpyAsync(W.usave, u, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
    st = x_step(m, u, h, o, W, ready, &S);
    if (st == LH_OK) st = finite_or_restore(m, u, W.usave);
    if (st == LH_OK) st = x_force(m, o, W, u, &est, &S);   // estimate at the new state (F reused next step)
    if (st != LH_OK && st != LH_ENONFINITE) break;
    const double dt_new = o.cfl * est;
    if (st == LH_ENONFINITE || !(dt_new >= h)) {   // repeat the step with a smaller dt
      LH_CK(m, cudaMemcpyAsync(u, W.usave, sizeof(double) * m->n, cudaMemcpyDeviceToDevice, m->stream));
      ready = false;
      dt *= 0.85;
      ++S.rejected;
      st = LH_OK;
      if (S.rejected > 1000) {
        st = fail(m, LH_ENOCONV, "explicit advance: more than 1000 repeated steps");
        break;
      }
      continue;
    }
    ready = true;
    S.t += h;
    ++S.steps;
    if (dt_new > 1.25 * dt) dt *= 1.02;
  }
  LH_CK(m, cudaStreamSynchronize(m->stream));
  S.dt_last = dt;
  if (stats) *stats = S;
  return st;
}

}  // extern "C"

// ---- time loop with the Newton-count step control of Sec. 4 -----------------------------
namespace {

bool check_advance_opts(const lh_advance_opts& a, std::string* why) {
  if (a.scheme < 2 || a.scheme > 4) return *why = "scheme must be 2, 3 or 4", false;
  if (!(a.grow >= 1.0) || !(a.shrink > 0.0 && a.shrink < 1.0)) return *why = "need grow >= 1, 0 < shrink < 1", false;
  if (a.reject_its < 1 || a.grow_its >= a.reject_its) return *why = "need grow_its < reject_its, reject_its >= 1", false;
  if (!(a.dt0 >= 0.0) || !(a.fs_cfl > 0.0 || a.dt0 > 0.0)) return *why = "need fs_cfl > 0 or dt0 > 0", false;
  if (a.max_steps < 1) return *why = "max_steps must be >= 1", false;
  return true;
}

// The loop itself, shared by lh_advance and lh_advance_replay.  step(h, &its, &gmres)
// attempts a step of size h on trial storage and returns LH_OK (its = largest stage Newton
// count), a rejectable failure (LH_ENOCONV, LH_ETANGLED, LH_ENONFINITE) or a fatal status;
// commit() makes the trial state current.
template <class Step, class Commit>
lh_status advance_loop(double dt, double t_end, const lh_advance_opts& a, Step step, Commit commit,
                       lh_advance_stats* out, lh_advance_attempt* hist, int hist_cap, std::string* why) {
  lh_advance_stats S;
  std::memset(&S, 0, sizeof(S));
  lh_status ret = LH_OK;
  const double t_tol = 1e-14 * std::fmax(1.0, std::fabs(t_end));
  while (S.t < t_end - t_tol && S.steps < a.max_steps && (a.max_attempts <= 0 || S.attempts < a.max_attempts)) {
    if (!(dt >= a.dt_min) || !(dt > 0.0)) {
      *why = "time step control: dt fell below dt_min";
      ret = LH_ENOCONV;
      break;
    }
    const double h = std::fmin(dt, t_end - S.t);
    int its = -1, gm = 0;
    const lh_status st = step(h, &its, &gm);
    if (st != LH_OK && st != LH_ENOCONV && st != LH_ETANGLED && st != LH_ENONFINITE) {
      ret = st;
      break;
    }
    if (st != LH_OK) its = -1;
    const bool accepted = its >= 0 && its < a.reject_its;
    if (hist && S.attempts < hist_cap) hist[S.attempts] = lh_advance_attempt{dt, h, its, accepted ? 1 : 0};
    ++S.attempts;
    if (!accepted) {
      ++S.rejected;
      dt *= a.shrink;
      continue;
    }
    const lh_status cs = commit();
    if (cs != LH_OK) {
      ret = cs;
      break;
    }
    S.t += h;
    ++S.steps;
    S.newton_its += its;
    S.gmres_its += gm;
    if (its <= a.grow_its && a.enlarge) dt *= a.grow;
  }
  S.dt_next = dt;
  if (out) *out = S;
  return ret;
}

}  // namespace

extern "C" {

void lh_advance_opts_init(lh_advance_opts* a) {
  if (!a) return;
  std::memset(a, 0, sizeof(*a));
  a->scheme = 2;
  a->fs_cfl = 2.0;
  a->grow = 1.05;
  a->shrink = 0.85;
  a->grow_its = 1;
  a->reject_its = 4;
  a->enlarge = 1;
  a->max_steps = 1000000;
}

lh_status lh_advance(lh_mesh* m, double* u, double* k_prev, double t_end, const lh_newton_opts* nopts,
                     const lh_advance_opts* aopts, lh_advance_stats* stats, lh_advance_attempt* hist, int hist_cap) {
  if (!m || !u) return fail(m, LH_EINVAL, "NULL argument to lh_advance");
  if (!(t_end >= 0.0)) return fail(m, LH_EINVAL, "lh_advance: t_end must be >= 0");
  lh_advance_opts a;
  if (aopts) a = *aopts; else lh_advance_opts_init(&a);
  std::string why;
  if (!check_advance_opts(a, &why)) return fail(m, LH_EINVAL, "lh_advance: " + why);
  lh_newton_opts o;
  if (nopts) o = *nopts; else lh_newton_opts_init(&o);
  lh_status st = check_newton_opts(m, o);
  if (st != LH_OK) return st;
  const long long n = m->n;
  const size_t bytes = sizeof(double) * (size_t)n;
  if (!m->d_adv && cudaMalloc(&m->d_adv, 3 * bytes) != cudaSuccess)
    return fail(m, LH_ENOMEM, "cannot allocate the trial state of lh_advance");
  cudaStream_t s = m->stream;
  double* u_try = m->d_adv;
  double* k_try = m->d_adv + n;
  double* k_cur = k_prev ? k_prev : m->d_adv + 2 * n;
  if (!k_prev) LH_CK(m, cudaMemsetAsync(k_cur, 0, bytes, s));
  double dt = a.dt0;
  if (!(dt > 0.0)) {
    double est = 0.0;
    if ((st = lh_dt_estimate(m, u, &est)) != LH_OK) return st;
    dt = a.fs_cfl * est;
  }
  auto step = [&](double h, int* its, int* gm) -> lh_status {
    if (cudaMemcpyAsync(u_try, u, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(k_try, k_cur, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(m, LH_ECUDA, "lh_advance: trial copy failed");
    lh_step_stats S;
    std::memset(&S, 0, sizeof(S));
    const lh_status r = a.scheme == 2 ? lh_newton_step(m, u_try, k_try, h, &o, &S)
                                      : lh_sdirk_step(m, a.scheme, u_try, k_try, h, &o, &S);
    *its = S.newton_its_max;
    *gm = S.gmres_its_total;
    return r;
  };
  auto commit = [&]() -> lh_status {
    if (cudaMemcpyAsync(u, u_try, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(k_cur, k_try, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
      return fail(m, LH_ECUDA, "lh_advance: commit copy failed");
    return LH_OK;
  };
  st = advance_loop(dt, t_end, a, step, commit, stats, hist, hist_cap, &why);
  LH_CK(m, cudaStreamSynchronize(s));
  if (st == LH_ENOCONV && !why.empty()) return fail(m, st, "lh_advance: " + why);
  return st;
}

lh_status lh_advance_replay(const int* counts, int ncounts, double dt_est, double t_end,
                            const lh_advance_opts* aopts, lh_advance_stats* stats, lh_advance_attempt* hist,
                            int hist_cap) {
  if ((ncounts > 0 && !counts) || ncounts < 0 || !(dt_est > 0.0) || !(t_end >= 0.0))
    return set_global_error(LH_EINVAL, "lh_advance_replay: invalid argument");
  lh_advance_opts a;
  if (aopts) a = *aopts; else lh_advance_opts_init(&a);
  std::string why;
  if (!check_advance_opts(a, &why)) return set_global_error(LH_EINVAL, "lh_advance_replay: " + why);
  int next = 0;
  auto step = [&](double, int* its, int* gm) -> lh_status {
    const int c = next < ncounts ? counts[next] : 2;
    ++next;
    *gm = 0;
    if (c < 0) return LH_ENOCONV;
    *its = c;
    return LH_OK;
  };
  auto commit = []() -> lh_status { return LH_OK; };
  const double dt = a.dt0 > 0.0 ? a.dt0 : a.fs_cfl * dt_est;
  const lh_status st = advance_loop(dt, t_end, a, step, commit, stats, hist, hist_cap, &why);
  if (st != LH_OK) return set_global_error(st, "lh_advance_replay: " + why);
  return LH_OK;
}

lh_status lh_halo_len(const lh_mesh* m, int face, long long* len) {
  if (!m || !len) return set_global_error(LH_EINVAL, "NULL argument to lh_halo_len");
  if (face < 0 || face >= 2 * m->P.dim) return set_global_error(LH_EINVAL, "lh_halo_len: face out of range");
  *len = halo_len(m->P, face / 2);
  return LH_OK;
}

static lh_status halo_call(lh_mesh* m, int face, int mode, const void* src, void* dst, lh_prec prec) {
  if (!m || !src || !dst) return fail(m, LH_EINVAL, "NULL argument to lh_halo_pack/lh_halo_add");
  if (face < 0 || face >= 2 * m->P.dim) return fail(m, LH_EINVAL, "halo: face out of range");
  if ((m->P.bc >> face) & 1u) return fail(m, LH_EINVAL, "halo: the face is a wall of this mesh");
  if (prec == LH_FP64) {
    LH_CK(m, launch_halo<double>(m->P, m->stream, face, mode, static_cast<const double*>(src),
                                 static_cast<double*>(dst)));
  } else {
    LH_CK(m, launch_halo<float>(m->P, m->stream, face, mode, static_cast<const float*>(src),
                                static_cast<float*>(dst)));
  }
  return LH_OK;
}

lh_status lh_halo_pack(lh_mesh* m, int face, const void* r, void* buf, lh_prec prec) {
  return halo_call(m, face, 0, r, buf, prec);
}

lh_status lh_halo_add(lh_mesh* m, int face, const void* buf, void* r, lh_prec prec) {
  return halo_call(m, face, 1, buf, r, prec);
}

lh_status lh_tc_status(lh_mesh* m) {
  if (!m) return fail(nullptr, LH_EINVAL, "mesh is NULL");
  int flag = 0;
  LH_CK(m, cudaMemcpyAsync(&flag, tc_err(m), sizeof(int), cudaMemcpyDeviceToHost, m->stream));
  LH_CK(m, cudaStreamSynchronize(m->stream));
  if (flag) {
    LH_CK(m, cudaMemsetAsync(tc_err(m), 0, sizeof(int), m->stream));
    if (flag & kWaitErrPipe)
      return fail(m, LH_ECUDA, "record J.w: a bounded wait on the copy of an element's record timed out");
    return fail(m, LH_ECUDA, "tensor-core J.w: a bounded wait on the tensor cores timed out");
  }
  return LH_OK;
}

unsigned lh_tc_set_wait_polls(unsigned polls) { return set_tc_wait_polls(polls); }

const char* lh_last_error(const lh_mesh* m) { return m ? m->err.c_str() : g_err.c_str(); }

lh_status lh_profile_enable(lh_mesh* m, int enable) {
  if (!m) return fail(nullptr, LH_EINVAL, "mesh is NULL");
  Prof& p = m->prof;
  if (enable && !p.ev[0]) {
    for (int i = 0; i < 2 * Prof::kMax; ++i) LH_CK(m, cudaEventCreate(&p.ev[i]));
  }
  if (!enable) LH_CK(m, prof_flush(m));
  p.n = 0;
  for (int i = 0; i < 8; ++i) {
    p.ms[i] = 0.0;
    p.cnt[i] = 0;
  }
  p.on = enable != 0;
  return LH_OK;
}

lh_status lh_profile_read(lh_mesh* m, double* ms, long long* count) {
  if (!m || !ms || !count) return fail(m, LH_EINVAL, "NULL argument to lh_profile_read");
  LH_CK(m, prof_flush(m));
  for (int i = 0; i < LH_PROF_KINDS; ++i) {
    ms[i] = m->prof.ms[i];
    count[i] = m->prof.cnt[i];
  }
  return LH_OK;
}

long long lh_launch_count(void) { return launches(); }

lh_status lh_probe_fma(int prec, double* tflops) {
  if (!tflops) return fail(nullptr, LH_EINVAL, "tflops is NULL");
  if (prec != LH_FP64 && prec != LH_FP32) return fail(nullptr, LH_EINVAL, "prec must be LH_FP64 or LH_FP32");
  cudaError_t e = launch_probe_fma(prec, tflops);
  if (e != cudaSuccess) return fail(nullptr, LH_ECUDA, std::string("lh_probe_fma: ") + cudaGetErrorString(e));
  return LH_OK;
}

}  // extern "C"
