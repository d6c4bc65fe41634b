// Nonlinear problems U' + K U + phi(U) = f on a theta-method plan by the
// simplified Newton iteration of eq. 1.5 (Section 1, eq. 1.4).
//
// phi(u) = a1 u + a2 u^2 + a3 u^3 acts pointwise.  The all-at-once system is
// (B1 (x) I) u + (B2 (x) I) F(u) = b with F(u)_n = K U_n + phi(U_n); its
// Jacobian B1 (x) I + (B2 (x) I) blkdiag(K + diag phi'(U_n)) is replaced by the
// alpha-circulant P_alpha(u) = C1 (x) I + C2 (x) (K + sigma I), sigma the mean
// of phi'(U) over all time levels and grid points.  K + sigma I keeps the
// spatial eigenvectors of K, so P_alpha(u)^{-1} is the plan's preconditioner
// with every shifted system lambda_1k + lambda_2k (K + sigma) = (lambda_1k +
// sigma lambda_2k) + lambda_2k K: only the plan's table of lambda_1k changes.
//
// One Newton step: r = b - (B1 (x) I) u - (B2 (x) I) F(u) with ||r||^2 and the
// sum of phi'(U) (one FP64 kernel), the shifted table, z = P_alpha^{-1} r (the
// plan's three steps of eq. 1.3), u += z.
#include <cmath>
#include <complex>
#include <vector>

#include "pd_plan.h"

namespace {

constexpr int NB = 256;       // threads per block
constexpr int NL_ROWS = 16;   // time levels per thread in the residual

struct Reaction {
  double a1, a2, a3;
};

__device__ __forceinline__ double phi_of(const Reaction& c, double u) {
  return u * fma(u, fma(u, c.a3, c.a2), c.a1);
}
// phi'(u) in FP32 (it only enters the mean sigma)
__device__ __forceinline__ float dphi_of(const Reaction& c, float u) {
  return fmaf(u, fmaf(3.f * (float)c.a3, u, 2.f * (float)c.a2), (float)c.a1);
}

// (K U)(s) for one time level U: 3- or 5-point centred stencil
__device__ __forceinline__ double k_apply(const Stencil& st, const double* __restrict__ U, int s) {
  const int xg = s % st.nx, y = s / st.nx;
  double v = st.kc * U[s];
  if (xg > 0) v = fma(st.kxl, U[s - 1], v);
  else if (st.bcx == PD_PERIODIC && st.nx > 1) v = fma(st.kxl, U[s + st.nx - 1], v);
  if (xg < st.nx - 1) v = fma(st.kxu, U[s + 1], v);
  else if (st.bcx == PD_PERIODIC && st.nx > 1) v = fma(st.kxu, U[s - st.nx + 1], v);
  if (st.dim == 2) {
    if (y > 0) v = fma(st.kyl, U[s - st.nx], v);
    if (y < st.ny - 1) v = fma(st.kyu, U[s + st.nx], v);
  }
  return v;
}

template <typename T>
__device__ __forceinline__ void block_add(T v, T* red, T* out) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    T t = 0;
    for (int w = 0; w < NB / 32; ++w) t += red[w];
    atomicAdd(out, t);
  }
  __syncthreads();
}

// r = b - sum_m c1[m] U_{n-m} - c2[m] F_{n-m} (m = 0, 1; U_{-1} terms are in
// b); acc[0] += ||r||^2, acc[1] += sum phi'(U).  Thread: one grid point and
// NL_ROWS consecutive time levels, carrying U_{n-1} and F_{n-1}.  r and F are
// FP64; the two sums, which need a few digits only, are FP32 on the FP32
// parts of U and r (split with integer operations, off the FP64 pipe).
__global__ void __launch_bounds__(NB) k_nl_resid(Stencil st, TimeBand tb, int N, Reaction c,
                                                 const double* __restrict__ u,
                                                 const double* __restrict__ b,
                                                 double* __restrict__ r, double* acc) {
  __shared__ double red[NB / 32];
  const int s = blockIdx.x * NB + threadIdx.x;
  const int n0 = blockIdx.y * NL_ROWS;
  const size_t S = (size_t)st.S;
  float pr = 0.f, pd = 0.f;
  if (s < st.S) {
    double Up = 0.0, Fp = 0.0;
    if (n0 > 0) {
      const double* U = u + (size_t)(n0 - 1) * S;
      Up = U[s];
      Fp = k_apply(st, U, s) + phi_of(c, Up);
    }
    const int n1 = min(N, n0 + NL_ROWS);
    for (int n = n0; n < n1; ++n) {
      const double* U = u + (size_t)n * S;
      const double Un = U[s];
      const double Fn = k_apply(st, U, s) + phi_of(c, Un);
      double v = b[(size_t)n * S + s];
      v = fma(-tb.c1[0], Un, v);
      v = fma(-tb.c2[0], Fn, v);
      if (n > 0) {
        v = fma(-tb.c1[1], Up, v);
        v = fma(-tb.c2[1], Fp, v);
      }
      r[(size_t)n * S + s] = v;
      const float vf = df_from_double(v).hi;
      pr = fmaf(vf, vf, pr);
      pd += dphi_of(c, df_from_double(Un).hi);
      Up = Un;
      Fp = Fn;
    }
  }
  block_add((double)pr, red, acc);
  block_add((double)pd, red, acc + 1);
}

// first row of the right-hand side: b_0 -= c2[1] phi(U_0)
__global__ void k_nl_rhs(int S, double w, Reaction c, const double* __restrict__ u0,
                         double* __restrict__ b) {
  const int s = blockIdx.x * NB + threadIdx.x;
  if (s < S) b[s] = fma(-w, phi_of(c, u0[s]), b[s]);
}

__global__ void k_nl_update(double* __restrict__ u, const double* __restrict__ z, size_t n) {
  for (size_t i = blockIdx.x * (size_t)NB + threadIdx.x; i < n; i += (size_t)gridDim.x * NB)
    u[i] += z[i];
}

pd_status nl_err(pd_plan* p, pd_status s, const char* what) {
  snprintf(p->msg, sizeof(p->msg), "%s", what);
  return s;
}

pd_status nl_cuda(pd_plan* p, cudaError_t e, const char* what) {
  snprintf(p->msg, sizeof(p->msg), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
}

#define NLCU(call)                                       \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return nl_cuda(p, e_, #call); \
  } while (0)

#define NLLK(...)                                                  \
  do {                                                             \
    __VA_ARGS__;                                                   \
    ++p->launches;                                                 \
    cudaError_t e_ = cudaGetLastError();                           \
    if (e_ != cudaSuccess) return nl_cuda(p, e_, "kernel launch"); \
  } while (0)

pd_status nl_args(pd_plan* p, const double* a, Reaction* c) {
  if (p->scheme == PD_LEAPFROG)
    return nl_err(p, PD_ERR_UNSUPPORTED, "the nonlinear form needs a theta-method plan");
  if (!a) return nl_err(p, PD_ERR_ARG, "null reaction coefficients");
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(a[i])) return nl_err(p, PD_ERR_ARG, "non-finite reaction coefficient");
  c->a1 = a[0];
  c->a2 = a[1];
  c->a3 = a[2];
  return PD_OK;
}

// residual into r with acc[0..1] (device) accumulated; no synchronisation
pd_status nl_resid_launch(pd_plan* p, const Reaction& c, const double* b, const double* u,
                          double* r, double* acc) {
  NLCU(cudaMemsetAsync(acc, 0, 2 * sizeof(double), p->stream));
  const dim3 grid((unsigned)ceil_div(p->S, NB), (unsigned)ceil_div(p->nt, NL_ROWS));
  NLLK(k_nl_resid<<<grid, NB, 0, p->stream>>>(p->st, p->tb, p->nt, c, u, b, r, acc));
  return PD_OK;
}

// the plan's (lambda_1k, lambda_2k) in FP64, as the plan computed them:
// lambda_jk = sum_m c_j[m] w_k^m, w_k = alpha^{1/Nt} exp(-2 pi i k / Nt) (Lemma 1)
std::vector<std::complex<double>> plan_lambdas(const pd_plan* p) {
  using cd = std::complex<double>;
  const double PI = 3.14159265358979323846;
  const double ar = std::pow(p->alpha, 1.0 / p->nt);
  std::vector<cd> lam((size_t)2 * p->nh);
  for (int k = 0; k < p->nh; ++k) {
    const double th = -2.0 * PI * k / p->nt;
    const cd w = ar * cd(std::cos(th), std::sin(th));
    cd l1 = 0, l2 = 0, wm = 1;
    for (int m = 0; m <= p->tb.band && m < p->nt; ++m) {
      l1 += p->tb.c1[m] * wm;
      l2 += p->tb.c2[m] * wm;
      wm *= w;
    }
    lam[2 * k] = l1;
    lam[2 * k + 1] = l2;
  }
  return lam;
}

// device table <- (lambda_1k + sigma lambda_2k, lambda_2k), in the plan's precision
pd_status upload_shifted(pd_plan* p, const std::vector<std::complex<double>>& lam, double sigma) {
  const size_t m = lam.size();
  if (p->fp64) {
    std::vector<double2> h(m);
    for (size_t i = 0; i < m; i += 2) {
      const std::complex<double> l1 = lam[i] + sigma * lam[i + 1];
      h[i] = make_double2(l1.real(), l1.imag());
      h[i + 1] = make_double2(lam[i + 1].real(), lam[i + 1].imag());
    }
    NLCU(cudaMemcpyAsync(p->lam, h.data(), m * sizeof(double2), cudaMemcpyHostToDevice, p->stream));
    NLCU(cudaStreamSynchronize(p->stream));
  } else {
    std::vector<float2> h(m);
    for (size_t i = 0; i < m; i += 2) {
      const std::complex<double> l1 = lam[i] + sigma * lam[i + 1];
      h[i] = make_float2((float)l1.real(), (float)l1.imag());
      h[i + 1] = make_float2((float)lam[i + 1].real(), (float)lam[i + 1].imag());
    }
    NLCU(cudaMemcpyAsync(p->lam, h.data(), m * sizeof(float2), cudaMemcpyHostToDevice, p->stream));
    NLCU(cudaStreamSynchronize(p->stream));
  }
  return PD_OK;
}

pd_status ensure_nl_buffers(pd_plan* p) {
  const size_t bytes = (size_t)p->nt * p->S * sizeof(double);
  if (!p->nl_r) {
    NLCU(cudaMalloc((void**)&p->nl_r, bytes));
    p->bytes += bytes;
  }
  if (!p->nl_z) {
    NLCU(cudaMalloc((void**)&p->nl_z, bytes));
    p->bytes += bytes;
  }
  return PD_OK;
}

}  // namespace

extern "C" pd_status pd_nl_build_rhs(pd_plan* p, const double* a, const double* u0,
                                     const double* f, double* b) {
  if (!p) return PD_ERR_ARG;
  if (!u0 || !b) return nl_err(p, PD_ERR_ARG, "null argument");
  Reaction c;
  pd_status s = nl_args(p, a, &c);
  if (s != PD_OK) return s;
  s = pd_build_rhs(p, u0, nullptr, f, b);
  if (s != PD_OK) return s;
  // the U_0 level of the first row: -(1 - theta) phi(U_0)
  if (p->tb.c2[1] != 0.0)
    NLLK(k_nl_rhs<<<ceil_div(p->S, NB), NB, 0, p->stream>>>(p->S, p->tb.c2[1], c, u0, b));
  return PD_OK;
}

extern "C" pd_status pd_nl_residual(pd_plan* p, const double* a, const double* b, const double* u,
                                    double* r, double* sigma, double* rnorm2) {
  if (!p) return PD_ERR_ARG;
  if (!b || !u || !r) return nl_err(p, PD_ERR_ARG, "null argument");
  Reaction c;
  pd_status s = nl_args(p, a, &c);
  if (s != PD_OK) return s;
  s = nl_resid_launch(p, c, b, u, r, p->dsc);
  if (s != PD_OK) return s;
  if (sigma || rnorm2) {
    double h[2];
    NLCU(cudaMemcpyAsync(h, p->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    NLCU(cudaStreamSynchronize(p->stream));
    if (rnorm2) *rnorm2 = h[0];
    if (sigma) *sigma = h[1] / ((double)p->nt * p->S);
  }
  return PD_OK;
}

extern "C" pd_status pd_nl_solve(pd_plan* p, const double* a, const double* b, double* u,
                                 double tol, int maxit, int* iters, double* relres) {
  if (!p) return PD_ERR_ARG;
  if (!b || !u) return nl_err(p, PD_ERR_ARG, "null argument");
  if (!(tol >= 0.0) || maxit < 0) return nl_err(p, PD_ERR_ARG, "bad tolerance or iteration cap");
  Reaction c;
  pd_status s = nl_args(p, a, &c);
  if (s != PD_OK) return s;
  s = ensure_nl_buffers(p);
  if (s != PD_OK) return s;
  const size_t ns = (size_t)p->nt * p->S;
  // ||b||^2
  NLCU(cudaMemsetAsync(p->dsc + 2, 0, sizeof(double), p->stream));
  ++p->launches;
  NLCU(launch_norm2(b, ns, p->dsc + 2, p->stream));
  double nb2 = 0.0;
  NLCU(cudaMemcpyAsync(&nb2, p->dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  NLCU(cudaStreamSynchronize(p->stream));
  const double nb = std::sqrt(nb2);
  const std::vector<std::complex<double>> lam = plan_lambdas(p);
  int it = 0;
  double rel = 0.0;
  pd_status out = PD_OK;
  for (;;) {
    s = nl_resid_launch(p, c, b, u, p->nl_r, p->dsc);
    if (s != PD_OK) { out = s; break; }
    double h[2];
    NLCU(cudaMemcpyAsync(h, p->dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
    NLCU(cudaStreamSynchronize(p->stream));
    rel = nb > 0.0 ? std::sqrt(h[0]) / nb : std::sqrt(h[0]);
    if (!std::isfinite(rel) || !std::isfinite(h[1])) {
      out = nl_err(p, PD_ERR_NONFINITE, "non-finite value in the simplified Newton iteration");
      break;
    }
    if (rel <= tol) break;
    if (it >= maxit) {
      out = nl_err(p, PD_ERR_NOT_CONVERGED, "simplified Newton did not reach the tolerance");
      break;
    }
    const double sigma = h[1] / (double)ns;
    s = upload_shifted(p, lam, sigma);
    if (s != PD_OK) { out = s; break; }
    s = plan_precond(p, p->nl_r, p->nl_z);
    if (s != PD_OK) { out = s; break; }
    NLLK(k_nl_update<<<2 * 152, NB, 0, p->stream>>>(u, p->nl_z, ns));
    ++it;
  }
  // the plan's own table back (its linear solves use it)
  const pd_status s2 = upload_shifted(p, lam, 0.0);
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return out != PD_OK ? out : s2;
}
