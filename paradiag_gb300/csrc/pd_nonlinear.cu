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
// sum of phi'(U) (one kernel: FP64 on FP64 plans, double-float on mixed ones),
// the shifted table (a small kernel reading the sum on the device), z =
// P_alpha^{-1} r (the plan's three steps of eq. 1.3), u += z.
#include <algorithm>
#include <cmath>
#include <cstdio>

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

// ---- double-float residual (mixed plans): the same r on the FP32 pipes ----

// coefficients of the double-float residual (host-rounded double-float pairs)
struct NlDf {
  df kc, kxl, kxu, kyl, kyu;  // stencil
  df c10, c11, c20, c21;      // time weights c1[0], c1[1], c2[0], c2[1]
  df a1, a2, a3;              // reaction
};

__device__ __forceinline__ df ld_df(const double* __restrict__ x, size_t i) {
  return df_from_double(x[i]);
}
__device__ __forceinline__ df ld_df(const float2* __restrict__ x, size_t i) {
  const float2 v = __ldg(&x[i]);
  return df_make(v.x, v.y);
}

// compensated sum (value = s + e): every term enters with one two-sum of its
// high part; low parts and rounding errors gather in e
struct NlAcc {
  float s, e;
};
__device__ __forceinline__ void nl_add(NlAcc& A, float h, float l) {
  const float t = __fadd_rn(A.s, h);
  const float bb = __fsub_rn(t, A.s);
  const float err = __fadd_rn(__fsub_rn(A.s, __fsub_rn(t, bb)), __fsub_rn(h, bb));
  A.s = t;
  A.e = __fadd_rn(A.e, __fadd_rn(err, l));
}
// A += k u: the product of the high parts exactly (FMA), the cross terms into e
__device__ __forceinline__ void nl_add_prod(NlAcc& A, df k, df u) {
  const float p = __fmul_rn(k.hi, u.hi);
  float pe = __fmaf_rn(k.hi, u.hi, -p);
  pe = __fmaf_rn(k.hi, u.lo, pe);
  pe = __fmaf_rn(k.lo, u.hi, pe);
  nl_add(A, p, pe);
}
__device__ __forceinline__ df nl_val(const NlAcc& A) { return fast_two_sum(A.s, A.e); }

// The stencil neighbours of point s (offsets from s; 0: no neighbour), fixed
// for every time row of a thread
struct NlNbh {
  int l, r, d, u;
};
__device__ __forceinline__ NlNbh nl_nbh(const Stencil& st, int s) {
  const int xg = s % st.nx, y = s / st.nx;
  NlNbh g;
  g.l = xg > 0 ? -1 : (st.bcx == PD_PERIODIC && st.nx > 1 ? st.nx - 1 : 0);
  g.r = xg < st.nx - 1 ? 1 : (st.bcx == PD_PERIODIC && st.nx > 1 ? -(st.nx - 1) : 0);
  g.d = (st.dim == 2 && y > 0) ? -st.nx : 0;
  g.u = (st.dim == 2 && y < st.ny - 1) ? st.nx : 0;
  return g;
}

// F(U)(s) = (K U)(s) + phi(U(s)) as one compensated sum of eight terms
template <typename T>
__device__ __forceinline__ df f_of_df(const NlDf& c, const T* __restrict__ U, int s,
                                      const NlNbh& g, df uc) {
  NlAcc A = {0.f, 0.f};
  nl_add_prod(A, c.kc, uc);
  if (g.l) nl_add_prod(A, c.kxl, ld_df(U, s + g.l));
  if (g.r) nl_add_prod(A, c.kxu, ld_df(U, s + g.r));
  if (g.d) nl_add_prod(A, c.kyl, ld_df(U, s + g.d));
  if (g.u) nl_add_prod(A, c.kyu, ld_df(U, s + g.u));
  // phi(u) = a1 u + a2 u^2 + a3 u^3
  const df u2 = df_mul(uc, uc);
  const df u3 = df_mul(u2, uc);
  nl_add_prod(A, c.a1, uc);
  nl_add_prod(A, c.a2, u2);
  nl_add_prod(A, c.a3, u3);
  return nl_val(A);
}

// k_nl_resid with double-float inputs and compensated sums (unit roundoff
// about 2^-48 against the largest term): the FP64 inputs are split with
// integer operations and r is written as hi + lo (one FP64 addition)
// T = double: FP64 inputs, split on load; T = float2: double-float inputs
template <typename T>
__global__ void __launch_bounds__(NB) k_nl_resid_df(Stencil st, NlDf c, Reaction cr, int N,
                                                    const T* __restrict__ u,
                                                    const T* __restrict__ b,
                                                    double* __restrict__ r, double* acc) {
  __shared__ double red[NB / 32];
  const int s = blockIdx.x * NB + threadIdx.x;
  const int n0 = blockIdx.y * NL_ROWS;
  const size_t S = (size_t)st.S;
  // the time weights negated once: v = b - c1[0] U_n - c2[0] F_n - c1[1] U_{n-1} - c2[1] F_{n-1}
  const df m10 = df_neg(c.c10), m20 = df_neg(c.c20), m11 = df_neg(c.c11), m21 = df_neg(c.c21);
  float pr = 0.f, pd = 0.f;
  if (s < st.S) {
    const NlNbh g = nl_nbh(st, s);
    df Up = df_make(0.f, 0.f), Fp = Up;
    if (n0 > 0) {
      const T* U = u + (size_t)(n0 - 1) * S;
      Up = ld_df(U, s);
      Fp = f_of_df(c, U, s, g, Up);
    }
    const int n1 = min(N, n0 + NL_ROWS);
    for (int n = n0; n < n1; ++n) {
      const T* U = u + (size_t)n * S;
      const df Un = ld_df(U, s);
      const df Fn = f_of_df(c, U, s, g, Un);
      const df bn = ld_df(b, (size_t)n * S + s);
      NlAcc V = {bn.hi, bn.lo};
      nl_add_prod(V, m10, Un);
      nl_add_prod(V, m20, Fn);
      if (n > 0) {
        nl_add_prod(V, m11, Up);
        nl_add_prod(V, m21, Fp);
      }
      const df v = nl_val(V);
      r[(size_t)n * S + s] = double_from_float(v.hi) + double_from_float(v.lo);
      pr = fmaf(v.hi, v.hi, pr);
      pd += dphi_of(cr, Un.hi);
      Up = Un;
      Fp = Fn;
    }
  }
  block_add((double)pr, red, acc);
  block_add((double)pd, red, acc + 1);
}

df df_host(double v) {
  const dfc c = dfc_from(v);
  df d;
  d.hi = c.hi;
  d.lo = c.lo;
  return d;
}

// first row of the right-hand side: b_0 -= c2[1] phi(U_0)
__global__ void k_nl_rhs(int S, double w, Reaction c, const double* __restrict__ u0,
                         double* __restrict__ b) {
  const int s = blockIdx.x * NB + threadIdx.x;
  if (s < S) b[s] = fma(-w, phi_of(c, u0[s]), b[s]);
}

// u += z; with udf, also the double-float copy of the new u
__global__ void k_nl_update(double* __restrict__ u, const double* __restrict__ z,
                            float2* __restrict__ udf, size_t n) {
  for (size_t i = blockIdx.x * (size_t)NB + threadIdx.x; i < n; i += (size_t)gridDim.x * NB) {
    const double v = u[i] + z[i];
    u[i] = v;
    if (udf != nullptr) {
      const df d = df_from_double(v);
      udf[i] = make_float2(d.hi, d.lo);
    }
  }
}

// lam[2k] = lam0[2k] + sigma lam0[2k+1], lam[2k+1] = lam0[2k+1] with sigma =
// acc[1] / ns read from device memory (left there by the residual kernel)
template <typename C>
__global__ void k_nl_shift(C* __restrict__ lam, const C* __restrict__ lam0,
                           const double* __restrict__ acc, double ns, int nh) {
  const double sigma = acc[1] / ns;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < nh; k += gridDim.x * blockDim.x) {
    const C l1 = lam0[2 * k], l2 = lam0[2 * k + 1];
    C o;
    o.x = l1.x + (decltype(o.x))sigma * l2.x;
    o.y = l1.y + (decltype(o.y))sigma * l2.y;
    lam[2 * k] = o;
    lam[2 * k + 1] = l2;
  }
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

// residual into r with acc[0..1] (device) accumulated; no synchronisation.
// Mixed plans with double-float copies (udf, bdf) of u and b read those.
pd_status nl_resid_launch(pd_plan* p, const Reaction& c, const double* b, const double* u,
                          double* r, double* acc, const float2* udf = nullptr,
                          const float2* bdf = nullptr) {
  NLCU(cudaMemsetAsync(acc, 0, 2 * sizeof(double), p->stream));
  const dim3 grid((unsigned)ceil_div(p->S, NB), (unsigned)ceil_div(p->nt, NL_ROWS));
  if (p->fp64) {
    NLLK(k_nl_resid<<<grid, NB, 0, p->stream>>>(p->st, p->tb, p->nt, c, u, b, r, acc));
  } else {
    // mixed plans: the same residual in double-float on the FP32 pipes
    NlDf d;
    d.kc = df_host(p->st.kc); d.kxl = df_host(p->st.kxl); d.kxu = df_host(p->st.kxu);
    d.kyl = df_host(p->st.kyl); d.kyu = df_host(p->st.kyu);
    d.c10 = df_host(p->tb.c1[0]); d.c11 = df_host(p->tb.c1[1]);
    d.c20 = df_host(p->tb.c2[0]); d.c21 = df_host(p->tb.c2[1]);
    d.a1 = df_host(c.a1); d.a2 = df_host(c.a2); d.a3 = df_host(c.a3);
    if (udf != nullptr && bdf != nullptr)
      NLLK(k_nl_resid_df<float2><<<grid, NB, 0, p->stream>>>(p->st, d, c, p->nt, udf, bdf, r, acc));
    else
      NLLK(k_nl_resid_df<double><<<grid, NB, 0, p->stream>>>(p->st, d, c, p->nt, u, b, r, acc));
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
  if (!p->nl_lam0) {
    // the plan's own eigenvalue table (unshifted: every solve restores it)
    const size_t lb = (size_t)2 * p->nh * (p->fp64 ? sizeof(double2) : sizeof(float2));
    NLCU(cudaMalloc(&p->nl_lam0, lb));
    p->bytes += lb;
    NLCU(cudaMemcpyAsync(p->nl_lam0, p->lam, lb, cudaMemcpyDeviceToDevice, p->stream));
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
  // mixed plans: u and b split into double-float once (the plan's solver
  // state); the update keeps the copy of u current
  float2* udf = (!p->fp64 && p->Udf && p->Bdf) ? p->Udf : nullptr;
  if (udf) {
    NLCU(cudaMemsetAsync(p->dsc + 4, 0, sizeof(double), p->stream));
    ++p->launches;
    NLCU(launch_entry_df(u, b, 1.0, p->Udf, p->Bdf, ns, p->dsc + 4, p->stream));
  }
  int it = 0;
  double rel = 0.0;
  pd_status out = PD_OK;
  for (;;) {
    s = nl_resid_launch(p, c, b, u, p->nl_r, p->dsc, udf, udf ? p->Bdf : nullptr);
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
    // the shifted table on the device, from the residual kernel's sum
    if (p->fp64)
      NLLK(k_nl_shift<<<ceil_div(p->nh, NB), NB, 0, p->stream>>>(
          static_cast<double2*>(p->lam), static_cast<const double2*>(p->nl_lam0), p->dsc,
          (double)ns, p->nh));
    else
      NLLK(k_nl_shift<<<ceil_div(p->nh, NB), NB, 0, p->stream>>>(
          static_cast<float2*>(p->lam), static_cast<const float2*>(p->nl_lam0), p->dsc,
          (double)ns, p->nh));
    s = plan_precond(p, p->nl_r, p->nl_z);
    if (s != PD_OK) { out = s; break; }
    NLLK(k_nl_update<<<2 * 152, NB, 0, p->stream>>>(u, p->nl_z, udf, ns));
    ++it;
  }
  // the plan's own table back (its linear solves use it)
  pd_status s2 = PD_OK;
  {
    const size_t lb = (size_t)2 * p->nh * (p->fp64 ? sizeof(double2) : sizeof(float2));
    const cudaError_t e = cudaMemcpyAsync(p->lam, p->nl_lam0, lb, cudaMemcpyDeviceToDevice,
                                          p->stream);
    if (e != cudaSuccess) s2 = nl_cuda(p, e, "restoring the eigenvalue table");
  }
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return out != PD_OK ? out : s2;
}

extern "C" pd_status pd_nl_solve_windows(pd_plan* p, const double* a, const double* u0,
                                         const double* f, int nwin, double* u, double tol,
                                         int maxit, int* iters_total, double* relres_max) {
  if (!p) return PD_ERR_ARG;
  if (!u0 || !u || nwin < 1) return nl_err(p, PD_ERR_ARG, "bad argument");
  Reaction c;
  pd_status s = nl_args(p, a, &c);
  if (s != PD_OK) return s;
  const size_t ns = (size_t)p->nt * p->S;
  const size_t S = (size_t)p->S;
  if (!p->nl_b) {
    NLCU(cudaMalloc((void**)&p->nl_b, ns * sizeof(double)));
    p->bytes += ns * sizeof(double);
  }
  int total = 0;
  double worst = 0.0;
  for (int w = 0; w < nwin; ++w) {
    double* uw = u + (size_t)w * ns;
    const double* start = w == 0 ? u0 : uw - S;  // last time level of the previous window
    const double* fw = f ? f + (size_t)w * p->nt * S : nullptr;
    s = pd_nl_build_rhs(p, a, start, fw, p->nl_b);
    if (s == PD_OK) {
      NLCU(cudaMemsetAsync(uw, 0, ns * sizeof(double), p->stream));
      int it = 0;
      double rel = 0.0;
      s = pd_nl_solve(p, a, p->nl_b, uw, tol, maxit, &it, &rel);
      total += it;
      worst = std::max(worst, rel);
    }
    if (s != PD_OK) break;
  }
  if (iters_total) *iters_total = total;
  if (relres_max) *relres_max = worst;
  return s;
}

