// ParaDiag-II for the optimal control of the wave equation (Section 4): the
// saddle-point all-at-once system of the implicit leap-frog scheme, solved
// by flexible GMRES with the gamma-balanced block circulant preconditioner.
//
// The system is scaled by dt^2 as in the section.  With
//   T1 = lower Toeplitz (1, -2, 1), T2 = lower Toeplitz (1, 0, 1) dt^2/2,
//   Ih = diag(1/2, 1, ..., 1), Ic = diag(1, ..., 1, 1/2), beta = dt^2/sqrt(gamma),
// the balanced system (unknowns (gamma^{1/2} u, p)) is
//   A = [[T1, -beta Ih], [beta Ic, T1^T]] (x) I + blockdiag(T2, T2^T) (x) K
// and the preconditioner replaces T1, T2 by their Strang circulants C1, C2 and
// Ih, Ic by I.  P = P~ (blockdiag(C2, C2^T) (x) I) (eq. 4.3), and P~ is block
// diagonal in the Fourier basis (Theorem 4): with d1, d2 the circulant
// eigenvalues (transform X_k = sum_n x_n exp(-2 pi i n k / Nt)), frequency k
// carries the 2 x 2 block [[lam, -beta/conj(d2)], [beta/d2, lam]] + I (x) K,
// lam = d1/d2 real, eigenvalues sigma_+- = lam +- i beta/|d2| and eigenvectors
// Q = [[1, 1], [-i phibar, i phibar]], phibar = conj(d2)/|d2| (Q/sqrt 2 is
// unitary: Cond_2(V) = 1).  So z = P^{-1} r is
//   R = FFT_t(r1), FFT_t(r2)                                  (K1, two launches)
//   (z+, z-) = Q^{-1} (R1, R2) = ((R1 + i phi R2)/2, (R1 - i phi R2)/2)
//   (sigma_+- I + K) y_+- = z_+-                              (step (b), 2 Nh rows)
//   (Z1, Z2) = (Q (y+, y-)) / (d2, conj d2)
//   z = IFFT_t(Z1), IFFT_t(Z2)                                (K3, two launches).
// Real data: only the half spectrum k = 0..Nt/2 is formed (the outputs are
// real, so their spectra are Hermitian).  Nt divisible by 4 makes C2 singular
// (d2 = 0 at k = Nt/4) and is rejected.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pd_plan.h"

using cdc = std::complex<double>;

namespace {

constexpr int CT_TB = 256;

struct MixArgs {
  int nh, specS;
  const void* tab;      // per k: phi = d2/|d2|, 1/d2 (complex, float or double)
  void* A;              // spectrum of field 1 [nh][specS]
  void* B;              // spectrum of field 2
  void* Z;              // step (b) rows [2 nh][specS]
  unsigned* amax;       // mixed + tensor-core x-transform: max |Z| into *amax
  unsigned* amax_reset;
};

template <typename R>
__global__ void __launch_bounds__(CT_TB) k_ctl_mix_in(const MixArgs a) {
  using C = cplx_t<R>;
  const size_t i = (size_t)blockIdx.x * CT_TB + threadIdx.x;
  const size_t total = (size_t)a.nh * a.specS;
  float amx = 0.f;
  if (i < total) {
    const int k = (int)(i / a.specS);
    const C* tab = reinterpret_cast<const C*>(a.tab);
    const C phi = tab[2 * k];
    const C r1 = reinterpret_cast<const C*>(a.A)[i];
    const C r2 = reinterpret_cast<const C*>(a.B)[i];
    const C ipr = cmul_pi(cmul(phi, r2));             // i phi R2
    const C zp = cscale(cadd(r1, ipr), (R)0.5);
    const C zm = cscale(csub(r1, ipr), (R)0.5);
    C* Z = reinterpret_cast<C*>(a.Z);
    Z[i] = zp;
    Z[i + total] = zm;
    amx = fmaxf(fmaxf(fabsf((float)zp.x), fabsf((float)zp.y)),
                fmaxf(fabsf((float)zm.x), fabsf((float)zm.y)));
  }
  if (a.amax != nullptr) {
    for (int o = 16; o > 0; o >>= 1) amx = fmaxf(amx, __shfl_xor_sync(0xffffffffu, amx, o));
    if ((threadIdx.x & 31) == 0) atomicMax(a.amax, __float_as_uint(amx));
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.amax_reset) *a.amax_reset = 0u;
  }
}

template <typename R>
__global__ void __launch_bounds__(CT_TB) k_ctl_mix_out(const MixArgs a) {
  using C = cplx_t<R>;
  const size_t i = (size_t)blockIdx.x * CT_TB + threadIdx.x;
  const size_t total = (size_t)a.nh * a.specS;
  if (i >= total) return;
  const int k = (int)(i / a.specS);
  const C* tab = reinterpret_cast<const C*>(a.tab);
  const C phi = tab[2 * k], id2 = tab[2 * k + 1];
  const C* Z = reinterpret_cast<const C*>(a.Z);
  const C yp = Z[i], ym = Z[i + total];
  // Y1 = (y+ + y-) / d2;  Y2 = i phibar (y- - y+) / conj(d2)
  const C y1 = cmul(cadd(yp, ym), id2);
  const C t = cmul_pi(cmul(cconj(phi), csub(ym, yp)));
  const C y2 = cmul(t, cconj(id2));
  reinterpret_cast<C*>(a.A)[i] = y1;
  reinterpret_cast<C*>(a.B)[i] = y2;
}

// y = A x for the balanced saddle-point system (FP64); x, y = [2][Nt][S]
struct CtlApply {
  int N, S;
  Stencil st;
  double beta, c2;     // beta = dt^2/sqrt(gamma); c2 = dt^2/2 (T2 weights)
  const double* x;
  double* y;
  const double* b;     // if set: y = b - A x and ||y||^2 into *norm2
  double* norm2;
};

PD_D double ku_at(const Stencil& st, const double* U, int s) {
  const int x = s % st.nx, yy = s / st.nx;
  double k = st.kc * U[s];
  if (x > 0) k = fma(st.kxl, U[s - 1], k);
  else if (st.bcx == PD_PERIODIC) k = fma(st.kxl, U[s + st.nx - 1], k);
  if (x < st.nx - 1) k = fma(st.kxu, U[s + 1], k);
  else if (st.bcx == PD_PERIODIC) k = fma(st.kxu, U[s - (st.nx - 1)], k);
  if (st.dim == 2) {
    if (yy > 0) k = fma(st.kyl, U[s - st.nx], k);
    if (yy < st.ny - 1) k = fma(st.kyu, U[s + st.nx], k);
  }
  return k;
}

__global__ void __launch_bounds__(CT_TB) k_ctl_apply(const CtlApply a) {
  const int s = blockIdx.x * CT_TB + threadIdx.x;
  const int N = a.N, S = a.S;
  const size_t NS = (size_t)N * S;
  double nrm = 0.0;
  if (s < S) {
    const double* x1 = a.x;
    const double* x2 = a.x + NS;
    // field 1 (state rows, forward in time): window of x1 and K x1 at n-1, n-2
    double xm1 = 0.0, xm2 = 0.0, km1 = 0.0, km2 = 0.0;
    for (int n = 0; n < N; ++n) {
      const size_t i = (size_t)n * S + s;
      const double xn = x1[i];
      const double kn = ku_at(a.st, x1 + (size_t)n * S, s);
      double v = xn - 2.0 * xm1 + xm2 + a.c2 * (kn + km2);
      v -= a.beta * (n == 0 ? 0.5 : 1.0) * x2[i];
      if (a.b) { v = a.b[i] - v; nrm = fma(v, v, nrm); }
      a.y[i] = v;
      xm2 = xm1; xm1 = xn; km2 = km1; km1 = kn;
    }
    // field 2 (adjoint rows, backward in time): window at n+1, n+2
    double xp1 = 0.0, xp2 = 0.0, kp1 = 0.0, kp2 = 0.0;
    for (int n = N - 1; n >= 0; --n) {
      const size_t i = (size_t)n * S + s;
      const double xn = x2[i];
      const double kn = ku_at(a.st, x2 + (size_t)n * S, s);
      double v = xn - 2.0 * xp1 + xp2 + a.c2 * (kn + kp2);
      v += a.beta * (n == N - 1 ? 0.5 : 1.0) * x1[i];
      if (a.b) { v = a.b[NS + i] - v; nrm = fma(v, v, nrm); }
      a.y[NS + i] = v;
      xp2 = xp1; xp1 = xn; kp2 = kp1; kp1 = kn;
    }
  }
  if (a.norm2) {
    for (int o = 16; o > 0; o >>= 1) nrm += __shfl_xor_sync(0xffffffffu, nrm, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(a.norm2, nrm);
  }
}

// y = a x on the first half, y = x on the second (balancing of the two fields)
__global__ void k_ctl_scale_half(double a, const double* x, double* y, size_t n) {
  const size_t i = (size_t)blockIdx.x * CT_TB + threadIdx.x;
  if (i < 2 * n) y[i] = i < n ? a * x[i] : x[i];
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct pdc_plan {
  pd_plan* tp = nullptr;          // time transforms (alpha = 1): K1 / K3 standalone
  pd_plan* rp = nullptr;          // step (b) on 2 Nh rows with shifts sigma_+-
  int nt = 0, nh = 0, S = 0;
  bool fp64 = false;
  double T = 0, dt = 0, gamma = 0, beta = 0;
  void* specB = nullptr;          // spectrum of the second field
  void* tab = nullptr;            // per k: phi, 1/d2
  // GMRES workspace
  double* V = nullptr;
  double* Z = nullptr;
  double* w = nullptr;            // balanced rhs / solution
  double* x = nullptr;
  double* dsc = nullptr;          // device scalars
  double* hsc = nullptr;          // pinned host scalars
  int gm_cap = 0;
  unsigned long long launches = 0;
  char msg[256] = {0};
};

namespace {

constexpr int CSC = 96;

pd_status pc_err(pdc_plan* q, pd_status s, const char* what) {
  if (q) snprintf(q->msg, sizeof(q->msg), "%s", what);
  return s;
}
pd_status pc_cuda(pdc_plan* q, cudaError_t e, const char* what) {
  if (q) snprintf(q->msg, sizeof(q->msg), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
}
#define PCCU(call)                                        \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    if (e_ != cudaSuccess) return pc_cuda(q, e_, #call);  \
  } while (0)
#define PCLK(call)                                        \
  do {                                                    \
    cudaError_t e_ = (call);                              \
    ++q->launches;                                        \
    if (e_ != cudaSuccess) return pc_cuda(q, e_, #call);  \
  } while (0)
#define PCCHK(call)               \
  do {                            \
    pd_status s_ = (call);        \
    if (s_ != PD_OK) return s_;   \
  } while (0)

void free_pc(pdc_plan* q) {
  if (!q) return;
  void* ptrs[] = {q->specB, q->tab, q->V, q->Z, q->w, q->x, q->dsc};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (q->hsc) cudaFreeHost(q->hsc);
  if (q->tp) pd_plan_destroy(q->tp);
  if (q->rp) pd_plan_destroy(q->rp);
  delete q;
}

size_t n2(const pdc_plan* q) { return (size_t)2 * q->nt * q->S; }

MixArgs mix_args(const pdc_plan* q) {
  MixArgs m;
  memset(&m, 0, sizeof(m));
  m.nh = q->nh;
  m.specS = q->tp->sg.specS;
  m.tab = q->tab;
  m.A = q->tp->spec;
  m.B = q->specB;
  m.Z = q->rp->spec;
  if (q->rp->xform_tc) {
    m.amax = q->rp->amax;
    m.amax_reset = q->rp->amax + 1;
  }
  return m;
}

pd_status sub_status(pdc_plan* q, pd_plan* p, pd_status s) {
  if (s != PD_OK) snprintf(q->msg, sizeof(q->msg), "%s", pd_last_error(p));
  return s;
}

// z = P^{-1} r (both fields), r, z = [2][Nt][S] FP64
pd_status precond(pdc_plan* q, const double* r, double* z) {
  pd_plan* tp = q->tp;
  cudaStream_t st = tp->stream;
  const size_t ns = (size_t)q->nt * q->S;
  FwdArgs fa = plan_fwd_args(tp);
  fa.mode = FWD_STANDALONE;
  fa.amax = nullptr;
  fa.amax_reset = nullptr;
  fa.r64 = r;
  fa.out = tp->spec;
  PCLK(launch_time_fwd(fa, q->fp64, st));
  fa.r64 = r + ns;
  fa.out = q->specB;
  PCLK(launch_time_fwd(fa, q->fp64, st));
  const MixArgs m = mix_args(q);
  const unsigned grid = (unsigned)(((size_t)q->nh * m.specS + CT_TB - 1) / CT_TB);
  if (q->fp64) k_ctl_mix_in<double><<<grid, CT_TB, 0, st>>>(m);
  else k_ctl_mix_in<float><<<grid, CT_TB, 0, st>>>(m);
  PCLK(cudaGetLastError());
  const unsigned long long before = q->rp->launches;
  PCCHK(sub_status(q, q->rp, plan_step_b(q->rp)));
  q->launches += q->rp->launches - before;
  if (q->fp64) k_ctl_mix_out<double><<<grid, CT_TB, 0, st>>>(m);
  else k_ctl_mix_out<float><<<grid, CT_TB, 0, st>>>(m);
  PCLK(cudaGetLastError());
  InvArgs ia = plan_inv_args(tp);
  ia.mode = INV_OUT64;
  ia.in = tp->spec;
  ia.out64 = z;
  PCLK(launch_time_inv(ia, q->fp64, st));
  ia.in = q->specB;
  ia.out64 = z + ns;
  PCLK(launch_time_inv(ia, q->fp64, st));
  return PD_OK;
}

CtlApply apply_args(const pdc_plan* q) {
  CtlApply a;
  memset(&a, 0, sizeof(a));
  a.N = q->nt;
  a.S = q->S;
  a.st = q->tp->st;
  a.beta = q->beta;
  a.c2 = q->dt * q->dt / 2.0;
  return a;
}

pd_status apply(pdc_plan* q, const double* x, double* y, const double* b, double* norm2) {
  CtlApply a = apply_args(q);
  a.x = x;
  a.y = y;
  a.b = b;
  a.norm2 = norm2;
  k_ctl_apply<<<(q->S + CT_TB - 1) / CT_TB, CT_TB, 0, q->tp->stream>>>(a);
  PCLK(cudaGetLastError());
  return PD_OK;
}

pd_status ensure_gmres(pdc_plan* q, int m) {
  if (q->gm_cap >= m) return PD_OK;
  if (q->V) { cudaFree(q->V); q->V = nullptr; }
  if (q->Z) { cudaFree(q->Z); q->Z = nullptr; }
  const size_t n = n2(q);
  PCCU(cudaMalloc((void**)&q->V, (size_t)(m + 1) * n * sizeof(double)));
  PCCU(cudaMalloc((void**)&q->Z, (size_t)m * n * sizeof(double)));
  q->gm_cap = m;
  return PD_OK;
}

pd_status sync_scalars(pdc_plan* q, int first, int count) {
  cudaStream_t st = q->tp->stream;
  PCCU(cudaMemcpyAsync(q->hsc + first, q->dsc + first, count * sizeof(double),
                       cudaMemcpyDeviceToHost, st));
  PCCU(cudaMemcpyAsync(q->hsc + CSC - 1, q->tp->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  PCCU(cudaMemcpyAsync(q->hsc + CSC - 2, q->rp->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
  PCCU(cudaStreamSynchronize(st));
  return PD_OK;
}

// device flags of the time transforms and of step (b): bit 0 a non-finite
// value, bit 1 an expired wait in the tensor-core x-transform
int flag_of(const pdc_plan* q) {
  int f, g;
  memcpy(&f, q->hsc + CSC - 1, sizeof(int));
  memcpy(&g, q->hsc + CSC - 2, sizeof(int));
  return f | g;
}

// GMRES(m) on the balanced system A x = b (FP64).  right: flexible GMRES on
// A P^{-1}, stopping on ||b - A x|| / ||b||.  left: GMRES on P^{-1} A x =
// P^{-1} b, stopping on ||P^{-1}(b - A x)|| / ||P^{-1} b||, x = x0 + V y (Z
// serves as scratch).
pd_status fgmres(pdc_plan* q, const double* b, double* x, double tol, int maxit, int restart,
                 int* iters, double* relres, bool left = false) {
  const size_t n = n2(q);
  cudaStream_t st = q->tp->stream;
  int m = restart > 0 ? restart : 30;
  m = std::min(m, std::max(1, maxit));
  PCCHK(ensure_gmres(q, m));
  PCCU(cudaMemsetAsync(q->dsc, 0, 3 * sizeof(double), st));
  PCCU(cudaMemsetAsync(q->tp->dflag, 0, sizeof(int), st));
  PCCU(cudaMemsetAsync(q->rp->dflag, 0, sizeof(int), st));
  if (left) {
    // ||P^{-1} b||
    PCCHK(precond(q, b, q->Z));
    PCLK(launch_norm2(q->Z, n, q->dsc, st));
  } else {
    PCLK(launch_norm2(b, n, q->dsc, st));
  }
  PCCHK(sync_scalars(q, 0, 1));
  const double nb = std::sqrt(q->hsc[0]);
  if (nb == 0.0) {
    PCCU(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    PCCU(cudaStreamSynchronize(st));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return PD_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int total = 0;
  double rel = 0.0;
  pd_status status = PD_OK;
  for (;;) {
    PCCU(cudaMemsetAsync(q->dsc + 1, 0, sizeof(double), st));
    if (left) {
      // V_0 = P^{-1}(b - A x)
      PCCHK(apply(q, x, q->Z, b, nullptr));
      PCCHK(precond(q, q->Z, q->V));
      PCLK(launch_norm2(q->V, n, q->dsc + 1, st));
    } else {
      PCCHK(apply(q, x, q->V, b, q->dsc + 1));
    }
    PCCHK(sync_scalars(q, 1, 1));
    const double beta = std::sqrt(q->hsc[1]);
    rel = beta / nb;
    if (!std::isfinite(rel)) { status = pc_err(q, PD_ERR_NONFINITE, "non-finite value in GMRES"); break; }
    if (rel <= tol) break;
    if (total >= maxit) { status = pc_err(q, PD_ERR_NOT_CONVERGED, "GMRES reached maxit"); break; }
    PCLK(launch_scale_copy(1.0 / beta, q->V, q->V, n, st));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = q->V + (size_t)j * n;
      double* Zj = q->Z + (size_t)j * n;
      double* w = q->V + (size_t)(j + 1) * n;
      if (left) {
        PCCHK(apply(q, Vj, Zj, nullptr, nullptr));
        PCCHK(precond(q, Zj, w));
      } else {
        PCCHK(precond(q, Vj, Zj));
        PCCHK(apply(q, Zj, w, nullptr, nullptr));
      }
      for (int pass = 0; pass < 2; ++pass) {
        PCCU(cudaMemsetAsync(q->dsc + 8, 0, (j + 1) * sizeof(double), st));
        PCLK(launch_dots(q->V, j + 1, n, w, q->dsc + 8, st));
        PCLK(launch_gemv_sub(q->V, j + 1, n, q->dsc + 8, w, st));
        PCCHK(sync_scalars(q, 8, j + 1));
        for (int i = 0; i <= j; ++i) Hat(i, j) += q->hsc[8 + i];
      }
      PCCU(cudaMemsetAsync(q->dsc + 2, 0, sizeof(double), st));
      PCLK(launch_norm2(w, n, q->dsc + 2, st));
      PCCHK(sync_scalars(q, 2, 1));
      const int fl = flag_of(q);
      if (fl & 2) return pc_err(q, PD_ERR_CUDA, "a bounded wait of the tensor-core x-transform expired");
      if (fl != 0) return pc_err(q, PD_ERR_NONFINITE, "non-finite value in the preconditioner");
      const double hn = std::sqrt(q->hsc[2]);
      Hat(j + 1, j) = hn;
      if (hn > 0.0) PCLK(launch_scale_copy(1.0 / hn, w, w, n, st));
      for (int i = 0; i < j; ++i) {
        const double t = cs[i] * Hat(i, j) + sn[i] * Hat(i + 1, j);
        Hat(i + 1, j) = -sn[i] * Hat(i, j) + cs[i] * Hat(i + 1, j);
        Hat(i, j) = t;
      }
      const double den = std::hypot(Hat(j, j), Hat(j + 1, j));
      cs[j] = den > 0 ? Hat(j, j) / den : 1.0;
      sn[j] = den > 0 ? Hat(j + 1, j) / den : 0.0;
      Hat(j, j) = den;
      Hat(j + 1, j) = 0.0;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      ++total;
      jdone = j + 1;
      if (std::fabs(g[j + 1]) <= tol * nb || total >= maxit || hn == 0.0) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < jdone; ++k) s -= Hat(i, k) * y[k];
      y[i] = Hat(i, i) != 0.0 ? s / Hat(i, i) : 0.0;
    }
    for (int i = 0; i < jdone; ++i) q->hsc[8 + i] = y[i];
    PCCU(cudaMemcpyAsync(q->dsc + 8, q->hsc + 8, jdone * sizeof(double), cudaMemcpyHostToDevice, st));
    PCLK(launch_combine(left ? q->V : q->Z, jdone, n, q->dsc + 8, x, st));
  }
  PCCU(cudaStreamSynchronize(st));
  if (iters) *iters = total;
  if (relres) *relres = rel;
  return status;
}

}  // namespace

extern "C" {

pd_status pdc_plan_create(const pd_space* sp, int nt, double T, double gamma, int precision,
                          void* stream, pdc_plan** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (!sp || nt < 3) return PD_ERR_ARG;
  if (!(T > 0.0) || !std::isfinite(T) || !(gamma > 0.0) || !std::isfinite(gamma)) return PD_ERR_ARG;
  if (precision != PD_FP64 && precision != PD_MIXED) return PD_ERR_ARG;
  if (nt % 4 == 0) return PD_ERR_UNSUPPORTED;   // C2 singular at k = Nt/4
  pdc_plan* q = new (std::nothrow) pdc_plan();
  if (!q) return PD_ERR_NOMEM;
  q->nt = nt;
  q->T = T;
  q->dt = T / nt;
  q->gamma = gamma;
  q->beta = q->dt * q->dt / std::sqrt(gamma);
  q->fp64 = precision == PD_FP64;
  q->nh = nt / 2 + 1;
  const int nh = q->nh;
  // circulant spectra and the per-frequency blocks (FP64, host)
  const double PI = 3.14159265358979323846;
  std::vector<cdc> tab((size_t)2 * nh);
  std::vector<double> lam((size_t)8 * nh, 0.0);
  const double c2w = q->dt * q->dt / 2.0;
  for (int k = 0; k < nh; ++k) {
    const cdc w = std::polar(1.0, -2.0 * PI * k / nt);
    const cdc d1 = 1.0 - 2.0 * w + w * w;
    const cdc d2 = c2w * (1.0 + w * w);
    const double ad2 = std::abs(d2);
    if (!(ad2 > 1e-12 * c2w)) { delete q; return PD_ERR_UNSUPPORTED; }
    const double l = (d1 / d2).real();
    tab[2 * k] = d2 / ad2;       // phi
    tab[2 * k + 1] = 1.0 / d2;
    const cdc sp_ = cdc(l, q->beta / ad2), sm_ = cdc(l, -q->beta / ad2);
    lam[4 * k] = sp_.real(); lam[4 * k + 1] = sp_.imag(); lam[4 * k + 2] = 1.0;
    lam[4 * (nh + k)] = sm_.real(); lam[4 * (nh + k) + 1] = sm_.imag(); lam[4 * (nh + k) + 2] = 1.0;
  }
  pd_status s = plan_create_internal(sp, nt, q->dt, 1.0, PD_LEAPFROG, 0.5, precision, stream,
                                     false, &q->tp);
  if (s == PD_OK)
    s = plan_create_internal(sp, 2 * nh, q->dt, 1.0, PD_BE, 1.0, precision, stream, false,
                             &q->rp, lam.data());
  if (s != PD_OK) {
    free_pc(q);
    return s;
  }
  q->S = q->tp->S;
  const size_t cb = q->fp64 ? sizeof(double2) : sizeof(float2);
  cudaError_t e = cudaMalloc(&q->specB, (size_t)nh * q->tp->sg.specS * cb);
  if (e == cudaSuccess) e = cudaMalloc(&q->tab, tab.size() * cb);
  if (e == cudaSuccess) {
    if (q->fp64) {
      e = cudaMemcpy(q->tab, tab.data(), tab.size() * sizeof(double2), cudaMemcpyHostToDevice);
    } else {
      std::vector<float2> tf(tab.size());
      for (size_t i = 0; i < tab.size(); ++i) tf[i] = make_float2((float)tab[i].real(), (float)tab[i].imag());
      e = cudaMemcpy(q->tab, tf.data(), tf.size() * sizeof(float2), cudaMemcpyHostToDevice);
    }
  }
  if (e == cudaSuccess) e = cudaMalloc((void**)&q->w, n2(q) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&q->x, n2(q) * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&q->dsc, CSC * sizeof(double));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&q->hsc, CSC * sizeof(double));
  if (e != cudaSuccess) {
    pc_cuda(q, e, "allocation");
    free_pc(q);
    return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
  }
  *out = q;
  return PD_OK;
}

pd_status pdc_plan_destroy(pdc_plan* q) {
  if (!q) return PD_ERR_ARG;
  if (q->tp && q->tp->stream) cudaStreamSynchronize(q->tp->stream);
  else cudaDeviceSynchronize();
  free_pc(q);
  return PD_OK;
}

pd_status pdc_apply_A(pdc_plan* q, const double* x, double* y) {
  if (!q || !x || !y) return PD_ERR_ARG;
  return apply(q, x, y, nullptr, nullptr);
}

pd_status pdc_apply_precond(pdc_plan* q, const double* r, double* z) {
  if (!q || !r || !z) return PD_ERR_ARG;
  return precond(q, r, z);
}

pd_status solve_side(pdc_plan* q, const double* b, double* x, double tol, int maxit,
                     int restart, int* iters, double* relres, bool left);

pd_status pdc_solve(pdc_plan* q, const double* b, double* x, double tol, int maxit, int restart,
                    int* iters, double* relres) {
  PdRange range("pd.control_solve");
  return solve_side(q, b, x, tol, maxit, restart, iters, relres, false);
}

pd_status pdc_solve_left(pdc_plan* q, const double* b, double* x, double tol, int maxit,
                         int restart, int* iters, double* relres) {
  return solve_side(q, b, x, tol, maxit, restart, iters, relres, true);
}

}  // extern "C"

pd_status solve_side(pdc_plan* q, const double* b, double* x, double tol, int maxit,
                     int restart, int* iters, double* relres, bool left) {
  if (!q || !b || !x) return PD_ERR_ARG;
  if (!(tol >= 0.0) || maxit < 0 || restart < 0 || restart > 64) return PD_ERR_ARG;
  const size_t ns = (size_t)q->nt * q->S;
  const double sg = std::sqrt(q->gamma);
  cudaStream_t st = q->tp->stream;
  const unsigned grid = (unsigned)((2 * ns + CT_TB - 1) / CT_TB);
  // balanced right-hand side (gamma^{1/2} f, g), zero initial guess
  k_ctl_scale_half<<<grid, CT_TB, 0, st>>>(sg, b, q->w, ns);
  PCLK(cudaGetLastError());
  PCCU(cudaMemsetAsync(q->x, 0, 2 * ns * sizeof(double), st));
  const pd_status s = fgmres(q, q->w, q->x, tol, maxit, restart, iters, relres, left);
  if (s != PD_OK && s != PD_ERR_NOT_CONVERGED) return s;
  k_ctl_scale_half<<<grid, CT_TB, 0, st>>>(1.0 / sg, q->x, x, ns);
  PCLK(cudaGetLastError());
  PCCU(cudaStreamSynchronize(st));
  return s;
}

extern "C" {

pd_status pdc_launches(const pdc_plan* q, unsigned long long* count) {
  if (!q || !count) return PD_ERR_ARG;
  *count = q->launches;
  return PD_OK;
}

const char* pdc_last_error(const pdc_plan* q) { return q ? q->msg : "null plan"; }

}  // extern "C"
