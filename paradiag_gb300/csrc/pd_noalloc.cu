// pd_apply_precond_noalloc: z = P_alpha^{-1} r for a 1D Dirichlet problem
// without any device allocation, for callers that cannot call cudaMalloc
// (for example code that runs while an application's memory pool is frozen,
// plug-ins whose host owns every device allocation, or callers inside a
// region where allocation is forbidden).  The scratch that the plan-based path
// allocates (the half spectrum and the eigenvalue / Gamma / twiddle tables)
// lives here in one file-scope __device__ array of fixed size, which every GPU
// that loads this library holds until the process exits.
//
// The kernels are the same as the plan-based mixed-precision path: the
// residual-free forward time kernel, the shifted tridiagonal solver along x,
// and the inverse time kernel writing z in FP64.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <vector>

#include "pd_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[PD_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {nullptr};  // device address of the array, per device

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Device address of the static scratch on the current device (looked up once
// per device; host code may not use the symbol itself as an address).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (g_noalloc_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" pd_status pd_apply_precond_noalloc(const pd_space* sp, int nt, double dt, double alpha,
                                              int scheme, double theta, const double* r,
                                              double* z, void* stream,
                                              unsigned long long* scratch_needed) {
  if (!sp || !r || !z) return PD_ERR_ARG;
  if (sp->dim != 1 || sp->bc_x != PD_DIRICHLET || sp->nx < 1) return PD_ERR_UNSUPPORTED;
  if (!(sp->nu >= 0.0) || !(sp->lx > 0.0) || !std::isfinite(sp->ax)) return PD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt) || !(alpha > 0.0 && alpha <= 1.0)) return PD_ERR_ARG;
  if (scheme < PD_BE || scheme > PD_LEAPFROG) return PD_ERR_ARG;
  if (scheme == PD_THETA && !(theta >= 0.0 && theta <= 1.0)) return PD_ERR_ARG;
  // the plan path's mixed-precision limits: a time tile holds at most 4096
  // rows (two columns of 16 complex elements per thread), and a tridiagonal
  // system at most TRI_NMAX rows
  if (nt < 1 || !is_pow2(nt) || nt > 4096) return PD_ERR_UNSUPPORTED;
  if (sp->nx > TRI_NMAX) return PD_ERR_UNSUPPORTED;

  const int nx = sp->nx, S = nx, nh = nt / 2 + 1;
  // scratch layout: spectrum | lambda pairs | gamma | gamma^-1/Nt | twiddles | flag
  const size_t off_spec = 0;
  const size_t off_lam = align256(off_spec + (size_t)nh * S * sizeof(float2));
  const size_t off_gam = align256(off_lam + (size_t)2 * nh * sizeof(float2));
  const size_t off_igam = align256(off_gam + (size_t)nt * sizeof(float));
  const size_t off_tw = align256(off_igam + (size_t)nt * sizeof(float));
  const size_t off_flag = align256(off_tw + (size_t)nt * sizeof(float2));
  const size_t need = off_flag + sizeof(int);
  if (scratch_needed) *scratch_needed = need;
  if (need > (size_t)PD_NOALLOC_SCRATCH_BYTES) return PD_ERR_ARG;

  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return PD_ERR_CUDA;
  unsigned char* b = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)stream;

  // operator and time-band coefficients (as in pd_plan_create)
  const double h = sp->lx / (nx + 1);
  const double kc = 2.0 * sp->nu / (h * h);
  const double kl = -sp->nu / (h * h) - sp->ax / (2.0 * h);
  const double ku = -sp->nu / (h * h) + sp->ax / (2.0 * h);
  double c1[3] = {0, 0, 0}, c2[3] = {0, 0, 0};
  int band = 1;
  const double th = scheme == PD_BE ? 1.0 : scheme == PD_CN ? 0.5 : theta;
  if (scheme == PD_LEAPFROG) {
    band = 2;
    c1[0] = 1.0 / (dt * dt); c1[1] = -2.0 / (dt * dt); c1[2] = 1.0 / (dt * dt);
    c2[0] = 0.5; c2[2] = 0.5;
  } else {
    c1[0] = 1.0 / dt; c1[1] = -1.0 / dt;
    c2[0] = th; c2[1] = 1.0 - th;
  }

  // host tables: Lemma 1 eigenvalues (half spectrum), Gamma, twiddles
  const double PI = 3.14159265358979323846;
  const double ar = std::pow(alpha, 1.0 / nt);
  std::vector<float2> lam((size_t)2 * nh), tw(nt);
  std::vector<std::complex<double>> lamd((size_t)2 * nh);
  std::vector<float> gam(nt), igam(nt);
  for (int k = 0; k < nh; ++k) {
    const double a = -2.0 * PI * k / nt;
    const std::complex<double> w = ar * std::complex<double>(std::cos(a), std::sin(a));
    std::complex<double> l1 = 0, l2 = 0, wm = 1;
    for (int m = 0; m <= band && m < nt; ++m) {
      l1 += c1[m] * wm;
      l2 += c2[m] * wm;
      wm *= w;
    }
    lamd[2 * k] = l1;
    lamd[2 * k + 1] = l2;
    lam[2 * k] = make_float2((float)l1.real(), (float)l1.imag());
    lam[2 * k + 1] = make_float2((float)l2.real(), (float)l2.imag());
  }
  if (alpha == 1.0) {
    // as pd_plan_create: without the alpha scaling a shifted system
    // lambda_1 + lambda_2 mu_i (mu_i = kc + 2 sqrt(kl ku) cos(pi i / (nx + 1)),
    // the eigenvalues of the tridiagonal K) may be singular; reject it
    const std::complex<double> sq = std::sqrt(std::complex<double>(kl * ku, 0.0));
    for (int k = 0; k < nh; ++k) {
      const std::complex<double> l1 = lamd[2 * k], l2 = lamd[2 * k + 1];
      for (int i = 1; i <= nx; ++i) {
        const std::complex<double> mu = kc + 2.0 * sq * std::cos(PI * i / (nx + 1));
        const double sc = std::abs(l1) + std::abs(l2) * std::abs(mu) + 1e-300;
        if (std::abs(l1 + l2 * mu) <= 1e-12 * sc) return PD_ERR_ARG;
      }
    }
  }
  for (int n = 0; n < nt; ++n) {
    gam[n] = (float)std::pow(alpha, (double)n / nt);
    igam[n] = (float)(std::pow(alpha, -(double)n / nt) / nt);
    const double a = -2.0 * PI * n / nt;
    tw[n] = make_float2((float)std::cos(a), (float)std::sin(a));
  }
  if (cudaMemcpyAsync(b + off_lam, lam.data(), lam.size() * sizeof(float2),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b + off_gam, gam.data(), gam.size() * sizeof(float), cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemcpyAsync(b + off_igam, igam.data(), igam.size() * sizeof(float),
                      cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(b + off_tw, tw.data(), tw.size() * sizeof(float2), cudaMemcpyHostToDevice,
                      st) != cudaSuccess ||
      cudaMemsetAsync(b + off_flag, 0, sizeof(int), st) != cudaSuccess)
    return PD_ERR_CUDA;

  FwdArgs fa;
  memset(&fa, 0, sizeof(fa));
  fa.N = nt; fa.logN = ilog2(nt); fa.nh = nh; fa.S = S;
  fa.sg.specS = S; fa.sg.nx = nx; fa.sg.nxp = nx;
  fa.TX = std::max(2, std::min(32, 8192 / nt));
  fa.st.dim = 1; fa.st.nx = nx; fa.st.ny = 1; fa.st.S = S; fa.st.bcx = PD_DIRICHLET;
  fa.st.bcy = PD_DIRICHLET; fa.st.kc = kc; fa.st.kxl = kl; fa.st.kxu = ku;
  fa.tb.band = band;
  for (int m = 0; m < 3; ++m) { fa.tb.c1[m] = c1[m]; fa.tb.c2[m] = c2[m]; }
  fa.mode = FWD_STANDALONE;
  fa.r64 = r;
  fa.gam = b + off_gam;
  fa.tw = b + off_tw;
  fa.out = b + off_spec;
  if (launch_time_fwd(fa, false, st) != cudaSuccess) return PD_ERR_CUDA;

  TriArgs ta;
  ta.nh = nh; ta.J = 1; ta.n = nx; ta.S = S; ta.stride = 1;
  ta.cl = kl; ta.cd = kc; ta.cu = ku;
  ta.lam = b + off_lam; ta.mu = nullptr; ta.data = b + off_spec;
  ta.flag = reinterpret_cast<int*>(b + off_flag);
  if (launch_tridiag(ta, false, st) != cudaSuccess) return PD_ERR_CUDA;

  InvArgs ia;
  memset(&ia, 0, sizeof(ia));
  ia.N = nt; ia.logN = fa.logN; ia.nh = nh; ia.S = S; ia.TX = fa.TX;
  ia.sg = fa.sg;
  ia.mode = INV_OUT64;
  ia.in = b + off_spec;
  ia.igam = b + off_igam;
  ia.tw = b + off_tw;
  ia.out64 = z;
  ia.flag = reinterpret_cast<int*>(b + off_flag);
  if (launch_time_inv(ia, false, st) != cudaSuccess) return PD_ERR_CUDA;
  // the device flag (bit 0: a non-finite value in r, the spectrum or z) is
  // read back, so the call returns once its work on the stream has finished
  int flag = 0;
  if (cudaMemcpyAsync(&flag, b + off_flag, sizeof(int), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return PD_ERR_CUDA;
  return flag != 0 ? PD_ERR_NONFINITE : PD_OK;
}
