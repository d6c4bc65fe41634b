// Internal definitions shared by the host API and the kernel launchers.
#pragma once
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include "../../include/paradiag.h"
#include "pd_common.cuh"

// NVTX ranges around the solver phases (header-only NVTX 3: a range costs a
// few instructions unless a profiling tool is attached, which then records
// it).  Names are prefixed "pd." and follow the paper's steps: "pd.residual"
// (r = b - A u, eq. 5.1, fused with step (a)), "pd.step_a" (Gamma and the FFT
// along time), "pd.step_b" (the shifted solves, with the x-eigentransform),
// "pd.step_c" (inverse FFT, Gamma^{-1}, update), and one range per solve.
#include <nvtx3/nvToolsExt.h>
struct PdRange {
  explicit PdRange(const char* name) { nvtxRangePushA(name); }
  ~PdRange() { nvtxRangePop(); }
  PdRange(const PdRange&) = delete;
  PdRange& operator=(const PdRange&) = delete;
};

// Double-float constant (value = hi + lo) prepared on the host.
struct dfc { float hi, lo; };
static inline dfc dfc_from(double v) {
  dfc c; c.hi = (float)v; c.lo = (float)(v - (double)c.hi); return c;
}

// Spatial operator K of the all-at-once system (M = I), constant coefficients:
// K u(s) = kc u(s) + kxl u(x-1) + kxu u(x+1) + kyl u(y-1) + kyu u(y+1).
struct Stencil {
  int dim, nx, ny, S, bcx, bcy;
  double kc, kxl, kxu, kyl, kyu;
};

// Time-band coefficients: (A u)_n = sum_{m<=band} c1[m] U_{n-m} + K sum_m c2[m] U_{n-m}.
struct TimeBand {
  int band;          // 1 (theta-method) or 2 (leap-frog)
  double c1[3], c2[3];
};

// Spectrum layout: entry (k, s) of the half spectrum lives at
// k * specS + (s / nx) * nxp + s % nx (nxp >= nx pads every grid line of the
// x-transformed problems to an even length so rows are 16-byte aligned).
struct SpecGeom {
  int specS, nx, nxp;
};
PD_HD size_t spec_index(const SpecGeom& g, int k, int s) {
  const int off = (g.nxp == g.nx) ? s : (s / g.nx) * g.nxp + (s % g.nx);
  return (size_t)k * g.specS + off;
}

// Arguments of the forward time kernel (K1).
// Time transform of length N: a power-of-two Stockham FFT when M == 0;
// otherwise Bluestein's chirp-z form, two power-of-two FFTs of length
// M >= 2N - 1 (logM) with the chirp w_n = exp(-i pi n^2 / N) and the
// transformed filter bhat = FFT_M(conj chirp, wrapped) / M; tw then holds the
// M-point twiddles.
struct TimeXf {
  int M, logM;
  const void* chirp;
  const void* bhat;
};

struct FwdArgs {
  int N, logN, nh, S, TX;
  TimeXf xf;
  SpecGeom sg;
  Stencil st;
  TimeBand tb;
  int mode;                       // FWD_STANDALONE or FWD_RESIDUAL
  const double* r64;              // standalone input r (FP64, [N][S])
  const float2* Udf;              // mixed residual: iterate as double-float [N][S]
  const float2* Bdf;              // mixed residual: s*b as double-float [N][S]
  const double* U64;              // FP64 residual: iterate
  const double* B64;              // FP64 residual: b
  dfc kap[5];                     // mixed: s*K coefficients (c, xl, xu, yl, yu)
  dfc e2[3];                      // mixed: c2[m]
  int c2exact = 0;                // mixed: every c2[m] is 0 or a power of two
  double rscale2;                 // mixed: 1/s^2 (norm of r' = s r)
  const void* gam;                // gamma_n (float or double)
  const void* tw;                 // e^{-2 pi i m / N}, m < N (float2 or double2)
  void* out;                      // half spectrum [nh][S] (float2 or double2)
  double* norm2;                  // += ||r||_2^2 (may be null)
  // mixed path with the tensor-core x-transform: max |out| (float bits) is
  // raised into *amax, and *amax_reset (the other transform's word) is zeroed
  unsigned* amax = nullptr;
  unsigned* amax_reset = nullptr;
  const int* mode_dev = nullptr;  // if set, the mode is read from device memory
  int CR = 1;                     // blocks per tile (a cluster; 0 or 1: one block)
};

// Arguments of the inverse time kernel (K3).
struct InvArgs {
  int N, logN, nh, S, TX;
  TimeXf xf;
  SpecGeom sg;
  int mode;                       // INV_UPDATE_DF, INV_OUT64, INV_UPDATE64
  const void* in;                 // half spectrum [nh][S]
  const void* igam;               // gamma_n^{-1} / N (float or double)
  const void* tw;
  float2* Udf;                    // mixed: iterate (double-float), updated in place
  double* out64;                  // FP64 output (z) or FP64 iterate (updated)
  int* flag;                      // bit 0 set on a non-finite value (may be null)
  const int* mode_dev = nullptr;  // if set, the mode is read from device memory
  int CR = 1;                     // blocks per tile (a cluster; 0 or 1: one block)
};

// FWD_RESIDUAL_NORM: the residual and its norm only (no transform, no spectrum)
// FWD_ZERO_GUESS: the residual of a zero iterate, r = s b (no iterate loads,
// no stencil; the same arithmetic as FWD_RESIDUAL with U = 0, mixed path only)
enum { FWD_STANDALONE = 0, FWD_RESIDUAL = 1, FWD_RESIDUAL_NORM = 2, FWD_ZERO_GUESS = 3 };
// INV_SET_DF: U = z (the first update of a zero iterate; equal to INV_UPDATE_DF
// on U = 0 without reading U)
enum { INV_UPDATE_DF = 0, INV_OUT64 = 1, INV_UPDATE64 = 2, INV_SET_DF = 3 };

// Arguments of the batched shifted tridiagonal solve (K2, step (b)).
// System q = k*J + j (k < nh time frequencies, j < J spatial modes) of length n:
//   l z_{i-1} + d z_i + u z_{i+1} = s_i, l = lam2_k cl, d = lam1_k + lam2_k (cd + mu_j),
//   u = lam2_k cu; element i lives at base + k*S + j + i*stride.
struct TriArgs {
  int nh, J, n, S, stride;
  double cl, cd, cu;
  const void* lam;                // [nh] complex pairs (lam1, lam2) as 2 complex each
  const void* mu;                 // [J] complex spatial eigenvalues (or null: 0)
  void* data;                     // in: right-hand sides, out: solutions
  int* flag;
  // as in FwdArgs: max |solution| raised into *amax, *amax_reset zeroed (FP32 only)
  unsigned* amax = nullptr;
  unsigned* amax_reset = nullptr;
  // lane class (2^cls lanes per system) chosen by the plan's autotuner, or -1
  // for the default tridiag_class(n); never below the default
  int cls = -1;
  // FP32 only: rows per lane held in registers, 16 for the short-chunk form
  // (lane classes then count from tridiag_class(n, false, 16)), 0 for the default
  int rows = 0;
};

// Arguments of the dense x-eigentransform (2D, step (a') / (c')): along x, for
// every row of the half spectrum: out[row][j] = sum_x Q[j][x] in[row][x].
struct XformArgs {
  int rows, nx, ld;                // ld: row stride in complex elements
  const void* Q;                  // [nx][nx] complex
  const void* in;
  void* out;
};

// Arguments of the FP64 x-eigentransform by FFT: every row of the half
// spectrum (nx complex values, row stride ld) is transformed by a length-L
// DFT, L = nx for a periodic x direction (the DFT diagonalises the circulant
// K_x) or L = 2 (nx + 1) for a symmetric Dirichlet x direction (the sine
// transform as the DFT of the odd extension).  A power-of-two L uses the
// Stockham FFT directly (xf.M = 0, tw: L twiddles); other lengths Bluestein's
// form with xf (M-point twiddles in tw).
struct XfftArgs {
  int rows, nx, ld, L, logL;
  int dst;                        // 1: sine transform (Dirichlet x), 0: DFT (periodic x)
  int inv;                        // 1: inverse transform (scaled), 0: forward
  TimeXf xf;
  const void* tw;                 // complex twiddles (double2 / float2, as the data)
  const void* in;
  void* out;
  // L = L1 L2 (both <= 32, L not a power of two): one Cooley-Tukey step with
  // two direct DFTs, tw = W_L^m for m < L; 0: Stockham / Bluestein
  int L1 = 0, L2 = 0;
};

// Launchers (return a cudaError_t).
cudaError_t launch_xform_fft(const XfftArgs& a, bool fp64, cudaStream_t st);
cudaError_t launch_time_fwd(const FwdArgs& a, bool fp64, cudaStream_t st);
cudaError_t launch_time_inv(const InvArgs& a, bool fp64, cudaStream_t st);
cudaError_t launch_tridiag(const TriArgs& a, bool fp64, cudaStream_t st);
cudaError_t launch_xform(const XformArgs& a, bool fp64, cudaStream_t st);

// Batched launches: work[b] = (problem, tile) for block b; descs in device memory.
int time_tile_ept(int N, int TX);
size_t time_inv_smem(int N, int rows, int TX, bool fp64, bool upd);
cudaError_t launch_time_fwd_batch(const FwdArgs* descs, const int2* work, int nblocks, int band,
                                  size_t smem, int ept, bool fp64, cudaStream_t st);
cudaError_t launch_time_inv_batch(const InvArgs* descs, const int2* work, int nblocks,
                                  size_t smem, int ept, bool fp64, cudaStream_t st);  // smem: time_inv_smem
// Tridiagonal systems of length n <= TRI_NMAX are solved by 2^cls lanes each,
// cls = tridiag_class(n, fp64) < TRI_NCLASS; a batch groups its problems by
// class and launches tiles of tridiag_batch_sb(cls) systems of one problem.
constexpr int TRI_NMAX = 4096;
constexpr int TRI_NCLASS = 9;
int tridiag_class(int n, bool fp64, int rows = 0);
int tridiag_batch_sb(int cls, bool fp64);
// persistent: *counter (device, zeroed before the launch) hands out the tiles
cudaError_t launch_tridiag_batch(const TriArgs* descs, const int2* work, int ntiles, int cls,
                                 bool fp64, int* counter, cudaStream_t st);
#include "pd_xform_tc.h"

// Auxiliary kernels (pd_ops.cu)
cudaError_t launch_apply_A(const Stencil& st, const TimeBand& tb, int N, const double* u,
                           const double* b, double* y, double* norm2, int transpose,
                           cudaStream_t s);
cudaError_t launch_build_rhs(const Stencil& st, const TimeBand& tb, int scheme, int N, double dt,
                             const double* u0, const double* u1, const double* f, double* b,
                             cudaStream_t s);
cudaError_t launch_to_df(const double* x, double scale, float2* y, size_t n, cudaStream_t s);
cudaError_t launch_from_df(const float2* x, double* y, size_t n, cudaStream_t s);
// U = split(u), B = split(scale b), *norm2 += ||scale b||^2 (FP32 partial sums)
// nonzero (may be null): set to 1 when some entry of u is not zero
cudaError_t launch_entry_df(const double* u, const double* b, double scale, float2* U, float2* B,
                            size_t n, double* norm2, cudaStream_t s, int* nonzero = nullptr);
cudaError_t launch_norm2(const double* x, size_t n, double* out, cudaStream_t s);
cudaError_t launch_flip_time(const double* x, double* y, int N, int S, cudaStream_t s);
cudaError_t launch_dots(const double* V, int nv, size_t n, const double* w, double* h,
                        cudaStream_t s);
cudaError_t launch_gemv_sub(const double* V, int nv, size_t n, const double* h, double* w,
                            cudaStream_t s);
cudaError_t launch_axpby(double a, const double* x, double b, double* y, size_t n,
                         cudaStream_t s);
cudaError_t launch_scale_copy(double a, const double* x, double* y, size_t n, cudaStream_t s);
cudaError_t launch_combine(const double* Z, int nz, size_t n, const double* y, double* u,
                           cudaStream_t s);
