// ParaDiag-I with geometrically increasing time steps (Section 2.1.1): the
// direct all-at-once solver.
//
// The theta-method with the steps dt_n = dt_Nt tau^(n-Nt) (eq. 2.8) gives
// A = B1 (x) I + B2 (x) K with lower-bidiagonal B1, B2 (eq. 2.5b).  With
// B = B2^{-1} B1 = V D V^{-1} (the theorem of Section 2.1.1, V and V^{-1}
// unit lower-triangular Toeplitz in closed form, D = diag(1/(theta dt_n)))
// and an optional column scaling V -> V D~, the solve A u = r is
//   (a) S1 = (W (x) I) r,  W = D~^{-1} V^{-1} B2^{-1}  (eq. 2.6 and step (a)
//       of eq. 2.7 in one lower-triangular Nt x Nt matrix),
//   (b) S2_n = (1/(theta dt_n) I + K)^{-1} S1_n,  n = 1..Nt,
//   (c) u = (V D~ (x) I) S2.
// Step (b) is the shifted spatial solve of the ParaDiag-II path (the
// x-eigentransform in 2D and the tridiagonal solver), here with real shifts
// lambda_1n = 1/(theta dt_n), lambda_2n = 1 on one spectrum row per time row.
//
// Kernels.  Steps (a) and (c) contract the time index of every spatial point
// with a lower-triangular Nt x Nt matrix (Nt <= 32): about Nt/2 FMAs per
// element moved, below the FP32 CUDA-core ridge of the GPU, so they are
// HBM-bound CUDA-core kernels, one thread per spatial point, the matrix in
// shared memory (broadcast reads) and the Nt partial sums in registers
// (outer-product order: row m of the input updates rows n >= m).  Step (a)
// is fused with the residual r = b - A u of the refinement sweeps
// (double-float on the mixed path, FP64 otherwise) and with ||r||^2;
// step (c) is fused with the update of the iterate.
//
// Precision.  The roundoff of the direct solve grows like Cond_2(V) (Section
// 2.1.1).  PD_FP64 runs every step in FP64.  PD_MIXED runs steps (a)-(c) in
// FP32 and corrects with the residual in double-float: the sweep
// u <- u + P^{-1}(b - A u), P^{-1} the FP32 ParaDiag-I solve, converges when
// Cond(V D~) times the FP32 unit roundoff is well below one.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "pd_plan.h"

namespace {

constexpr int P1_NT = 32;    // largest window: register arrays of the kernels
constexpr int P1_TB = 128;   // threads per block, one spatial point each

enum { P1_DIRECT = 0, P1_RESID = 1, P1_NORM = 2 };
enum { P1_SET = 0, P1_ADD = 1 };

struct P1Fwd {
  int N, S;
  Stencil st;
  SpecGeom sg;
  double theta;
  float th_f, omth_f;           // theta and 1 - theta (exact in FP32: 1, 1/2, 0)
  double c1[P1_NT];             // 1/dt_n
  dfc c1d[P1_NT];               // 1/dt_n as double-float
  dfc kap[5];                   // K coefficients (c, xl, xu, yl, yu) as double-float
  const double* b64;            // right-hand side (FP64)
  const double* u64;            // FP64 iterate
  float2* Bdf;                  // mixed: b as double-float (written by P1_DIRECT)
  const float2* Udf;            // mixed: iterate
  const void* W;                // [N][N]: W[m * N + n] = (step (a) matrix)[n][m]
  void* out;                    // spectrum rows [N][specS], complex
  double* norm2;                // += ||r||^2 (||b||^2 for P1_DIRECT)
  unsigned* amax;               // mixed + tensor-core x-transform: max |S1|
  unsigned* amax_reset;
};

struct P1Inv {
  int N, S;
  SpecGeom sg;
  const void* V;                // [N][N]: V[m * N + n] = (V D~)[n][m]
  const void* in;               // spectrum rows [N][specS], complex (real part used)
  double* u64;
  float2* Udf;
  int* flag;                    // bit 0: a non-finite value
};

// neighbours of spatial point s (x fastest); -1 where the grid has none
struct Nb {
  int l, r, d, u;
};
PD_D Nb neighbours(const Stencil& st, int s) {
  Nb g;
  const int x = s % st.nx, y = s / st.nx;
  g.l = x > 0 ? s - 1 : (st.bcx == PD_PERIODIC ? s + st.nx - 1 : -1);
  g.r = x < st.nx - 1 ? s + 1 : (st.bcx == PD_PERIODIC ? s - (st.nx - 1) : -1);
  g.d = (st.dim == 2 && y > 0) ? s - st.nx : -1;
  g.u = (st.dim == 2 && y < st.ny - 1) ? s + st.nx : -1;
  return g;
}

// (K U)(s) of one time row in FP64
PD_D double ku_64(const Stencil& st, const Nb& g, const double* U, int s) {
  double k = st.kc * __ldg(&U[s]);
  if (g.l >= 0) k = fma(st.kxl, __ldg(&U[g.l]), k);
  if (g.r >= 0) k = fma(st.kxu, __ldg(&U[g.r]), k);
  if (g.d >= 0) k = fma(st.kyl, __ldg(&U[g.d]), k);
  if (g.u >= 0) k = fma(st.kyu, __ldg(&U[g.u]), k);
  return k;
}

template <typename R>
PD_D void load_matrix(R* sM, const void* M, int N) {
  const R* g = reinterpret_cast<const R*>(M);
  for (int i = threadIdx.x; i < P1_NT * P1_NT; i += P1_TB) {
    const int m = i / P1_NT, n = i % P1_NT;
    sM[i] = (m < N && n < N) ? g[m * N + n] : (R)0;
  }
}

PD_D float warp_max(float v) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
PD_D T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Loads of one time row at spatial point s: centre, the four neighbours and b.
// Rows at or beyond N (and points beyond S) read as zero; the loads of all
// rows are independent of the arithmetic, so the unrolled kernels below issue
// them ahead of use.
template <typename V>
struct RowIn {
  V b, c, l, r, d, u;
};
template <typename V>
PD_D RowIn<V> load_row(const V* B, const V* U, const Nb& g, int s, size_t base, bool on) {
  RowIn<V> x;
  const V z{};
  x.b = on ? __ldg(&B[base + s]) : z;
  x.c = on ? __ldg(&U[base + s]) : z;
  x.l = (on && g.l >= 0) ? __ldg(&U[base + g.l]) : z;
  x.r = (on && g.r >= 0) ? __ldg(&U[base + g.r]) : z;
  x.d = (on && g.d >= 0) ? __ldg(&U[base + g.d]) : z;
  x.u = (on && g.u >= 0) ? __ldg(&U[base + g.u]) : z;
  return x;
}

// acc2[j] = (acc[2j], acc[2j+1]) += (M[2j][m], M[2j+1][m]) r for 2j+1 >= m:
// the shared-memory row m (transposed matrix) in aligned float4, paired FMAs
template <int NT>
PD_D void rank1_pair(float2 (&acc)[NT / 2], const float* sM, float r, int m) {
  const float4* row = reinterpret_cast<const float4*>(sM + m * P1_NT);
  const float2 rr = make_float2(r, r);
#pragma unroll
  for (int v = 0; v < NT / 4; ++v) {
    if (4 * v + 3 < m) continue;
    const float4 w = row[v];
    acc[2 * v] = f2fma(make_float2(w.x, w.y), rr, acc[2 * v]);
    acc[2 * v + 1] = f2fma(make_float2(w.z, w.w), rr, acc[2 * v + 1]);
  }
}
template <int NT>
PD_D void rank1_64(double (&acc)[NT], const double* sM, double r, int m) {
  const double2* row = reinterpret_cast<const double2*>(sM + m * P1_NT);
#pragma unroll
  for (int v = 0; v < NT / 2; ++v) {
    if (2 * v + 1 < m) continue;
    const double2 w = row[v];
    acc[2 * v] = fma(w.x, r, acc[2 * v]);
    acc[2 * v + 1] = fma(w.y, r, acc[2 * v + 1]);
  }
}

// ---------------------------------------------------------------------------
// Step (a), fused with the residual.  MODE P1_DIRECT: r = b (and, mixed, the
// double-float copy of b); P1_RESID: r = b - A u; P1_NORM: ||b - A u||^2 only.
// Windows of N <= NT rows; rows are handled in pairs (m, m+1).
// Mixed (PREC 0): the residual in double-float on paired FP32 instructions
// (lane x = row m, lane y = row m+1), the transform in FP32.
// ---------------------------------------------------------------------------
template <int MODE, int NT>
__global__ void __launch_bounds__(P1_TB) k_pd1_fwd_mixed(const P1Fwd a) {
  __shared__ __align__(16) float sW[P1_NT * P1_NT];
  if constexpr (MODE != P1_NORM) {
    load_matrix<float>(sW, a.W, a.N);
    __syncthreads();
  }
  const int N = a.N, S = a.S;
  const int s = blockIdx.x * P1_TB + threadIdx.x;
  const bool valid = s < S;
  const Nb g = neighbours(a.st, valid ? s : 0);
  const K2 kk[5] = {
      {make_float2(a.kap[0].hi, a.kap[0].hi), make_float2(-a.kap[0].hi, -a.kap[0].hi),
       make_float2(-a.kap[0].lo, -a.kap[0].lo)},
      {make_float2(a.kap[1].hi, a.kap[1].hi), make_float2(-a.kap[1].hi, -a.kap[1].hi),
       make_float2(-a.kap[1].lo, -a.kap[1].lo)},
      {make_float2(a.kap[2].hi, a.kap[2].hi), make_float2(-a.kap[2].hi, -a.kap[2].hi),
       make_float2(-a.kap[2].lo, -a.kap[2].lo)},
      {make_float2(a.kap[3].hi, a.kap[3].hi), make_float2(-a.kap[3].hi, -a.kap[3].hi),
       make_float2(-a.kap[3].lo, -a.kap[3].lo)},
      {make_float2(a.kap[4].hi, a.kap[4].hi), make_float2(-a.kap[4].hi, -a.kap[4].hi),
       make_float2(-a.kap[4].lo, -a.kap[4].lo)}};
  const float2 th2 = make_float2(a.th_f, a.th_f), om2 = make_float2(a.omth_f, a.omth_f);

  float2 acc[NT / 2];
#pragma unroll
  for (int j = 0; j < NT / 2; ++j) acc[j] = make_float2(0.f, 0.f);
  float nrm = 0.f;
  // row m-1 (the second row of the previous pair): U and K U (double-float)
  df up = df_make(0.f, 0.f), kup = df_make(0.f, 0.f);

#pragma unroll
  for (int m = 0; m < NT; m += 2) {
    const bool onA = valid && m < N, onB = valid && m + 1 < N;
    float2 r2;
    if constexpr (MODE == P1_DIRECT) {
      const double bA = onA ? __ldg(&a.b64[(size_t)m * S + s]) : 0.0;
      const double bB = onB ? __ldg(&a.b64[(size_t)(m + 1) * S + s]) : 0.0;
      const df dA = df_from_double(bA), dB = df_from_double(bB);
      if (onA) a.Bdf[(size_t)m * S + s] = make_float2(dA.hi, dA.lo);
      if (onB) a.Bdf[(size_t)(m + 1) * S + s] = make_float2(dB.hi, dB.lo);
      r2 = make_float2(dA.hi, dB.hi);
    } else {
      const RowIn<float2> A = load_row(a.Bdf, a.Udf, g, s, (size_t)m * S, onA);
      const RowIn<float2> B = load_row(a.Bdf, a.Udf, g, s, (size_t)(m + 1) * S, onB);
      // (K U) of both rows
      const DF2 uc = df2_pack(A.c, B.c);
      Acc2 ku = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      acc2_add_prod(ku, kk[0], uc);
      acc2_add_prod(ku, kk[1], df2_pack(A.l, B.l));
      acc2_add_prod(ku, kk[2], df2_pack(A.r, B.r));
      acc2_add_prod(ku, kk[3], df2_pack(A.d, B.d));
      acc2_add_prod(ku, kk[4], df2_pack(A.u, B.u));
      const df kuA = fast_two_sum(ku.s.x, ku.e.x), kuB = fast_two_sum(ku.s.y, ku.e.y);
      // r = b - c1 (U_m - U_{m-1}) - theta K U_m - (1 - theta) K U_{m-1}
      const dfc cA = a.c1d[m], cB = a.c1d[m + 1 < P1_NT ? m + 1 : m];
      const K2 c1n = {make_float2(-cA.hi, -cB.hi), make_float2(cA.hi, cB.hi),
                      make_float2(cA.lo, cB.lo)};
      const K2 c1p = {make_float2(cA.hi, cB.hi), make_float2(-cA.hi, -cB.hi),
                      make_float2(-cA.lo, -cB.lo)};
      Acc2 R = {make_float2(A.b.x, B.b.x), make_float2(A.b.y, B.b.y)};
      acc2_add_prod(R, c1n, uc);
      acc2_add_prod(R, c1p, DF2{make_float2(up.hi, A.c.x), make_float2(up.lo, A.c.y)});
      acc2_sub(R, f2mul(th2, make_float2(kuA.hi, kuB.hi)), f2mul(th2, make_float2(kuA.lo, kuB.lo)));
      acc2_sub(R, f2mul(om2, make_float2(kup.hi, kuA.hi)), f2mul(om2, make_float2(kup.lo, kuA.lo)));
      r2 = make_float2(fast_two_sum(R.s.x, R.e.x).hi, fast_two_sum(R.s.y, R.e.y).hi);
      up = df_make(B.c.x, B.c.y);
      kup = kuB;
    }
    if (!onA) r2.x = 0.f;
    if (!onB) r2.y = 0.f;
    nrm = fmaf(r2.x, r2.x, fmaf(r2.y, r2.y, nrm));
    if constexpr (MODE != P1_NORM) {
      rank1_pair<NT>(acc, sW, r2.x, m);
      rank1_pair<NT>(acc, sW, r2.y, m + 1);
    }
  }

  const float wn = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0 && a.norm2 != nullptr) atomicAdd(a.norm2, (double)wn);
  if constexpr (MODE == P1_NORM) return;

  float2* out = reinterpret_cast<float2*>(a.out);
  float amx = 0.f;
  if (valid) {
    const size_t o = spec_index(a.sg, 0, s);
#pragma unroll
    for (int j = 0; j < NT / 2; ++j) {
      if (2 * j < N) {
        out[o + (size_t)(2 * j) * a.sg.specS] = make_float2(acc[j].x, 0.f);
        amx = fmaxf(amx, fabsf(acc[j].x));
      }
      if (2 * j + 1 < N) {
        out[o + (size_t)(2 * j + 1) * a.sg.specS] = make_float2(acc[j].y, 0.f);
        amx = fmaxf(amx, fabsf(acc[j].y));
      }
    }
  }
  if (a.amax != nullptr) {
    amx = warp_max(amx);
    if ((threadIdx.x & 31) == 0) atomicMax(a.amax, __float_as_uint(amx));
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.amax_reset != nullptr) *a.amax_reset = 0u;
  }
}

// FP64 form (PREC 1): every step in FP64.
template <int MODE, int NT>
__global__ void __launch_bounds__(P1_TB) k_pd1_fwd_64(const P1Fwd a) {
  __shared__ __align__(16) double sW[P1_NT * P1_NT];
  if constexpr (MODE != P1_NORM) {
    load_matrix<double>(sW, a.W, a.N);
    __syncthreads();
  }
  const int N = a.N, S = a.S;
  const int s = blockIdx.x * P1_TB + threadIdx.x;
  const bool valid = s < S;
  const Nb g = neighbours(a.st, valid ? s : 0);
  const Stencil& st = a.st;
  double acc[NT];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n] = 0.0;
  double nrm = 0.0, up = 0.0, kup = 0.0;
#pragma unroll
  for (int m = 0; m < NT; ++m) {
    const bool on = valid && m < N;
    double r;
    if constexpr (MODE == P1_DIRECT) {
      r = on ? __ldg(&a.b64[(size_t)m * S + s]) : 0.0;
    } else {
      const RowIn<double> x = load_row(a.b64, a.u64, g, s, (size_t)m * S, on);
      double ku = st.kc * x.c;
      ku = fma(st.kxl, x.l, ku);
      ku = fma(st.kxu, x.r, ku);
      ku = fma(st.kyl, x.d, ku);
      ku = fma(st.kyu, x.u, ku);
      double v = x.b - a.c1[m] * (x.c - up);
      v = fma(-a.theta, ku, v);
      v = fma(-(1.0 - a.theta), kup, v);
      r = on ? v : 0.0;
      up = x.c;
      kup = ku;
    }
    nrm = fma(r, r, nrm);
    if constexpr (MODE != P1_NORM) rank1_64<NT>(acc, sW, r, m);
  }
  const double wn = warp_sum(nrm);
  if ((threadIdx.x & 31) == 0 && a.norm2 != nullptr) atomicAdd(a.norm2, wn);
  if constexpr (MODE == P1_NORM) return;
  if (valid) {
    double2* out = reinterpret_cast<double2*>(a.out);
    const size_t o = spec_index(a.sg, 0, s);
#pragma unroll
    for (int n = 0; n < NT; ++n)
      if (n < N) out[o + (size_t)n * a.sg.specS] = make_double2(acc[n], 0.0);
  }
}

// ---------------------------------------------------------------------------
// Step (c), fused with the update: u = (V D~) S2 (P1_SET) or u += (V D~) S2
// (P1_ADD).  All spectrum loads are issued first, then the rank-one updates.
// Mixed: u is double-float, the transform FP32 (paired FMAs).
// ---------------------------------------------------------------------------
template <int MODE, int NT>
__global__ void __launch_bounds__(P1_TB) k_pd1_inv_mixed(const P1Inv a) {
  __shared__ __align__(16) float sV[P1_NT * P1_NT];
  load_matrix<float>(sV, a.V, a.N);
  __syncthreads();
  const int N = a.N, S = a.S;
  const int s = blockIdx.x * P1_TB + threadIdx.x;
  if (s >= S) return;
  const float2* in = reinterpret_cast<const float2*>(a.in);
  const size_t o = spec_index(a.sg, 0, s);
  float z[NT];
#pragma unroll
  for (int m = 0; m < NT; ++m) z[m] = m < N ? in[o + (size_t)m * a.sg.specS].x : 0.f;
  float2 acc[NT / 2];
#pragma unroll
  for (int j = 0; j < NT / 2; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll
  for (int m = 0; m < NT; ++m) rank1_pair<NT>(acc, sV, z[m], m);
  bool bad = false;
  float2 uo[NT];
  if constexpr (MODE == P1_ADD) {
#pragma unroll
    for (int n = 0; n < NT; ++n) uo[n] = n < N ? a.Udf[(size_t)n * S + s] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    if (n < N) {
      const float v = (n & 1) ? acc[n >> 1].y : acc[n >> 1].x;
      bad |= !isfinite(v);
      if constexpr (MODE == P1_SET) {
        a.Udf[(size_t)n * S + s] = make_float2(v, 0.f);
      } else {
        df t = two_sum(uo[n].x, v);
        t = fast_two_sum(t.hi, t.lo + uo[n].y);
        a.Udf[(size_t)n * S + s] = make_float2(t.hi, t.lo);
      }
    }
  }
  if (bad && a.flag != nullptr) atomicOr(a.flag, 1);
}

template <int MODE, int NT>
__global__ void __launch_bounds__(P1_TB) k_pd1_inv_64(const P1Inv a) {
  __shared__ __align__(16) double sV[P1_NT * P1_NT];
  load_matrix<double>(sV, a.V, a.N);
  __syncthreads();
  const int N = a.N, S = a.S;
  const int s = blockIdx.x * P1_TB + threadIdx.x;
  if (s >= S) return;
  const double2* in = reinterpret_cast<const double2*>(a.in);
  const size_t o = spec_index(a.sg, 0, s);
  double z[NT];
#pragma unroll
  for (int m = 0; m < NT; ++m) z[m] = m < N ? in[o + (size_t)m * a.sg.specS].x : 0.0;
  double acc[NT];
#pragma unroll
  for (int n = 0; n < NT; ++n) acc[n] = 0.0;
#pragma unroll
  for (int m = 0; m < NT; ++m) rank1_64<NT>(acc, sV, z[m], m);
  bool bad = false;
#pragma unroll
  for (int n = 0; n < NT; ++n) {
    if (n < N) {
      bad |= !isfinite(acc[n]);
      const size_t i = (size_t)n * S + s;
      if constexpr (MODE == P1_SET) a.u64[i] = acc[n];
      else a.u64[i] += acc[n];
    }
  }
  if (bad && a.flag != nullptr) atomicOr(a.flag, 1);
}

// ---------------------------------------------------------------------------
// Auxiliary FP64 kernels: y = A u and the right-hand side b.
// ---------------------------------------------------------------------------
__global__ void k_pd1_apply(const P1Fwd a, const double* u, double* y) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const Nb g = neighbours(a.st, s);
  double up = 0.0, kup = 0.0;
  for (int n = 0; n < a.N; ++n) {
    const double* U = u + (size_t)n * a.S;
    const double un = U[s];
    const double kun = ku_64(a.st, g, U, s);
    y[(size_t)n * a.S + s] = a.c1[n] * (un - up) + a.theta * kun + (1.0 - a.theta) * kup;
    up = un;
    kup = kun;
  }
}

// b_n = theta f(t_n) + (1 - theta) f(t_{n-1}), plus (I/dt_1 - (1-theta) K) u0
// in the first row; f ([N+1][S]) may be null
__global__ void k_pd1_rhs(const P1Fwd a, const double* u0, const double* f, double* b) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.S) return;
  const Nb g = neighbours(a.st, s);
  for (int n = 0; n < a.N; ++n) {
    double v = 0.0;
    if (f != nullptr)
      v = a.theta * f[(size_t)(n + 1) * a.S + s] + (1.0 - a.theta) * f[(size_t)n * a.S + s];
    if (n == 0) v += a.c1[0] * u0[s] - (1.0 - a.theta) * ku_64(a.st, g, u0, s);
    b[(size_t)n * a.S + s] = v;
  }
}

int grid_of(int S) { return (S + P1_TB - 1) / P1_TB; }

template <int NT>
void fwd_nt(const P1Fwd& a, int mode, bool fp64, dim3 grid, cudaStream_t st) {
  const dim3 block(P1_TB);
  if (fp64) {
    if (mode == P1_DIRECT) k_pd1_fwd_64<P1_DIRECT, NT><<<grid, block, 0, st>>>(a);
    else if (mode == P1_RESID) k_pd1_fwd_64<P1_RESID, NT><<<grid, block, 0, st>>>(a);
    else k_pd1_fwd_64<P1_NORM, NT><<<grid, block, 0, st>>>(a);
  } else {
    if (mode == P1_DIRECT) k_pd1_fwd_mixed<P1_DIRECT, NT><<<grid, block, 0, st>>>(a);
    else if (mode == P1_RESID) k_pd1_fwd_mixed<P1_RESID, NT><<<grid, block, 0, st>>>(a);
    else k_pd1_fwd_mixed<P1_NORM, NT><<<grid, block, 0, st>>>(a);
  }
}

template <int NT>
void inv_nt(const P1Inv& a, int mode, bool fp64, dim3 grid, cudaStream_t st) {
  const dim3 block(P1_TB);
  if (fp64) {
    if (mode == P1_SET) k_pd1_inv_64<P1_SET, NT><<<grid, block, 0, st>>>(a);
    else k_pd1_inv_64<P1_ADD, NT><<<grid, block, 0, st>>>(a);
  } else {
    if (mode == P1_SET) k_pd1_inv_mixed<P1_SET, NT><<<grid, block, 0, st>>>(a);
    else k_pd1_inv_mixed<P1_ADD, NT><<<grid, block, 0, st>>>(a);
  }
}

// register arrays sized for the window: 8, 16 or 32 rows
cudaError_t launch_pd1_fwd(const P1Fwd& a, int mode, bool fp64, cudaStream_t st) {
  const dim3 grid(grid_of(a.S));
  if (a.N <= 8) fwd_nt<8>(a, mode, fp64, grid, st);
  else if (a.N <= 16) fwd_nt<16>(a, mode, fp64, grid, st);
  else fwd_nt<32>(a, mode, fp64, grid, st);
  return cudaGetLastError();
}

cudaError_t launch_pd1_inv(const P1Inv& a, int mode, bool fp64, cudaStream_t st) {
  const dim3 grid(grid_of(a.S));
  if (a.N <= 8) inv_nt<8>(a, mode, fp64, grid, st);
  else if (a.N <= 16) inv_nt<16>(a, mode, fp64, grid, st);
  else inv_nt<32>(a, mode, fp64, grid, st);
  return cudaGetLastError();
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct pd1_plan {
  pd_plan* sp = nullptr;          // spatial operators, step (b) and its workspace
  int nt = 0, scheme = 0, scaled = 1, precision = 0;
  bool fp64 = false;
  double dt_last = 0, tau = 0, theta = 1;
  std::vector<double> dts;
  double cond_v = 0;              // Cond_2 estimate: ||V D~||_F ||(V D~)^{-1}||_F
  void* W = nullptr;              // step (a) matrix, transposed (float / double)
  void* V = nullptr;              // step (c) matrix, transposed
  double* dnorm = nullptr;        // device: [0] ||b||^2, [1] ||r||^2
  double* hnorm = nullptr;        // pinned host copy
  int* hflag = nullptr;
  unsigned long long launches = 0;
  int last_refinements = 0;
  char msg[256] = {0};
};

namespace {

pd_status p1_err(pd1_plan* q, pd_status s, const char* what) {
  if (q) snprintf(q->msg, sizeof(q->msg), "%s", what);
  return s;
}
pd_status p1_cuda(pd1_plan* q, cudaError_t e, const char* what) {
  if (q) snprintf(q->msg, sizeof(q->msg), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
}
#define P1CU(call)                                           \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return p1_cuda(q, e_, #call);     \
  } while (0)
#define P1LK(call)                                           \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    ++q->launches;                                           \
    if (e_ != cudaSuccess) return p1_cuda(q, e_, #call);     \
  } while (0)

void free_p1(pd1_plan* q) {
  if (!q) return;
  if (q->W) cudaFree(q->W);
  if (q->V) cudaFree(q->V);
  if (q->dnorm) cudaFree(q->dnorm);
  if (q->hnorm) cudaFreeHost(q->hnorm);
  if (q->sp) pd_plan_destroy(q->sp);
  delete q;
}

// the closed forms of Section 2.1.1 (p_0 = q_0 = 1)
void closed_forms(int nt, double tau, double theta, std::vector<double>& p, std::vector<double>& qv) {
  p.assign(nt, 1.0);
  qv.assign(nt, 1.0);
  for (int n = 1; n < nt; ++n) {
    if (theta == 1.0) {
      double den = 1.0;
      for (int j = 1; j <= n; ++j) den *= 1.0 - std::pow(tau, j);
      p[n] = 1.0 / den;
      qv[n] = ((n & 1) ? -1.0 : 1.0) * std::pow(tau, 0.5 * n * (n - 1)) * p[n];
    } else {
      double pn = 1.0, qn = std::pow(tau, -n);
      for (int j = 1; j <= n; ++j) {
        pn *= (1.0 + std::pow(tau, j)) / (1.0 - std::pow(tau, j));
        qn *= (1.0 + std::pow(tau, 2 - j)) / (1.0 - std::pow(tau, -j));
      }
      p[n] = pn;
      qv[n] = qn;
    }
  }
}

P1Fwd fwd_args(const pd1_plan* q) {
  P1Fwd a;
  memset(&a, 0, sizeof(a));
  const pd_plan* p = q->sp;
  a.N = q->nt;
  a.S = p->S;
  a.st = p->st;
  a.sg = p->sg;
  a.theta = q->theta;
  a.th_f = (float)q->theta;
  a.omth_f = (float)(1.0 - q->theta);
  for (int n = 0; n < q->nt; ++n) {
    a.c1[n] = 1.0 / q->dts[n];
    a.c1d[n] = dfc_from(a.c1[n]);
  }
  const double kap[5] = {p->st.kc, p->st.kxl, p->st.kxu, p->st.kyl, p->st.kyu};
  for (int i = 0; i < 5; ++i) a.kap[i] = dfc_from(kap[i]);
  a.Bdf = p->Bdf;
  a.Udf = p->Udf;
  a.W = q->W;
  a.out = p->spec;
  a.norm2 = q->dnorm;
  if (p->xform_tc) {
    a.amax = p->amax;
    a.amax_reset = p->amax + 1;
  }
  return a;
}

P1Inv inv_args(const pd1_plan* q) {
  P1Inv a;
  memset(&a, 0, sizeof(a));
  a.N = q->nt;
  a.S = q->sp->S;
  a.sg = q->sp->sg;
  a.V = q->V;
  a.in = q->sp->spec;
  a.Udf = q->sp->Udf;
  a.flag = q->sp->dflag;
  return a;
}

template <typename T>
pd_status upload_matrix(pd1_plan* q, void** dst, const std::vector<double>& M) {
  std::vector<T> h(M.size());
  for (size_t i = 0; i < M.size(); ++i) h[i] = (T)M[i];
  P1CU(cudaMalloc(dst, h.size() * sizeof(T)));
  P1CU(cudaMemcpy(*dst, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PD_OK;
}

pd_status step_b(pd1_plan* q) {
  const unsigned long long before = q->sp->launches;
  const pd_status s = plan_step_b(q->sp);
  q->launches += q->sp->launches - before;
  if (s != PD_OK) snprintf(q->msg, sizeof(q->msg), "%s", pd_last_error(q->sp));
  return s;
}

}  // namespace

extern "C" {

pd_status pd1_plan_create(const pd_space* sp, int nt, double dt_last, double tau, int scheme,
                          int column_scaling, int precision, void* stream, pd1_plan** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (!sp) return PD_ERR_ARG;
  if (nt < 1 || nt > P1_NT) return nt < 1 ? PD_ERR_ARG : PD_ERR_UNSUPPORTED;
  if (!(dt_last > 0.0) || !std::isfinite(dt_last)) return PD_ERR_ARG;
  if (!(tau > 1.0) || !std::isfinite(tau)) return PD_ERR_ARG;
  if (scheme != PD_BE && scheme != PD_CN) return PD_ERR_ARG;
  if (column_scaling != 0 && column_scaling != 1) return PD_ERR_ARG;
  if (precision != PD_FP64 && precision != PD_MIXED) return PD_ERR_ARG;

  pd1_plan* q = new (std::nothrow) pd1_plan();
  if (!q) return PD_ERR_NOMEM;
  q->nt = nt;
  q->scheme = scheme;
  q->scaled = column_scaling;
  q->precision = precision;
  q->fp64 = precision == PD_FP64;
  q->dt_last = dt_last;
  q->tau = tau;
  q->theta = scheme == PD_BE ? 1.0 : 0.5;
  const double th = q->theta;
  // eq. 2.8: dt_n = dt_Nt tau^(n - Nt), n = 1..Nt
  q->dts.resize(nt);
  for (int n = 1; n <= nt; ++n) q->dts[n - 1] = dt_last * std::pow(tau, (double)(n - nt));

  // step (b): lambda_1n = 1/(theta dt_n), lambda_2n = 1 (real)
  std::vector<double> lam((size_t)4 * nt, 0.0);
  for (int n = 0; n < nt; ++n) {
    lam[4 * n] = 1.0 / (th * q->dts[n]);
    lam[4 * n + 2] = 1.0;
  }
  pd_status s = plan_create_internal(sp, nt, q->dts[nt - 1], 1.0, scheme, th, precision, stream,
                                     true, &q->sp, lam.data());
  if (s != PD_OK) {
    delete q;
    return s;
  }

  // V (closed form), V^{-1} (closed form), D~, B2^{-1}; all in FP64
  std::vector<double> pc, qc;
  closed_forms(nt, tau, th, pc, qc);
  std::vector<double> dsc(nt, 1.0);
  if (column_scaling) {
    for (int n = 1; n <= nt; ++n) {
      double acc = 1.0;
      for (int j = 1; j <= nt - n; ++j) acc += pc[j] * pc[j];
      dsc[n - 1] = 1.0 / std::sqrt(acc);
    }
  }
  // (V D~)[n][m] = p_{n-m} dsc_m, ((V D~)^{-1})[n][m] = q_{n-m} / dsc_n,
  // (B2^{-1})[n][m] = (1/theta) (-(1-theta)/theta)^{n-m}
  std::vector<double> Wt((size_t)nt * nt, 0.0), Vt((size_t)nt * nt, 0.0);
  std::vector<double> b2i(nt);
  b2i[0] = 1.0 / th;
  for (int k = 1; k < nt; ++k) b2i[k] = b2i[k - 1] * (-(1.0 - th) / th);
  double fv = 0.0, fvi = 0.0;
  for (int n = 0; n < nt; ++n)
    for (int m = 0; m <= n; ++m) {
      // W[n][m] = sum_{k=m..n} Vi[n][k] B2inv[k][m]
      double w = 0.0;
      for (int k = m; k <= n; ++k) w += qc[n - k] / dsc[n] * b2i[k - m];
      Wt[(size_t)m * nt + n] = w;
      Vt[(size_t)m * nt + n] = pc[n - m] * dsc[m];
      fv += Vt[(size_t)m * nt + n] * Vt[(size_t)m * nt + n];
      const double vi = qc[n - m] / dsc[n];
      fvi += vi * vi;
    }
  q->cond_v = std::sqrt(fv * fvi);
  s = q->fp64 ? upload_matrix<double>(q, &q->W, Wt) : upload_matrix<float>(q, &q->W, Wt);
  if (s == PD_OK)
    s = q->fp64 ? upload_matrix<double>(q, &q->V, Vt) : upload_matrix<float>(q, &q->V, Vt);
  if (s == PD_OK) {
    cudaError_t e = cudaMalloc((void**)&q->dnorm, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&q->hnorm, 2 * sizeof(double) + sizeof(int));
    if (e != cudaSuccess) s = p1_cuda(q, e, "allocation");
  }
  if (s != PD_OK) {
    free_p1(q);
    return s;
  }
  q->hflag = reinterpret_cast<int*>(q->hnorm + 2);
  *out = q;
  return PD_OK;
}

pd_status pd1_plan_destroy(pd1_plan* q) {
  if (!q) return PD_ERR_ARG;
  if (q->sp && q->sp->stream) cudaStreamSynchronize(q->sp->stream);
  else cudaDeviceSynchronize();
  free_p1(q);
  return PD_OK;
}

pd_status pd1_step_sizes(const pd1_plan* q, double* dts) {
  if (!q || !dts) return PD_ERR_ARG;
  for (int n = 0; n < q->nt; ++n) dts[n] = q->dts[n];
  return PD_OK;
}

pd_status pd1_condition(const pd1_plan* q, double* cond) {
  if (!q || !cond) return PD_ERR_ARG;
  *cond = q->cond_v;
  return PD_OK;
}

pd_status pd1_apply_A(pd1_plan* q, const double* u, double* y) {
  if (!q || !u || !y) return PD_ERR_ARG;
  const P1Fwd a = fwd_args(q);
  k_pd1_apply<<<grid_of(a.S), P1_TB, 0, q->sp->stream>>>(a, u, y);
  P1LK(cudaGetLastError());
  return PD_OK;
}

pd_status pd1_build_rhs(pd1_plan* q, const double* u0, const double* f, double* b) {
  if (!q || !u0 || !b) return PD_ERR_ARG;
  const P1Fwd a = fwd_args(q);
  k_pd1_rhs<<<grid_of(a.S), P1_TB, 0, q->sp->stream>>>(a, u0, f, b);
  P1LK(cudaGetLastError());
  return PD_OK;
}

pd_status pd1_solve(pd1_plan* q, const double* b, double* u, double tol, int max_refine,
                    int* refinements, double* relres) {
  PdRange range("pd.pd1_solve");
  if (!q || !b || !u || max_refine < 0 || !(tol >= 0.0)) return PD_ERR_ARG;
  pd_plan* p = q->sp;
  cudaStream_t st = p->stream;
  const bool fp64 = q->fp64;
  const size_t ns = (size_t)q->nt * p->S;
  P1CU(cudaMemsetAsync(q->dnorm, 0, 2 * sizeof(double), st));
  P1CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), st));

  P1Fwd fa = fwd_args(q);
  fa.b64 = b;
  fa.u64 = u;
  fa.norm2 = q->dnorm;            // ||b||^2
  P1Inv ia = inv_args(q);
  ia.u64 = u;

  // the direct solve (eq. 2.7) from r = b
  P1LK(launch_pd1_fwd(fa, P1_DIRECT, fp64, st));
  {
    pd_status s = step_b(q);
    if (s != PD_OK) return s;
  }
  P1LK(launch_pd1_inv(ia, P1_SET, fp64, st));

  int done = 0;
  double rel = -1.0;
  const bool want_norm = max_refine > 0 || relres != nullptr;
  fa.norm2 = q->dnorm + 1;        // ||b - A u||^2
  for (int k = 0; want_norm; ++k) {
    const bool last = k == max_refine;
    P1CU(cudaMemsetAsync(q->dnorm + 1, 0, sizeof(double), st));
    P1LK(launch_pd1_fwd(fa, last ? P1_NORM : P1_RESID, fp64, st));
    P1CU(cudaMemcpyAsync(q->hnorm, q->dnorm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    P1CU(cudaMemcpyAsync(q->hflag, p->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    P1CU(cudaStreamSynchronize(st));
    const double nb = std::sqrt(q->hnorm[0]);
    rel = nb > 0.0 ? std::sqrt(q->hnorm[1]) / nb : std::sqrt(q->hnorm[1]);
    if (*q->hflag != 0 || !std::isfinite(rel)) {
      q->last_refinements = done;
      if (refinements) *refinements = done;
      if (relres) *relres = rel;
      return p1_err(q, PD_ERR_NONFINITE, "non-finite value in the ParaDiag-I solve");
    }
    if (last || rel <= tol) break;
    pd_status s = step_b(q);
    if (s != PD_OK) return s;
    P1LK(launch_pd1_inv(ia, P1_ADD, fp64, st));
    ++done;
  }
  if (!fp64) {
    P1LK(launch_from_df(p->Udf, u, ns, st));
  }
  P1CU(cudaStreamSynchronize(st));
  q->last_refinements = done;
  if (refinements) *refinements = done;
  if (relres) *relres = rel;
  if (max_refine > 0 && tol > 0.0 && !(rel <= tol)) {
    return p1_err(q, PD_ERR_NOT_CONVERGED, "refinement sweeps did not reach the tolerance");
  }
  return PD_OK;
}

pd_status pd1_solve_windows(pd1_plan* q, const double* u0, const double* f, int nwin, double* u,
                            double tol, int max_refine, int* refinements_total,
                            double* relres_max) {
  if (!q || !u0 || !u || nwin < 1 || max_refine < 0 || !(tol >= 0.0)) return PD_ERR_ARG;
  pd_plan* p = q->sp;
  const size_t S = (size_t)p->S;
  const size_t ns = (size_t)q->nt * S;
  if (!p->w64a) {
    cudaError_t e = cudaMalloc((void**)&p->w64a, ns * sizeof(double));
    if (e != cudaSuccess) {
      p->w64a = nullptr;
      return p1_cuda(q, e, "cudaMalloc");
    }
  }
  const P1Fwd a = fwd_args(q);
  int total = 0;
  double worst = 0.0;
  for (int w = 0; w < nwin; ++w) {
    double* uw = u + (size_t)w * ns;
    const double* start = w == 0 ? u0 : uw - S;      // last time level of the previous window
    const double* fw = f ? f + (size_t)w * q->nt * S : nullptr;
    k_pd1_rhs<<<grid_of(a.S), P1_TB, 0, p->stream>>>(a, start, fw, p->w64a);
    P1LK(cudaGetLastError());
    int it = 0;
    double rel = 0.0;
    const pd_status st = pd1_solve(q, p->w64a, uw, tol, max_refine, &it, &rel);
    total += it;
    worst = std::max(worst, rel);
    if (st != PD_OK) {
      if (refinements_total) *refinements_total = total;
      if (relres_max) *relres_max = worst;
      return st;
    }
  }
  if (refinements_total) *refinements_total = total;
  if (relres_max) *relres_max = worst;
  return PD_OK;
}

pd_status pd1_profile_sweep(pd1_plan* q, const double* b, double* u, int reps, float* ms) {
  if (!q || !b || !u || !ms || reps < 1) return PD_ERR_ARG;
  pd_plan* p = q->sp;
  cudaStream_t st = p->stream;
  const bool fp64 = q->fp64;
  P1Fwd fa = fwd_args(q);
  fa.b64 = b;
  fa.u64 = u;
  fa.norm2 = q->dnorm;
  P1Inv ia = inv_args(q);
  ia.u64 = u;
  // a state to sweep from: the direct solve
  P1LK(launch_pd1_fwd(fa, P1_DIRECT, fp64, st));
  {
    const pd_status s = step_b(q);
    if (s != PD_OK) return s;
  }
  P1LK(launch_pd1_inv(ia, P1_SET, fp64, st));
  fa.norm2 = q->dnorm + 1;
  cudaEvent_t ev[4];
  for (int i = 0; i < 4; ++i) P1CU(cudaEventCreate(&ev[i]));
  double acc[3] = {0, 0, 0};
  for (int r = 0; r < reps; ++r) {
    P1CU(cudaEventRecord(ev[0], st));
    P1LK(launch_pd1_fwd(fa, P1_RESID, fp64, st));
    P1CU(cudaEventRecord(ev[1], st));
    const pd_status s = step_b(q);
    if (s != PD_OK) return s;
    P1CU(cudaEventRecord(ev[2], st));
    P1LK(launch_pd1_inv(ia, P1_ADD, fp64, st));
    P1CU(cudaEventRecord(ev[3], st));
    P1CU(cudaEventSynchronize(ev[3]));
    for (int i = 0; i < 3; ++i) {
      float t = 0.f;
      P1CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      acc[i] += t;
    }
  }
  for (int i = 0; i < 4; ++i) cudaEventDestroy(ev[i]);
  for (int i = 0; i < 3; ++i) ms[i] = (float)(acc[i] / reps);
  if (!fp64) {
    P1LK(launch_from_df(p->Udf, u, (size_t)q->nt * p->S, st));
  }
  P1CU(cudaStreamSynchronize(st));
  return PD_OK;
}

pd_status pd1_launches(const pd1_plan* q, unsigned long long* count) {
  if (!q || !count) return PD_ERR_ARG;
  *count = q->launches;
  return PD_OK;
}

pd_status pd1_workspace(const pd1_plan* q, unsigned long long* bytes) {
  if (!q || !bytes) return PD_ERR_ARG;
  const size_t m = (size_t)q->nt * q->nt * (q->fp64 ? sizeof(double) : sizeof(float));
  *bytes = q->sp->bytes + 2 * m + 2 * sizeof(double);
  return PD_OK;
}

const char* pd1_last_error(const pd1_plan* q) { return q ? q->msg : "null plan"; }

}  // extern "C"
