// Auxiliary kernels: the FP64 all-at-once operator A (and A^T) of eq. 1.1,
// the right-hand side b of the theta-method / leap-frog systems, conversions
// between FP64 and double-float storage, reductions and the vector updates
// of flexible GMRES.
#include "pd_internal.h"

namespace {

constexpr int TB = 256;

__device__ __forceinline__ double stencil64(const Stencil& st, const double* U, int s, int tr) {
  // (K U)(s) or (K^T U)(s) for one time row U
  const int xg = s % st.nx, y = s / st.nx;
  double kxl = tr ? st.kxu : st.kxl, kxu = tr ? st.kxl : st.kxu;
  double kyl = tr ? st.kyu : st.kyl, kyu = tr ? st.kyl : st.kyu;
  double v = st.kc * U[s];
  if (xg > 0) v = fma(kxl, U[s - 1], v);
  else if (st.bcx == PD_PERIODIC && st.nx > 1) v = fma(kxl, U[s + st.nx - 1], v);
  if (xg < st.nx - 1) v = fma(kxu, U[s + 1], v);
  else if (st.bcx == PD_PERIODIC && st.nx > 1) v = fma(kxu, U[s - st.nx + 1], v);
  if (st.dim == 2) {
    if (y > 0) v = fma(kyl, U[s - st.nx], v);
    if (y < st.ny - 1) v = fma(kyu, U[s + st.nx], v);
  }
  return v;
}

// y = A u (transpose = 0) or A^T u (transpose = 1); with b: y = b - A u and
// norm2 += ||y||^2.
__global__ void k_apply_A(Stencil st, TimeBand tb, int N, const double* __restrict__ u,
                          const double* __restrict__ b, double* __restrict__ y, double* norm2,
                          int transpose) {
  __shared__ double red[TB / 32];
  const size_t total = (size_t)N * st.S;
  double part = 0.0;
  for (size_t e = blockIdx.x * (size_t)TB + threadIdx.x; e < total; e += (size_t)gridDim.x * TB) {
    const int n = (int)(e / st.S), s = (int)(e % st.S);
    double v = 0.0;
    for (int m = 0; m <= tb.band; ++m) {
      const int nn = transpose ? n + m : n - m;
      if (nn < 0 || nn >= N) continue;
      const double* U = u + (size_t)nn * st.S;
      if (tb.c1[m] != 0.0) v = fma(tb.c1[m], U[s], v);
      if (tb.c2[m] != 0.0) v = fma(tb.c2[m], stencil64(st, U, s, transpose), v);
    }
    if (b != nullptr) v = b[e] - v;
    y[e] = v;
    part = fma(v, v, part);
  }
  if (norm2 != nullptr) {
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0;
      for (int w = 0; w < TB / 32; ++w) s += red[w];
      atomicAdd(norm2, s);
    }
  }
}

// right-hand side b (theta-method: eq. 2.4 rows; leap-frog: eq. 3.2b rows
// with the ghost value U_{-1} = U_1 - 2 dt u_1 in the first step)
__global__ void k_build_rhs(Stencil st, int leap, double theta, int N, double dt,
                            const double* __restrict__ u0, const double* __restrict__ u1,
                            const double* __restrict__ f, double* __restrict__ b) {
  const size_t total = (size_t)N * st.S;
  for (size_t e = blockIdx.x * (size_t)TB + threadIdx.x; e < total; e += (size_t)gridDim.x * TB) {
    const int n = (int)(e / st.S), s = (int)(e % st.S);
    const size_t S = st.S;
    double v = 0.0;
    if (!leap) {
      if (f != nullptr) v = theta * f[(size_t)(n + 1) * S + s] + (1.0 - theta) * f[(size_t)n * S + s];
      if (n == 0) v += u0[s] / dt - (1.0 - theta) * stencil64(st, u0, s, 0);
    } else {
      if (f != nullptr) v = (n == 0) ? 0.5 * f[s] : f[(size_t)n * S + s];
      if (n == 0) {
        v += u0[s] / (dt * dt);
        if (u1 != nullptr) v += u1[s] / dt + 0.5 * dt * stencil64(st, u1, s, 0);
      } else if (n == 1) {
        v += -u0[s] / (dt * dt) - 0.5 * stencil64(st, u0, s, 0);
      }
    }
    b[e] = v;
  }
}

__global__ void k_to_df(const double* __restrict__ x, dfc scale, float2* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    df v = df_from_double(x[i]);
    v = df_mul(v, df_make(scale.hi, scale.lo));
    y[i] = make_float2(v.hi, v.lo);
  }
}

// Entry of the mixed stationary solve in one pass: U = split(u), B = split(s b)
// and ||s b||^2 accumulated from the FP32 high parts (FP64 arithmetic is slow
// on this GPU; a few significant digits suffice for the relative residual).
__global__ void k_entry_df(const double* __restrict__ u, const double* __restrict__ b, dfc scale,
                           float2* __restrict__ U, float2* __restrict__ B, size_t n,
                           double* norm2, int* nonzero) {
  __shared__ double red[TB / 32];
  float part = 0.f;
  bool nz = false;
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    const double ui = u[i], bi = b[i];
    nz |= ui != 0.0;
    const df uv = df_from_double(ui);
    const df bv = df_mul(df_from_double(bi), df_make(scale.hi, scale.lo));
    U[i] = make_float2(uv.hi, uv.lo);
    B[i] = make_float2(bv.hi, bv.lo);
    part = fmaf(bv.hi, bv.hi, part);
  }
  if (nonzero != nullptr && __any_sync(0xffffffffu, nz) && (threadIdx.x & 31) == 0)
    atomicOr(nonzero, 1);
  double pd = (double)part;
  for (int o = 16; o > 0; o >>= 1) pd += __shfl_down_sync(0xffffffffu, pd, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pd;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < TB / 32; ++w) s += red[w];
    atomicAdd(norm2, s);
  }
}

__global__ void k_from_df(const float2* __restrict__ x, double* __restrict__ y, size_t n) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    const float2 v = x[i];
    y[i] = double_from_float(v.x) + double_from_float(v.y);
  }
}

__global__ void k_norm2(const double* __restrict__ x, size_t n, double* out) {
  __shared__ double red[TB / 32];
  double part = 0.0;
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB)
    part = fma(x[i], x[i], part);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int w = 0; w < TB / 32; ++w) s += red[w];
    atomicAdd(out, s);
  }
}

__global__ void k_flip_time(const double* __restrict__ x, double* __restrict__ y, int N, int S) {
  const size_t total = (size_t)N * S;
  for (size_t e = blockIdx.x * (size_t)TB + threadIdx.x; e < total; e += (size_t)gridDim.x * TB) {
    const int n = (int)(e / S), s = (int)(e % S);
    y[e] = x[(size_t)(N - 1 - n) * S + s];
  }
}

// h[i] += <V_i, w> for i = blockIdx.y
__global__ void k_dots(const double* __restrict__ V, size_t n, const double* __restrict__ w,
                       double* h) {
  __shared__ double red[TB / 32];
  const double* v = V + (size_t)blockIdx.y * n;
  double part = 0.0;
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB)
    part = fma(v[i], w[i], part);
  for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int q = 0; q < TB / 32; ++q) s += red[q];
    atomicAdd(&h[blockIdx.y], s);
  }
}

__global__ void k_gemv_sub(const double* __restrict__ V, int nv, size_t n,
                           const double* __restrict__ h, double* __restrict__ w) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    double v = w[i];
    for (int q = 0; q < nv; ++q) v = fma(-h[q], V[(size_t)q * n + i], v);
    w[i] = v;
  }
}

__global__ void k_axpby(double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        size_t n) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB)
    y[i] = fma(a, x[i], b * y[i]);
}

__global__ void k_scale_copy(double a, const double* __restrict__ x, double* __restrict__ y,
                             size_t n) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB)
    y[i] = a * x[i];
}

__global__ void k_combine(const double* __restrict__ Z, int nz, size_t n,
                          const double* __restrict__ yv, double* __restrict__ u) {
  for (size_t i = blockIdx.x * (size_t)TB + threadIdx.x; i < n; i += (size_t)gridDim.x * TB) {
    double v = u[i];
    for (int q = 0; q < nz; ++q) v = fma(yv[q], Z[(size_t)q * n + i], v);
    u[i] = v;
  }
}

inline int grid_for(size_t n) {
  size_t g = (n + TB - 1) / TB;
  if (g > 152 * 16) g = 152 * 16;
  return g == 0 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_apply_A(const Stencil& st, const TimeBand& tb, int N, const double* u,
                           const double* b, double* y, double* norm2, int transpose,
                           cudaStream_t s) {
  k_apply_A<<<grid_for((size_t)N * st.S), TB, 0, s>>>(st, tb, N, u, b, y, norm2, transpose);
  return cudaGetLastError();
}

cudaError_t launch_build_rhs(const Stencil& st, const TimeBand& tb, int scheme, int N, double dt,
                             const double* u0, const double* u1, const double* f, double* b,
                             cudaStream_t s) {
  const int leap = tb.band == 2;
  const double theta = leap ? 0.0 : tb.c2[0];
  (void)scheme;
  k_build_rhs<<<grid_for((size_t)N * st.S), TB, 0, s>>>(st, leap, theta, N, dt, u0, u1, f, b);
  return cudaGetLastError();
}

cudaError_t launch_to_df(const double* x, double scale, float2* y, size_t n, cudaStream_t s) {
  k_to_df<<<grid_for(n), TB, 0, s>>>(x, dfc_from(scale), y, n);
  return cudaGetLastError();
}

cudaError_t launch_entry_df(const double* u, const double* b, double scale, float2* U, float2* B,
                            size_t n, double* norm2, cudaStream_t s, int* nonzero) {
  k_entry_df<<<grid_for(n), TB, 0, s>>>(u, b, dfc_from(scale), U, B, n, norm2, nonzero);
  return cudaGetLastError();
}

cudaError_t launch_from_df(const float2* x, double* y, size_t n, cudaStream_t s) {
  k_from_df<<<grid_for(n), TB, 0, s>>>(x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_norm2(const double* x, size_t n, double* out, cudaStream_t s) {
  k_norm2<<<grid_for(n), TB, 0, s>>>(x, n, out);
  return cudaGetLastError();
}

cudaError_t launch_flip_time(const double* x, double* y, int N, int S, cudaStream_t s) {
  k_flip_time<<<grid_for((size_t)N * S), TB, 0, s>>>(x, y, N, S);
  return cudaGetLastError();
}

cudaError_t launch_dots(const double* V, int nv, size_t n, const double* w, double* h,
                        cudaStream_t s) {
  int gx = grid_for(n) / 4;
  if (gx < 1) gx = 1;
  dim3 grid(gx, nv);
  k_dots<<<grid, TB, 0, s>>>(V, n, w, h);
  return cudaGetLastError();
}

cudaError_t launch_gemv_sub(const double* V, int nv, size_t n, const double* h, double* w,
                            cudaStream_t s) {
  k_gemv_sub<<<grid_for(n), TB, 0, s>>>(V, nv, n, h, w);
  return cudaGetLastError();
}

cudaError_t launch_axpby(double a, const double* x, double b, double* y, size_t n,
                         cudaStream_t s) {
  k_axpby<<<grid_for(n), TB, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_copy(double a, const double* x, double* y, size_t n, cudaStream_t s) {
  k_scale_copy<<<grid_for(n), TB, 0, s>>>(a, x, y, n);
  return cudaGetLastError();
}

cudaError_t launch_combine(const double* Z, int nz, size_t n, const double* y, double* u,
                           cudaStream_t s) {
  k_combine<<<grid_for(n), TB, 0, s>>>(Z, nz, n, y, u);
  return cudaGetLastError();
}
