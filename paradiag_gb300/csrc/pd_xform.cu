// x-eigentransform of 2D problems (and of periodic 1D problems): every row of
// the half spectrum (one row per time frequency k and grid line y) is
// multiplied by the nx-by-nx eigenvector matrix of K_x, which diagonalises the
// x part of the shifted operator lambda_1 I + lambda_2 K so that step (b) of
// eq. 1.3 reduces to tridiagonal solves in y.  This file holds the SIMT
// (CUDA-core) complex GEMM used by the FP64 path:
//   out[r][j] = sum_x Q[j][x] in[r][x].
#include "pd_internal.h"

namespace {

constexpr int BR = 32, BJ = 64, BK = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_xform_simt(XformArgs a) {
  using C = cplx_t<R>;
  __shared__ C sx[BR][BK + 1];
  __shared__ C sq[BJ][BK + 1];
  const C* X = reinterpret_cast<const C*>(a.in);
  const C* Q = reinterpret_cast<const C*>(a.Q);
  C* Y = reinterpret_cast<C*>(a.out);
  const int r0 = blockIdx.x * BR, j0 = blockIdx.y * BJ;
  const int tr = threadIdx.x / 16, tj = threadIdx.x % 16;
  C acc[2][4];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = czero<C>();
  for (int k0 = 0; k0 < a.nx; k0 += BK) {
    for (int e = threadIdx.x; e < BR * BK; e += 256) {
      const int rr = e / BK, kk = e % BK;
      const int r = r0 + rr, k = k0 + kk;
      sx[rr][kk] = (r < a.rows && k < a.nx) ? X[(size_t)r * a.ld + k] : czero<C>();
    }
    for (int e = threadIdx.x; e < BJ * BK; e += 256) {
      const int jj = e / BK, kk = e % BK;
      const int j = j0 + jj, k = k0 + kk;
      sq[jj][kk] = (j < a.nx && k < a.nx) ? Q[(size_t)j * a.nx + k] : czero<C>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      C xv[2], qv[4];
#pragma unroll
      for (int u = 0; u < 2; ++u) xv[u] = sx[tr + 16 * u][kk];
#pragma unroll
      for (int v = 0; v < 4; ++v) qv[v] = sq[tj + 16 * v][kk];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          acc[u][v].x = fma(qv[v].x, xv[u].x, acc[u][v].x);
          acc[u][v].x = fma(-qv[v].y, xv[u].y, acc[u][v].x);
          acc[u][v].y = fma(qv[v].x, xv[u].y, acc[u][v].y);
          acc[u][v].y = fma(qv[v].y, xv[u].x, acc[u][v].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int r = r0 + tr + 16 * u, j = j0 + tj + 16 * v;
      if (r < a.rows && j < a.nx) Y[(size_t)r * a.ld + j] = acc[u][v];
    }
}

}  // namespace

cudaError_t launch_xform(const XformArgs& a, bool fp64, cudaStream_t st) {
  dim3 grid(ceil_div(a.rows, BR), ceil_div(a.nx, BJ));
  if (a.rows == 0) return cudaSuccess;
  if (fp64) k_xform_simt<double><<<grid, 256, 0, st>>>(a);
  else k_xform_simt<float><<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}
