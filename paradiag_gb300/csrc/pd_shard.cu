// The preconditioner in parts, for a solve spread over several GPUs.
//
// The steps of eq. 1.3 are independent across space (steps (a) and (c), the
// FFTs along time) and across the time frequency k (step (b), the shifted
// solves), so a distributed solve owns slabs of grid lines (y in 2D, x for a
// 1D Dirichlet problem) for the time steps and the residual, and slabs of
// frequencies for step (b), with an all-to-all transpose of the spectrum in
// between.  These entry points run the per-rank parts on one plan; the
// exchange itself is the caller's (torch.distributed in the Python binding).
//   pd_precond_forward    step (a): Gamma scaling and FFT along t of r, then
//                         (2D / periodic x) the forward x-eigentransform; the
//                         result is the plan's step-(b) spectrum
//   pd_precond_solve_rows step (b) for the frequencies k0 .. k1-1 on a
//                         caller-owned slab of that spectrum
//   pd_precond_backward   step (c): (2D) inverse x-transform, inverse FFT,
//                         Gamma^{-1}: z from the plan's step-(b) spectrum
//   pd_shard_norm2 / pd_shard_update: the residual norm and the update u += z
//                         restricted to the grid lines a rank owns
#include <cstring>

#include "pd_plan.h"

namespace {

#define SCU(call)                                                      \
  do {                                                                 \
    cudaError_t e_ = (call);                                           \
    if (e_ != cudaSuccess) return plan_fail_cuda(p, e_, #call);        \
  } while (0)

constexpr int NB = 256;

// max |x| over rows x cols floats with row stride ld (the padding of a row is
// skipped: it holds no value of the spectrum) into *out as float bits (the
// values are non-negative, so the unsigned order is the float order)
__global__ void k_amax(const float* __restrict__ x, size_t rows, int cols, int ld, unsigned* out) {
  float m = 0.f;
  const size_t n = rows * (size_t)cols;
  for (size_t i = blockIdx.x * (size_t)NB + threadIdx.x; i < n; i += (size_t)gridDim.x * NB)
    m = fmaxf(m, fabsf(x[(i / cols) * ld + i % cols]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));
}

// sum over time levels n and the points [s0, s0 + cnt) of line-major rows of
// S points: x[n S + s]^2 into *out
__global__ void k_norm2_lines(const double* __restrict__ x, int N, long long S, long long s0,
                              long long cnt, double* out) {
  __shared__ double red[NB / 32];
  double acc = 0.0;
  const long long tot = (long long)N * cnt;
  for (long long i = blockIdx.x * (long long)NB + threadIdx.x; i < tot; i += (long long)gridDim.x * NB) {
    const long long n = i / cnt, s = i - n * cnt;
    const double v = x[n * S + s0 + s];
    acc = fma(v, v, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < NB / 32; ++w) t += red[w];
    atomicAdd(out, t);
  }
}

// u[n S + s] += z[n S + s] for s in [s0, s0 + cnt)
__global__ void k_update_lines(const double* __restrict__ z, double* __restrict__ u, int N,
                               long long S, long long s0, long long cnt) {
  const long long tot = (long long)N * cnt;
  for (long long i = blockIdx.x * (long long)NB + threadIdx.x; i < tot; i += (long long)gridDim.x * NB) {
    const long long n = i / cnt, s = i - n * cnt;
    u[n * S + s0 + s] += z[n * S + s0 + s];
  }
}

int grid_of(long long n) {
  long long g = (n + NB - 1) / NB;
  if (g > 152LL * 8) g = 152LL * 8;
  return g < 1 ? 1 : (int)g;
}

// points per grid line of the slab direction, and the number of lines
void line_geometry(const pd_plan* p, long long* pts, int* lines) {
  if (p->sp.dim == 2) {
    *pts = p->sp.nx;
    *lines = p->sp.ny;
  } else {
    *pts = 1;
    *lines = p->sp.nx;
  }
}

}  // namespace

extern "C" {

pd_status pd_precond_forward(pd_plan* p, const double* r) {
  if (!p || !r) return PD_ERR_ARG;
  PdRange range("pd.shard.forward");
  FwdArgs fa = plan_fwd_args(p);
  fa.mode = FWD_STANDALONE;
  fa.r64 = r;
  fa.amax_reset = nullptr;        // the inverse transform's word is set by pd_precond_backward
  ++p->launches;
  SCU(launch_time_fwd(fa, p->fp64, p->stream));
  if (p->xform) return plan_xform(p, true);
  return PD_OK;
}

pd_status pd_plan_spectrum(pd_plan* p, void** data, int* nh, int* lines, int* pitch,
                           int* elem_bytes) {
  if (!p || !data || !nh || !lines || !pitch || !elem_bytes) return PD_ERR_ARG;
  if (p->sp.dim == 1 && p->sp.bc_x == PD_PERIODIC) return PD_ERR_UNSUPPORTED;
  *data = p->xform ? p->spec2 : p->spec;
  *nh = p->nh;
  if (p->sp.dim == 2) {
    *lines = p->sp.ny;
    *pitch = p->sg.nxp;
  } else {
    *lines = p->sp.nx;
    *pitch = 1;
  }
  *elem_bytes = p->fp64 ? (int)sizeof(double2) : (int)sizeof(float2);
  return PD_OK;
}

// [k0, k1) x [l0, l1) block of the step-(b) spectrum <-> a contiguous
// caller buffer [k1-k0][l1-l0][pitch] (one 2D copy: k rows of (l1-l0) lines)
pd_status spectrum_block(pd_plan* p, int k0, int k1, int l0, int l1, void* buf, bool get) {
  void* data;
  int nh, lines, pitch, eb;
  pd_status s = pd_plan_spectrum(p, &data, &nh, &lines, &pitch, &eb);
  if (s != PD_OK) return s;
  if (k0 < 0 || k1 > nh || k0 > k1 || l0 < 0 || l1 > lines || l0 > l1) return PD_ERR_ARG;
  if (k0 == k1 || l0 == l1) return PD_OK;
  const size_t row = (size_t)lines * pitch * eb;               // one frequency of the spectrum
  const size_t chunk = (size_t)(l1 - l0) * pitch * eb;         // the block's part of it
  char* sp = static_cast<char*>(data) + (size_t)k0 * row + (size_t)l0 * pitch * eb;
  if (get) {
    SCU(cudaMemcpy2DAsync(buf, chunk, sp, row, chunk, (size_t)(k1 - k0), cudaMemcpyDeviceToDevice,
                          p->stream));
  } else if (buf != nullptr) {
    SCU(cudaMemcpy2DAsync(sp, row, buf, chunk, chunk, (size_t)(k1 - k0), cudaMemcpyDeviceToDevice,
                          p->stream));
  } else {
    SCU(cudaMemset2DAsync(sp, row, 0, chunk, (size_t)(k1 - k0), p->stream));
  }
  return PD_OK;
}

pd_status pd_spectrum_get(pd_plan* p, int k0, int k1, int l0, int l1, void* dst) {
  if (!p || !dst) return PD_ERR_ARG;
  return spectrum_block(p, k0, k1, l0, l1, dst, true);
}

pd_status pd_spectrum_put(pd_plan* p, int k0, int k1, int l0, int l1, const void* src) {
  if (!p) return PD_ERR_ARG;
  return spectrum_block(p, k0, k1, l0, l1, const_cast<void*>(src), false);
}

pd_status pd_precond_solve_rows(pd_plan* p, int k0, int k1, void* data) {
  if (!p || !data) return PD_ERR_ARG;
  if (k0 < 0 || k1 > p->nh || k0 > k1) return PD_ERR_ARG;
  if (p->sp.dim == 1 && p->sp.bc_x == PD_PERIODIC) return PD_ERR_UNSUPPORTED;
  if (k0 == k1) return PD_OK;
  PdRange range("pd.shard.solve_rows");
  TriArgs ta = plan_tri_args(p, data);
  ta.nh = k1 - k0;
  ta.lam = static_cast<const char*>(p->lam) + (size_t)2 * k0 * (p->fp64 ? sizeof(double2) : sizeof(float2));
  ta.amax = nullptr;              // the slab's maximum is taken by the rank that transforms it
  ta.amax_reset = nullptr;
  ++p->launches;
  SCU(launch_tridiag(ta, p->fp64, p->stream));
  return PD_OK;
}

pd_status pd_precond_backward(pd_plan* p, double* z) {
  if (!p || !z) return PD_ERR_ARG;
  PdRange range("pd.shard.backward");
  if (p->xform) {
    if (p->xform_tc) {
      // the inverse tensor-core transform scales by max |input|: take it from
      // the spectrum the exchange brought back; the forward word is zeroed
      // for the next forward pass
      SCU(cudaMemsetAsync(p->amax, 0, 2 * sizeof(unsigned), p->stream));
      const size_t rows = (size_t)p->nh * (p->sg.specS / p->sg.nxp);
      ++p->launches;
      k_amax<<<grid_of((long long)(rows * 2 * p->sp.nx)), NB, 0, p->stream>>>(
          static_cast<const float*>(p->spec2), rows, 2 * p->sp.nx, 2 * p->sg.nxp, p->amax + 1);
      SCU(cudaGetLastError());
    }
    const pd_status s = plan_xform(p, false);
    if (s != PD_OK) return s;
  }
  InvArgs ia = plan_inv_args(p);
  ia.mode = INV_OUT64;
  ia.out64 = z;
  ++p->launches;
  SCU(launch_time_inv(ia, p->fp64, p->stream));
  return PD_OK;
}

pd_status pd_shard_norm2(pd_plan* p, const double* x, int first_line, int nlines, double* out) {
  if (!p || !x || !out) return PD_ERR_ARG;
  long long pts;
  int lines;
  line_geometry(p, &pts, &lines);
  if (first_line < 0 || nlines < 0 || first_line + nlines > lines) return PD_ERR_ARG;
  double* d = p->dsc + 90;        // a scalar slot no solver uses
  SCU(cudaMemsetAsync(d, 0, sizeof(double), p->stream));
  const long long cnt = (long long)nlines * pts;
  if (cnt > 0) {
    ++p->launches;
    k_norm2_lines<<<grid_of((long long)p->nt * cnt), NB, 0, p->stream>>>(
        x, p->nt, p->S, (long long)first_line * pts, cnt, d);
    SCU(cudaGetLastError());
  }
  SCU(cudaMemcpyAsync(out, d, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  SCU(cudaStreamSynchronize(p->stream));
  return PD_OK;
}

pd_status pd_shard_update(pd_plan* p, const double* z, double* u, int first_line, int nlines) {
  if (!p || !z || !u) return PD_ERR_ARG;
  long long pts;
  int lines;
  line_geometry(p, &pts, &lines);
  if (first_line < 0 || nlines < 0 || first_line + nlines > lines) return PD_ERR_ARG;
  const long long cnt = (long long)nlines * pts;
  if (cnt == 0) return PD_OK;
  ++p->launches;
  k_update_lines<<<grid_of((long long)p->nt * cnt), NB, 0, p->stream>>>(
      z, u, p->nt, p->S, (long long)first_line * pts, cnt);
  SCU(cudaGetLastError());
  return PD_OK;
}

}  // extern "C"
