// Plans, solvers and the C ABI of the ParaDiag-II library (include/paradiag.h).
//
// Plan creation evaluates, on the host in FP64, everything that depends only
// on the problem: the first columns c1, c2 of the Toeplitz B1, B2 (eq. 2.5b,
// eq. 3.2b), the eigenvalues of the alpha-circulants C1, C2 (Lemma 1)
//   lambda_{j,k} = sum_m c_j[m] w_k^m,  w_k = alpha^{1/Nt} exp(-2 pi i k/Nt),
// which equal the diagonal of D_j for the forward transform with
// exp(-2 pi i k n/Nt) used by the kernels, the Gamma_alpha tables
// (gamma_n = alpha^{n/Nt}, n = 0..Nt-1), the FFT twiddles and, for 2D, the
// eigenvectors and eigenvalues of K_x.  Only k = 0..Nt/2 is kept: real data
// give a Hermitian spectrum, so the shifted solve at Nt-k is the conjugate of
// the one at k.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <functional>
#include <new>
#include <vector>

#include "pd_internal.h"

using cd = std::complex<double>;

#include "pd_plan.h"

// solver graph state (see solve_stationary_graph)
struct LoopState {
  double tol, s_scale, prev_rel, rel;
  int maxit, it, status, norm_only, n_body, n_update;
  int kmode;       // mode of the next forward kernel (read by it from device memory)
  int imode;       // mode of the next inverse kernel (likewise)
  int zero_guess;  // the solve started from u = 0
};
struct SolveGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cs = nullptr;
  LoopState* dst = nullptr;   // device loop state
  LoopState* res = nullptr;   // pinned copy of the final state of the last solve
  int pending = 0;            // solves enqueued since the last finish
  int update_kernels = 0;     // kernels in one update (IF body)
};

void destroy_graph(SolveGraph* G) {
  if (!G) return;
  if (G->ge) cudaGraphExecDestroy(G->ge);
  if (G->g) cudaGraphDestroy(G->g);
  if (G->cs) cudaStreamDestroy(G->cs);
  if (G->dst) cudaFree(G->dst);
  if (G->res) cudaFreeHost(G->res);
  delete G;
}


namespace {

constexpr int NSC = 96;  // device / host scalar slots

pd_status set_err(pd_plan* p, pd_status s, const char* what) {
  if (p) snprintf(p->msg, sizeof(p->msg), "%s", what);
  return s;
}

pd_status fail_cuda(pd_plan* p, cudaError_t e, const char* what) {
  if (p) snprintf(p->msg, sizeof(p->msg), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
}

#define CU(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return fail_cuda(p, e_, #call); \
  } while (0)

// a kernel launch through one of the launch_* wrappers (counted per plan)
#define LK(call)                                           \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    ++p->launches;                                         \
    if (e_ != cudaSuccess) return fail_cuda(p, e_, #call); \
  } while (0)

#define CHK(call)                      \
  do {                                 \
    pd_status s_ = (call);             \
    if (s_ != PD_OK) return s_;        \
  } while (0)

pd_status dalloc(pd_plan* p, void** ptr, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    return fail_cuda(p, e, "cudaMalloc");
  }
  p->bytes += bytes;
  return PD_OK;
}

template <typename T>
pd_status upload(pd_plan* p, void** dst, const std::vector<T>& v) {
  CHK(dalloc(p, dst, v.size() * sizeof(T)));
  CU(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PD_OK;
}

// upload complex values as float2 or double2
pd_status upload_cplx(pd_plan* p, void** dst, const std::vector<cd>& v, bool fp64) {
  if (fp64) {
    std::vector<double2> h(v.size());
    for (size_t i = 0; i < v.size(); ++i) h[i] = make_double2(v[i].real(), v[i].imag());
    return upload(p, dst, h);
  }
  std::vector<float2> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = make_float2((float)v[i].real(), (float)v[i].imag());
  return upload(p, dst, h);
}

pd_status upload_real(pd_plan* p, void** dst, const std::vector<double>& v, bool fp64) {
  if (fp64) return upload(p, dst, v);
  std::vector<float> h(v.size());
  for (size_t i = 0; i < v.size(); ++i) h[i] = (float)v[i];
  return upload(p, dst, h);
}

void free_plan(pd_plan* p) {
  if (!p) return;
  void* ptrs[] = {p->lam,  p->gam,  p->igam, p->igam_s, p->tw,    p->Qf,    p->Qi,
                  p->mu,   p->spec, p->spec2, p->Udf,  p->Bdf,   p->w64a,  p->w64b,
                  p->dsc,  p->dflag, p->V,   p->Z,      p->dh,    p->Gf_hi, p->Gf_lo,
                  p->Gi_hi, p->Gi_lo, const_cast<void*>(p->xf.chirp),
                  const_cast<void*>(p->xf.bhat), p->amax, p->nl_r, p->nl_z, p->nl_lam0, p->nl_b,
                  p->xq_tw, const_cast<void*>(p->xq_xf.chirp), const_cast<void*>(p->xq_xf.bhat)};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p->hsc) cudaFreeHost(p->hsc);
  if (p->graph) destroy_graph(p->graph);
  if (p->adj) free_plan(p->adj);
  delete p;
}

size_t NS(const pd_plan* p) { return (size_t)p->nt * p->S; }
size_t cbytes(const pd_plan* p) { return p->fp64 ? sizeof(double2) : sizeof(float2); }

FwdArgs fwd_base_impl(const pd_plan* p) {
  FwdArgs a;
  memset(&a, 0, sizeof(a));
  a.N = p->nt; a.logN = p->logN; a.nh = p->nh; a.S = p->S; a.TX = p->TX; a.CR = p->CR;
  a.sg = p->sg;
  a.xf = p->xf;
  a.st = p->st; a.tb = p->tb;
  const double s = p->s_scale;
  const double kap[5] = {p->st.kc, p->st.kxl, p->st.kxu, p->st.kyl, p->st.kyu};
  for (int i = 0; i < 5; ++i) {
    const dfc c = dfc_from(s * kap[i]);
    a.kap[i].hi = c.hi; a.kap[i].lo = c.lo;
  }
  a.c2exact = 1;
  for (int m = 0; m < 3; ++m) {
    const dfc c = dfc_from(p->tb.c2[m]);
    a.e2[m].hi = c.hi; a.e2[m].lo = c.lo;
    int e = 0;
    const double fr = std::frexp(std::fabs(p->tb.c2[m]), &e);
    if (!(p->tb.c2[m] == 0.0 || fr == 0.5)) a.c2exact = 0;
  }
  a.rscale2 = 1.0 / (s * s);
  a.gam = p->gam;
  a.tw = p->tw;
  a.out = p->spec;
  if (p->xform_tc) {
    a.amax = p->amax;
    a.amax_reset = p->amax + 1;
  }
  return a;
}

InvArgs inv_base_impl(const pd_plan* p) {
  InvArgs a;
  memset(&a, 0, sizeof(a));
  a.N = p->nt; a.logN = p->logN; a.nh = p->nh; a.S = p->S; a.TX = p->TX; a.CR = p->CR;
  a.sg = p->sg;
  a.xf = p->xf;
  a.in = p->spec;
  a.igam = p->igam;
  a.tw = p->tw;
  a.flag = p->dflag;
  return a;
}

// x-eigentransform of every spectrum row: forward (spec -> spec2) or inverse
// (spec2 -> spec); tensor cores on the mixed path, CUDA cores on the FP64 path
pd_status xform_dir(pd_plan* p, bool fwd) {
  if (p->xform_tc && p->xeng == PD_XFORM_TENSOR) {
    LK(launch_xform_tc(fwd ? p->xtc_fwd : p->xtc_inv, p->dflag, p->stream));
    return PD_OK;
  }
  if (p->xq) {
    XfftArgs xa;
    xa.rows = p->nh * (p->S / p->sp.nx);
    xa.nx = p->sp.nx;
    xa.ld = p->sg.nxp;
    xa.L = p->xq_L;
    xa.logL = ilog2(p->xq_L);
    xa.dst = p->xq_dst;
    xa.inv = fwd ? 0 : 1;
    xa.xf = p->xq_xf;
    xa.tw = p->xq_tw;
    xa.L1 = p->xq_L1;
    xa.L2 = p->xq_L2;
    xa.in = fwd ? p->spec : p->spec2;
    xa.out = fwd ? p->spec2 : p->spec;
    LK(launch_xform_fft(xa, p->fp64, p->stream));
    return PD_OK;
  }
  XformArgs xa;
  xa.rows = p->nh * (p->S / p->sp.nx);
  xa.nx = p->sp.nx;
  xa.ld = p->sg.nxp;
  xa.Q = fwd ? p->Qf : p->Qi;
  xa.in = fwd ? p->spec : p->spec2;
  xa.out = fwd ? p->spec2 : p->spec;
  LK(launch_xform(xa, p->fp64, p->stream));
  return PD_OK;
}

TriArgs tri_args_impl(const pd_plan* p, void* data) {
  TriArgs ta;
  ta.nh = p->nh; ta.J = p->J; ta.n = p->tri_n; ta.S = p->sg.specS; ta.stride = p->tri_stride;
  ta.cl = p->tri_cl; ta.cd = p->tri_cd; ta.cu = p->tri_cu;
  ta.lam = p->lam; ta.mu = p->xform ? p->mu : nullptr; ta.data = data; ta.flag = p->dflag;
  ta.amax = p->xform_tc ? p->amax + 1 : nullptr;
  ta.amax_reset = p->xform_tc ? p->amax : nullptr;
  ta.cls = p->tri_cls;
  ta.rows = p->tri_rows;
  return ta;
}

// step (b), with the x-eigentransform around it for 2D / periodic-x problems
pd_status step_b(pd_plan* p) {
  PdRange range("pd.step_b");
  void* data = p->spec;
  if (p->xform) {
    CHK(xform_dir(p, true));
    data = p->spec2;
  }
  LK(launch_tridiag(tri_args_impl(p, data), p->fp64, p->stream));
  if (p->xform) CHK(xform_dir(p, false));
  return PD_OK;
}

pd_status precond_into(pd_plan* p, const double* r, double* z) {
  {
    PdRange range("pd.step_a");
    FwdArgs fa = fwd_base_impl(p);
    fa.mode = FWD_STANDALONE;
    fa.r64 = r;
    LK(launch_time_fwd(fa, p->fp64, p->stream));
  }
  CHK(step_b(p));
  PdRange range("pd.step_c");
  InvArgs ia = inv_base_impl(p);
  ia.mode = INV_OUT64;
  ia.out64 = z;
  LK(launch_time_inv(ia, p->fp64, p->stream));
  return PD_OK;
}

pd_status sync_scalars(pd_plan* p, int nscal) {
  CU(cudaMemcpyAsync(p->hsc, p->dsc, nscal * sizeof(double), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaMemcpyAsync(p->hsc + NSC - 1, p->dflag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return PD_OK;
}

int flag_value(const pd_plan* p) {
  int f;
  memcpy(&f, p->hsc + NSC - 1, sizeof(int));
  return f;
}
bool flag_set(const pd_plan* p) { return flag_value(p) != 0; }

// status for a raised device flag: bit 1 = a bounded wait of the tensor-core
// pipeline expired, bit 0 = a non-finite value
pd_status flag_status(pd_plan* p) {
  const int f = flag_value(p);
  if (f & 2) return set_err(p, PD_ERR_CUDA, "tensor-core x-transform pipeline timed out");
  return set_err(p, PD_ERR_NONFINITE, "non-finite value in the solver");
}

// ---------------------------------------------------------------------------
// Plan-time autotuner (mixed plans with a solver state of at least 2^18
// unknowns): times, on the plan's own (zeroed) buffers with CUDA events, the
// iteration's time kernels for two tile widths (8 or 16 complex elements per
// thread) and the tridiagonal solve for two lane classes (the default and one
// more PCR level), and keeps the faster of each.  Both candidates of either
// choice are exact implementations of the same step, so results stay within
// the tolerances of the tests whichever is kept.
// ---------------------------------------------------------------------------
pd_status time_ms(pd_plan* p, int reps, float* ms, const std::function<pd_status()>& body) {
  cudaEvent_t e0, e1;
  CU(cudaEventCreate(&e0));
  CU(cudaEventCreate(&e1));
  pd_status st = body();  // warm-up (and attribute setup)
  if (st == PD_OK) {
    cudaEventRecord(e0, p->stream);
    for (int r = 0; r < reps && st == PD_OK; ++r) st = body();
    cudaEventRecord(e1, p->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return st;
}

pd_status autotune_plan(pd_plan* p) {
  if (p->fp64 || !p->Udf || NS(p) < (1u << 18)) return PD_OK;
  const unsigned long long launches = p->launches;
  CU(cudaMemsetAsync(p->Udf, 0, NS(p) * sizeof(float2), p->stream));
  CU(cudaMemsetAsync(p->Bdf, 0, NS(p) * sizeof(float2), p->stream));
  const int rows = p->xf.M ? p->xf.M : p->nt;
  // time kernels: one block per tile with budgets of 4096 and 8192 reals, or
  // the tile split over a cluster of 2, 4 or 8 blocks
  struct TimeCand { int cr, tx; };
  std::vector<TimeCand> tcands;
  int tx1 = 0;
  if (time_shape_ok(p, 1, &tx1)) {
    tcands.push_back({1, tx1});
    const int tx_a = std::max(2, std::min(32, 4096 / rows));
    if (tx_a != tx1) tcands.push_back({1, tx_a});
  }
  for (int cr : {2, 4, 8}) {
    int tx = 0;
    if (time_shape_ok(p, cr, &tx)) tcands.push_back({cr, tx});
  }
  if (tcands.size() > 1) {
    float best = -1.f;  // no candidate timed yet
    int best_tx = p->TX, best_cr = p->CR;
    for (const TimeCand& tcn : tcands) {
      p->TX = tcn.tx;
      p->CR = tcn.cr;
      float ms = 0.f;
      CHK(time_ms(p, 3, &ms, [&]() -> pd_status {
        FwdArgs fa = fwd_base_impl(p);
        fa.mode = FWD_RESIDUAL;
        fa.Udf = p->Udf;
        fa.Bdf = p->Bdf;
        LK(launch_time_fwd(fa, false, p->stream));
        InvArgs ia = inv_base_impl(p);
        ia.mode = INV_UPDATE_DF;
        ia.Udf = p->Udf;
        ia.igam = p->igam_s;
        LK(launch_time_inv(ia, false, p->stream));
        return PD_OK;
      }));
      if (best < 0.f || ms < best) { best = ms; best_tx = tcn.tx; best_cr = tcn.cr; }
    }
    p->TX = best_tx;
    p->CR = best_cr;
  }
  // tridiagonal: the default lane class, one more PCR level (chunks of at
  // least two rows), and the 16-rows-per-lane form at its own default class
  const int c0 = tridiag_class(p->tri_n, false);
  const int c16 = tridiag_class(p->tri_n, false, 16);
  if (c0 >= 0) {
    void* data = p->xform ? p->spec2 : p->spec;
    const size_t specb = (size_t)p->nh * p->sg.specS * sizeof(float2);
    CU(cudaMemsetAsync(data, 0, specb, p->stream));
    struct Cand { int cls, rows; };
    std::vector<Cand> cands = {{c0, 0}};
    if (c0 + 1 < TRI_NCLASS && (2 << c0) * 2 <= p->tri_n) cands.push_back({c0 + 1, 0});
    if (c16 >= 0 && c16 > c0) cands.push_back({c16, 16});
    float best = -1.f;  // no candidate timed yet
    Cand pick = cands[0];
    for (const Cand& c : cands) {
      p->tri_cls = c.cls;
      p->tri_rows = c.rows;
      float ms = 0.f;
      CHK(time_ms(p, 3, &ms, [&]() -> pd_status {
        LK(launch_tridiag(tri_args_impl(p, data), false, p->stream));
        return PD_OK;
      }));
      if (best < 0.f || ms < best) { best = ms; pick = c; }
    }
    p->tri_rows = pick.rows;
    p->tri_cls = (pick.rows == 0 && pick.cls == c0) || (pick.rows == 16 && pick.cls == c16) ? -1 : pick.cls;
  }
  // x-eigentransform: the tensor-core GEMM against the FP32 FFT
  if (p->xform_tc && p->xq) {
    const size_t specb = (size_t)p->nh * p->sg.specS * sizeof(float2);
    CU(cudaMemsetAsync(p->spec, 0, specb, p->stream));
    CU(cudaMemsetAsync(p->spec2, 0, specb, p->stream));
    CU(cudaMemsetAsync(p->amax, 0, 2 * sizeof(unsigned), p->stream));
    float best = -1.f;  // no candidate timed yet
    int pick = PD_XFORM_TENSOR;
    for (int eng : {PD_XFORM_TENSOR, PD_XFORM_FFT}) {
      p->xeng = eng;
      float ms = 0.f;
      CHK(time_ms(p, 3, &ms, [&]() -> pd_status {
        CHK(xform_dir(p, true));
        return xform_dir(p, false);
      }));
      if (best < 0.f || ms < best) { best = ms; pick = eng; }
    }
    p->xeng = pick;
  }
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  CU(cudaStreamSynchronize(p->stream));
  p->launches = launches;
  p->tuned = 1;
  return PD_OK;
}

// ---------------------------------------------------------------------------
// The mixed stationary iteration (eq. 5.1) as one CUDA graph: a WHILE node
// whose body is [forward kernel (residual, norm) -> check kernel -> IF node
// [step (b), inverse kernel + update]].  The check kernel takes the decisions
// of the host loop below (tolerance, maxit, device error flags, the norm-only
// prediction) on the device, so a solve has no host round trip per iteration.
// The entry and exit kernels touch the caller's arrays and stay outside.
// ---------------------------------------------------------------------------
enum { LS_RUNNING = 0, LS_CONVERGED, LS_MAXIT, LS_NONFINITE, LS_TIMEOUT, LS_ZERO_RHS };

__global__ void k_loop_check(LoopState* st, double* dsc, const int* flag,
                             cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hif) {
  if (threadIdx.x != 0) return;
  LoopState s = *st;
  ++s.n_body;
  bool stop = true, update = false;
  const double nb = sqrt(dsc[0]) / s.s_scale;
  if (nb == 0.0) {
    s.status = LS_ZERO_RHS;
    s.rel = 0.0;
  } else {
    const double rel = sqrt(dsc[1]) / nb;
    s.rel = rel;
    const int f = *flag;
    if (f != 0) {
      s.status = (f & 2) ? LS_TIMEOUT : LS_NONFINITE;
    } else if (!isfinite(rel)) {
      s.status = LS_NONFINITE;
    } else if (rel <= s.tol) {
      s.status = LS_CONVERGED;
    } else if (s.it >= s.maxit) {
      s.status = LS_MAXIT;
    } else if (s.norm_only) {  // predicted convergence missed: redo with the transform
      s.norm_only = 0;
      stop = false;
    } else {
      update = true;
      stop = false;
      ++s.it;
      ++s.n_update;
      // the first update of a zero iterate stores the correction
      s.imode = (s.zero_guess && s.n_update == 1) ? INV_SET_DF : INV_UPDATE_DF;
      if (s.prev_rel > 0.0) {
        const double rho = rel / s.prev_rel;
        s.norm_only = (rho < 1.0 && rel * rho <= 0.25 * s.tol) ? 1 : 0;
      }
      s.prev_rel = rel;
    }
  }
  dsc[1] = 0.0;  // accumulator of the next forward kernel
  s.kmode = s.norm_only ? FWD_RESIDUAL_NORM : FWD_RESIDUAL;
  *st = s;
  cudaGraphSetConditional(hif, update ? 1u : 0u);
  cudaGraphSetConditional(hw, stop ? 0u : 1u);
}

// start of a graph solve: the loop state set on the device (no host buffer
// that a queued copy could still be reading).  nonzero: raised by the entry
// kernel when the initial guess has a nonzero entry; from a zero guess the
// first forward kernel forms r = s b without reading the iterate
__global__ void k_loop_init(LoopState* st, double tol, double s_scale, int maxit,
                            const int* nonzero) {
  LoopState s;
  memset(&s, 0, sizeof(s));
  s.tol = tol;
  s.s_scale = s_scale;
  s.prev_rel = -1.0;
  s.maxit = maxit;
  s.zero_guess = *nonzero == 0 ? 1 : 0;
  s.kmode = s.zero_guess ? FWD_ZERO_GUESS : FWD_RESIDUAL;
  s.imode = INV_UPDATE_DF;
  *st = s;
}

// end of a graph solve: u = hi + lo of the double-float iterate, or zero when
// the right-hand side was zero (decided on the device)
__global__ void k_loop_exit(const LoopState* st, const float2* U, double* u, size_t n) {
  const bool zero = st->status == LS_ZERO_RHS;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x) {
    const float2 v = U[i];
    u[i] = zero ? 0.0 : double_from_float(v.x) + double_from_float(v.y);
  }
}

// the leaf node of a graph built by one stream capture (a chain)
cudaGraphNode_t graph_leaf(cudaGraph_t g) {
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return nullptr;
  std::vector<cudaGraphNode_t> nodes(n);
  if (cudaGraphGetNodes(g, nodes.data(), &n) != cudaSuccess) return nullptr;
  for (cudaGraphNode_t v : nodes) {
    size_t d = 0;
    if (cudaGraphNodeGetDependentNodes(v, nullptr, nullptr, &d) == cudaSuccess && d == 0) return v;
  }
  return nullptr;
}

// device address of pinned, device-mapped host memory (null for any other
// host pointer, which then goes through staging copies)
void* mapped_alias(const void* h) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, h) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

pd_status build_graph_impl(pd_plan* p, SolveGraph* G) {
  CU(cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking));
  CU(cudaMalloc(&G->dst, sizeof(LoopState)));
  CU(cudaMallocHost(&G->res, sizeof(LoopState)));
  CU(cudaGraphCreate(&G->g, 0));
  cudaGraphConditionalHandle hw, hif;
  CU(cudaGraphConditionalHandleCreate(&hw, G->g, 1u, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char wbuf[sizeof(cudaGraphNodeParams)];
  memset(wbuf, 0, sizeof(wbuf));
  cudaGraphNodeParams& wp = *reinterpret_cast<cudaGraphNodeParams*>(wbuf);
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  CU(cudaGraphAddNode(&wnode, G->g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  CU(cudaGraphConditionalHandleCreate(&hif, body, 0u, cudaGraphCondAssignDefault));

  // body: forward kernel (mode from the device word) + check
  const cudaStream_t saved = p->stream;
  const unsigned long long launches = p->launches;
  p->stream = G->cs;
  pd_status st = PD_OK;
  cudaError_t e = cudaStreamBeginCaptureToGraph(G->cs, body, nullptr, nullptr, 0,
                                                cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    FwdArgs fa = fwd_base_impl(p);
    fa.mode = FWD_RESIDUAL;
    fa.mode_dev = &G->dst->kmode;
    fa.norm2 = p->dsc + 1;
    fa.Udf = p->Udf;
    fa.Bdf = p->Bdf;
    e = launch_time_fwd(fa, false, G->cs);
    if (e == cudaSuccess) {
      k_loop_check<<<1, 32, 0, G->cs>>>(G->dst, p->dsc, p->dflag, hw, hif);
      e = cudaGetLastError();
    }
    cudaGraph_t out = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(G->cs, &out);
    if (e == cudaSuccess) e = e2;
  }
  cudaGraphNode_t leaf = e == cudaSuccess ? graph_leaf(body) : nullptr;
  if (e == cudaSuccess && leaf == nullptr) e = cudaErrorUnknown;
  cudaGraph_t ubody = nullptr;
  if (e == cudaSuccess) {
    alignas(cudaGraphNodeParams) unsigned char ibuf[sizeof(cudaGraphNodeParams)];
    memset(ibuf, 0, sizeof(ibuf));
    cudaGraphNodeParams& ip = *reinterpret_cast<cudaGraphNodeParams*>(ibuf);
    ip.type = cudaGraphNodeTypeConditional;
    ip.conditional.handle = hif;
    ip.conditional.type = cudaGraphCondTypeIf;
    ip.conditional.size = 1;
    cudaGraphNode_t inode;
    e = cudaGraphAddNode(&inode, body, &leaf, nullptr, 1, &ip);
    if (e == cudaSuccess) ubody = ip.conditional.phGraph_out[0];
  }
  // IF body: step (b) and the inverse kernel with the update
  if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(G->cs, ubody, nullptr, nullptr, 0,
                                                          cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const unsigned long long l0 = p->launches;
    st = step_b(p);
    if (st == PD_OK) {
      InvArgs ia = inv_base_impl(p);
      ia.mode = INV_UPDATE_DF;
      ia.mode_dev = &G->dst->imode;
      ia.Udf = p->Udf;
      ia.igam = p->igam_s;
      const cudaError_t e3 = launch_time_inv(ia, false, G->cs);
      ++p->launches;
      if (e3 != cudaSuccess) st = fail_cuda(p, e3, "inverse kernel capture");
    }
    G->update_kernels = (int)(p->launches - l0);
    cudaGraph_t out = nullptr;
    e = cudaStreamEndCapture(G->cs, &out);
  }
  p->stream = saved;
  p->launches = launches;
  if (st != PD_OK) return st;
  if (e != cudaSuccess) return fail_cuda(p, e, "solver graph capture");
  CU(cudaGraphInstantiate(&G->ge, G->g, 0));
  return PD_OK;
}

// the graph of plan p, built on first use; null if it cannot be built (the
// stationary solve then runs its host loop)
SolveGraph* plan_graph(pd_plan* p) {
  if (p->graph_state == 1) return p->graph;
  if (p->graph_state < 0) return nullptr;
  SolveGraph* G = new (std::nothrow) SolveGraph();
  if (!G) {
    p->graph_state = -1;
    return nullptr;
  }
  if (build_graph_impl(p, G) != PD_OK) {
    destroy_graph(G);
    cudaGetLastError();
    p->graph_state = -1;
    return nullptr;
  }
  p->graph = G;
  p->graph_state = 1;
  return G;
}

// Enqueue one graph solve (entry split, loop-state init, the graph, exit);
// the final loop state is copied to G->res.  No host synchronisation.
pd_status enqueue_graph_solve(pd_plan* p, SolveGraph* G, const double* b, double* u, double tol,
                              int maxit) {
  const size_t ns = NS(p);
  // dsc[0]: ||s b||^2, dsc[1]: ||r'||^2, dsc[3] (as int): nonzero initial guess
  int* nonzero = reinterpret_cast<int*>(p->dsc + 3);
  CU(cudaMemsetAsync(p->dsc, 0, 4 * sizeof(double), p->stream));
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  LK(launch_entry_df(u, b, p->s_scale, p->Udf, p->Bdf, ns, p->dsc, p->stream, nonzero));
  k_loop_init<<<1, 1, 0, p->stream>>>(G->dst, tol, p->s_scale, maxit, nonzero);
  LK(cudaGetLastError());
  CU(cudaGraphLaunch(G->ge, p->stream));
  const int grid = (int)std::min<size_t>((ns + 255) / 256, (size_t)152 * 16);
  k_loop_exit<<<grid, 256, 0, p->stream>>>(G->dst, p->Udf, u, ns);
  LK(cudaGetLastError());
  CU(cudaMemcpyAsync(G->res, G->dst, sizeof(LoopState), cudaMemcpyDeviceToHost, p->stream));
  ++G->pending;
  return PD_OK;
}

// Wait for the queued graph solves and report the last one.
pd_status finish_graph_solves(pd_plan* p, SolveGraph* G, int* iters, double* relres) {
  CU(cudaStreamSynchronize(p->stream));
  const LoopState* h = G->res;
  p->launches += (unsigned long long)G->pending *
                 ((unsigned long long)h->n_body * 2 + (unsigned long long)h->n_update * G->update_kernels);
  G->pending = 0;
  if (iters) *iters = h->it;
  if (relres) *relres = h->rel;
  switch (h->status) {
    case LS_CONVERGED:
    case LS_ZERO_RHS: return PD_OK;
    case LS_MAXIT: return set_err(p, PD_ERR_NOT_CONVERGED, "stationary iteration reached maxit");
    case LS_TIMEOUT: return set_err(p, PD_ERR_CUDA, "tensor-core x-transform pipeline timed out");
    case LS_NONFINITE: return set_err(p, PD_ERR_NONFINITE, "non-finite value in the solver");
    default: return set_err(p, PD_ERR_CUDA, "solver graph ended without a decision");
  }
}

pd_status solve_stationary_graph(pd_plan* p, SolveGraph* G, const double* b, double* u,
                                 double tol, int maxit, int* iters, double* relres) {
  CHK(enqueue_graph_solve(p, G, b, u, tol, maxit));
  return finish_graph_solves(p, G, iters, relres);
}

pd_status solve_stationary(pd_plan* p, const double* b, double* u, double tol, int maxit,
                           int* iters, double* relres) {
  if (!p->fp64) {
    SolveGraph* G = plan_graph(p);
    if (G) return solve_stationary_graph(p, G, b, u, tol, maxit, iters, relres);
  }
  const size_t ns = NS(p);
  CU(cudaMemsetAsync(p->dsc, 0, 2 * sizeof(double), p->stream));
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  // ||b||^2 into dsc[0]: FP64 on the FP64 path; on the mixed path ||s b||^2
  // from the split (rescaled after the copy to the host)
  if (p->fp64) LK(launch_norm2(b, ns, p->dsc, p->stream));
  else LK(launch_entry_df(u, b, p->s_scale, p->Udf, p->Bdf, ns, p->dsc, p->stream));
  int it = 0;
  double rel = 0.0, prev_rel = -1.0;
  // when the observed contraction predicts that the next residual meets the
  // tolerance with margin, the next forward kernel computes the residual norm
  // only; if the prediction fails it is run again with the transform
  bool norm_only = false;
  pd_status st = PD_OK;
  for (;;) {
    CU(cudaMemsetAsync(p->dsc + 1, 0, sizeof(double), p->stream));
    {
      PdRange range("pd.residual");
      FwdArgs fa = fwd_base_impl(p);
      fa.mode = norm_only ? FWD_RESIDUAL_NORM : FWD_RESIDUAL;
      fa.norm2 = p->dsc + 1;
      if (p->fp64) { fa.U64 = u; fa.B64 = b; }
      else { fa.Udf = p->Udf; fa.Bdf = p->Bdf; }
      LK(launch_time_fwd(fa, p->fp64, p->stream));
    }
    CHK(sync_scalars(p, 2));
    const double nb = std::sqrt(p->hsc[0]) / (p->fp64 ? 1.0 : p->s_scale);
    if (nb == 0.0) {
      CU(cudaMemsetAsync(u, 0, ns * sizeof(double), p->stream));
      CU(cudaStreamSynchronize(p->stream));
      rel = 0.0;
      break;
    }
    rel = std::sqrt(p->hsc[1]) / nb;
    if (flag_set(p)) { st = flag_status(p); break; }
    if (!std::isfinite(rel)) {
      st = set_err(p, PD_ERR_NONFINITE, "non-finite value in the stationary iteration");
      break;
    }
    if (rel <= tol) break;
    if (it >= maxit) {
      st = set_err(p, PD_ERR_NOT_CONVERGED, "stationary iteration reached maxit");
      break;
    }
    if (norm_only) {  // predicted convergence missed: redo this residual with the transform
      norm_only = false;
      continue;
    }
    CHK(step_b(p));
    {
      PdRange range("pd.step_c");
      InvArgs ia = inv_base_impl(p);
      if (p->fp64) { ia.mode = INV_UPDATE64; ia.out64 = u; }
      else { ia.mode = INV_UPDATE_DF; ia.Udf = p->Udf; ia.igam = p->igam_s; }
      LK(launch_time_inv(ia, p->fp64, p->stream));
    }
    ++it;
    if (prev_rel > 0.0) {
      const double rho = rel / prev_rel;
      norm_only = rho < 1.0 && rel * rho <= 0.25 * tol;
    }
    prev_rel = rel;
  }
  if (!p->fp64 && p->hsc[0] != 0.0) LK(launch_from_df(p->Udf, u, ns, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  if (iters) *iters = it;
  if (relres) *relres = rel;
  return st;
}

pd_status ensure_gmres(pd_plan* p, int m) {
  if (p->gm_cap >= m) return PD_OK;
  const size_t ns = NS(p);
  if (p->V) { cudaFree(p->V); p->V = nullptr; }
  if (p->Z) { cudaFree(p->Z); p->Z = nullptr; }
  if (p->dh) { cudaFree(p->dh); p->dh = nullptr; }
  CHK(dalloc(p, (void**)&p->V, (size_t)(m + 1) * ns * sizeof(double)));
  CHK(dalloc(p, (void**)&p->Z, (size_t)m * ns * sizeof(double)));
  CHK(dalloc(p, (void**)&p->dh, (size_t)(m + 2) * sizeof(double)));
  p->gm_cap = m;
  return PD_OK;
}

// Flexible GMRES(m), right preconditioned: u = u0 + Z y, Z_j = P^{-1} V_j;
// classical Gram-Schmidt applied twice; Givens rotations on the host.
pd_status solve_gmres(pd_plan* p, const double* b, double* u, double tol, int maxit, int restart,
                      int* iters, double* relres) {
  const size_t ns = NS(p);
  int m = restart > 0 ? restart : 30;
  m = std::min(m, std::max(1, maxit));
  CHK(ensure_gmres(p, m));
  CU(cudaMemsetAsync(p->dsc, 0, 2 * sizeof(double), p->stream));
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  LK(launch_norm2(b, ns, p->dsc, p->stream));
  CHK(sync_scalars(p, 1));
  const double nb = std::sqrt(p->hsc[0]);
  if (nb == 0.0) {
    CU(cudaMemsetAsync(u, 0, ns * sizeof(double), p->stream));
    CU(cudaStreamSynchronize(p->stream));
    if (iters) *iters = 0;
    if (relres) *relres = 0.0;
    return PD_OK;
  }
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  auto Hat = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  int total = 0;
  double rel = 0.0;
  pd_status st = PD_OK;
  for (;;) {
    CU(cudaMemsetAsync(p->dsc + 1, 0, sizeof(double), p->stream));
    CU(launch_apply_A(p->st, p->tb, p->nt, u, b, p->V, p->dsc + 1, 0, p->stream));
    CHK(sync_scalars(p, 2));
    const double beta = std::sqrt(p->hsc[1]);
    rel = beta / nb;
    if (flag_set(p)) { st = flag_status(p); break; }
    if (!std::isfinite(rel)) {
      st = set_err(p, PD_ERR_NONFINITE, "non-finite value in GMRES");
      break;
    }
    if (rel <= tol) break;
    if (total >= maxit) {
      st = set_err(p, PD_ERR_NOT_CONVERGED, "GMRES reached maxit");
      break;
    }
    LK(launch_scale_copy(1.0 / beta, p->V, p->V, ns, p->stream));
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(g.begin(), g.end(), 0.0);
    g[0] = beta;
    int jdone = 0;
    for (int j = 0; j < m; ++j) {
      double* Vj = p->V + (size_t)j * ns;
      double* Zj = p->Z + (size_t)j * ns;
      double* w = p->V + (size_t)(j + 1) * ns;
      CHK(precond_into(p, Vj, Zj));
      CU(launch_apply_A(p->st, p->tb, p->nt, Zj, nullptr, w, nullptr, 0, p->stream));
      for (int pass = 0; pass < 2; ++pass) {
        CU(cudaMemsetAsync(p->dh, 0, (j + 1) * sizeof(double), p->stream));
        LK(launch_dots(p->V, j + 1, ns, w, p->dh, p->stream));
        LK(launch_gemv_sub(p->V, j + 1, ns, p->dh, w, p->stream));
        CU(cudaMemcpyAsync(p->hsc + 8, p->dh, (j + 1) * sizeof(double), cudaMemcpyDeviceToHost,
                           p->stream));
        CU(cudaStreamSynchronize(p->stream));
        for (int i = 0; i <= j; ++i) Hat(i, j) += p->hsc[8 + i];
      }
      CU(cudaMemsetAsync(p->dsc + 2, 0, sizeof(double), p->stream));
      LK(launch_norm2(w, ns, p->dsc + 2, p->stream));
      CU(cudaMemcpyAsync(p->hsc + 2, p->dsc + 2, sizeof(double), cudaMemcpyDeviceToHost, p->stream));
      CU(cudaMemcpyAsync(p->hsc + NSC - 1, p->dflag, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
      CU(cudaStreamSynchronize(p->stream));
      if (flag_set(p)) return flag_status(p);
      const double hn = std::sqrt(p->hsc[2]);
      Hat(j + 1, j) = hn;
      if (hn > 0.0) LK(launch_scale_copy(1.0 / hn, w, w, ns, p->stream));
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
    for (int i = 0; i < jdone; ++i) p->hsc[8 + i] = y[i];
    CU(cudaMemcpyAsync(p->dh, p->hsc + 8, jdone * sizeof(double), cudaMemcpyHostToDevice, p->stream));
    LK(launch_combine(p->Z, jdone, ns, p->dh, u, p->stream));
  }
  CU(cudaStreamSynchronize(p->stream));
  if (iters) *iters = total;
  if (relres) *relres = rel;
  return st;
}

pd_status solve_any(pd_plan* p, const double* b, double* u, int mode, double tol, int maxit,
                    int restart, int* iters, double* relres) {
  if (!p || !b || !u) return set_err(p, PD_ERR_ARG, "null argument");
  if (!(tol >= 0.0) || maxit < 0) return set_err(p, PD_ERR_ARG, "tol must be >= 0 and maxit >= 0");
  PdRange range(mode == PD_GMRES ? "pd.solve.gmres" : "pd.solve.stationary");
  if (mode == PD_STATIONARY) return solve_stationary(p, b, u, tol, maxit, iters, relres);
  if (mode == PD_GMRES) {
    if (restart < 0 || restart > 64) return set_err(p, PD_ERR_ARG, "restart must be in [0, 64]");
    return solve_gmres(p, b, u, tol, maxit, restart, iters, relres);
  }
  return set_err(p, PD_ERR_ARG, "unknown solver mode");
}

// in-place radix-2 FFT (forward: exp(-2 pi i / n)) on the host in FP64, used
// to build the Bluestein filter
void host_fft(std::vector<cd>& a) {
  const size_t n = a.size();
  for (size_t i = 1, j = 0; i < n; ++i) {
    size_t bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  const double PI = 3.14159265358979323846;
  for (size_t len = 2; len <= n; len <<= 1) {
    for (size_t i = 0; i < n; i += len)
      for (size_t k = 0; k < len / 2; ++k) {
        const double th = -2.0 * PI * (double)k / (double)len;
        const cd w(std::cos(th), std::sin(th));
        const cd u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
  }
}

double hstep(int n, double L, int bc) { return L / (bc == PD_PERIODIC ? n : n + 1); }

// Tables of a length-L DFT on the GPU: for a power-of-two L the L twiddles
// e^{-2 pi i m / L}; for L = L1 L2 with L1 <= L2 <= 32 (L1 the largest such
// divisor) the same L twiddles, for one Cooley-Tukey step of two direct DFTs;
// otherwise Bluestein's form with M = 2^ceil(log2(2L - 1)): the chirp
// w_m = e^{-i pi m^2 / L} (m^2 reduced mod 2L for an accurate angle), the
// transformed filter bhat = FFT_M(conj w, wrapped) / M and the M twiddles.
// M = 0 for the first two forms.
struct DftTables {
  int M = 0;
  int L1 = 0, L2 = 0;
  std::vector<cd> tw, chirp, bhat;
};
DftTables dft_tables(int L) {
  const double PI = 3.14159265358979323846;
  DftTables t;
  if (!is_pow2(L)) {
    for (int l1 = 1; l1 * l1 <= L; ++l1)
      if (L % l1 == 0 && L / l1 <= 32) {
        t.L1 = l1;
        t.L2 = L / l1;
      }
  }
  if (!is_pow2(L) && t.L1 == 0) {
    t.M = 1;
    while (t.M < 2 * L - 1) t.M <<= 1;
    t.chirp.resize(L);
    for (int n = 0; n < L; ++n) {
      const long long q = ((long long)n * n) % (2LL * L);
      const double th = -PI * (double)q / L;
      t.chirp[n] = cd(std::cos(th), std::sin(th));
    }
    t.bhat.assign(t.M, cd(0.0, 0.0));
    t.bhat[0] = std::conj(t.chirp[0]);
    for (int m = 1; m < L; ++m) t.bhat[m] = t.bhat[t.M - m] = std::conj(t.chirp[m]);
    host_fft(t.bhat);
    for (cd& v : t.bhat) v /= (double)t.M;
  }
  const int ntw = t.M ? t.M : L;
  t.tw.resize(ntw);
  for (int m = 0; m < ntw; ++m) {
    const double th = -2.0 * PI * m / ntw;
    t.tw[m] = cd(std::cos(th), std::sin(th));
  }
  return t;
}

}  // namespace

// internal helpers shared with the batched solver (pd_batch.cu)
FwdArgs plan_fwd_args(const pd_plan* p) { return fwd_base_impl(p); }
InvArgs plan_inv_args(const pd_plan* p) { return inv_base_impl(p); }
TriArgs plan_tri_args(const pd_plan* p, void* data) { return tri_args_impl(p, data); }
pd_status plan_step_b(pd_plan* p) { return step_b(p); }
pd_status plan_xform(pd_plan* p, bool fwd) { return xform_dir(p, fwd); }
pd_status plan_fail_cuda(pd_plan* p, cudaError_t e, const char* what) { return fail_cuda(p, e, what); }
pd_status plan_precond(pd_plan* p, const double* r, double* z) { return precond_into(p, r, z); }

int time_budget(bool fp64) { return fp64 ? 2048 : 8192; }

bool time_shape_ok(const pd_plan* p, int cr, int* tx) {
  const int budget = time_budget(p->fp64);
  const int rows = p->xf.M ? p->xf.M : p->nt;
  if (cr == 1) {
    // one block of at least two columns: rows <= 4096 (mixed: 16 complex
    // elements per thread) or 2048 (FP64: 8)
    if (rows > (p->fp64 ? 2048 : 4096)) return false;
    *tx = std::max(2, std::min(32, budget / rows));
    return true;
  }
  // a cluster of cr blocks: power-of-two Nt with the half spectrum (no
  // Bluestein tables, no per-row eigenvalues), N TX = cr x budget, 2 <= TX <= 32
  if (cr != 2 && cr != 4 && cr != 8) return false;
  if (p->xf.M != 0 || !is_pow2(p->nt) || p->nh != p->nt / 2 + 1) return false;
  const long long t = (long long)budget * cr / p->nt;
  if (t < 2 || t > 32) return false;
  *tx = (int)t;
  return true;
}

extern "C" {

pd_status pd_plan_launches(const pd_plan* plan, unsigned long long* count) {
  if (!plan || !count) return PD_ERR_ARG;
  *count = plan->launches + (plan->adj ? plan->adj->launches : 0);
  return PD_OK;
}

pd_status pd_plan_tuning(const pd_plan* plan, int* tile_columns, int* tri_lanes) {
  if (!plan || !tile_columns || !tri_lanes) return PD_ERR_ARG;
  *tile_columns = plan->TX;
  const int c0 = tridiag_class(plan->tri_n, plan->fp64, plan->fp64 ? 0 : plan->tri_rows);
  const int c = plan->tri_cls > c0 ? plan->tri_cls : c0;
  *tri_lanes = c >= 0 ? 1 << c : 0;
  return PD_OK;
}

pd_status pd_plan_get_tuning(const pd_plan* plan, int* tile_columns, int* tri_lanes,
                             int* tri_rows) {
  if (!plan || !tri_rows) return PD_ERR_ARG;
  const pd_status s = pd_plan_tuning(plan, tile_columns, tri_lanes);
  if (s != PD_OK) return s;
  *tri_rows = plan->fp64 ? 16 : (plan->tri_rows == 16 ? 16 : 32);
  return PD_OK;
}

pd_status pd_plan_set_tuning(pd_plan* plan, int tile_columns, int tri_lanes, int tri_rows) {
  if (!plan) return PD_ERR_ARG;
  if (plan->fp64) return set_err(plan, PD_ERR_UNSUPPORTED, "FP64 plans use the default shapes");
  const int rows_fft = plan->xf.M ? plan->xf.M : plan->nt;
  if (plan->CR > 1) {
    if (tile_columns != plan->TX)
      return set_err(plan, PD_ERR_ARG, "tile_columns is fixed by the time cluster size");
  } else if (tile_columns < 2 || tile_columns > 32 || !is_pow2(tile_columns) ||
             (long long)tile_columns * rows_fft > 8192) {
    return set_err(plan, PD_ERR_ARG, "tile_columns out of range");
  }
  if (tri_rows != 16 && tri_rows != 32) return set_err(plan, PD_ERR_ARG, "tri_rows must be 16 or 32");
  const int c0 = tridiag_class(plan->tri_n, false, tri_rows);
  if (c0 < 0 || tri_lanes < (1 << c0) || tri_lanes > 256 || !is_pow2(tri_lanes))
    return set_err(plan, PD_ERR_ARG, "tri_lanes out of range");
  // the plan's stream may still run a solve with the old shapes
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  else cudaDeviceSynchronize();
  if (plan->graph) {
    destroy_graph(plan->graph);
    plan->graph = nullptr;
  }
  plan->graph_state = 0;
  plan->TX = tile_columns;
  plan->tri_rows = tri_rows == 16 ? 16 : 0;
  plan->tri_cls = ilog2(tri_lanes) == c0 ? -1 : ilog2(tri_lanes);
  return PD_OK;
}

pd_status pd_plan_time_cluster(const pd_plan* plan, int* blocks) {
  if (!plan || !blocks) return PD_ERR_ARG;
  *blocks = plan->CR;
  return PD_OK;
}

pd_status pd_plan_set_time_cluster(pd_plan* plan, int blocks) {
  if (!plan) return PD_ERR_ARG;
  int tx = 0;
  if (blocks != 1 && blocks != 2 && blocks != 4 && blocks != 8)
    return set_err(plan, PD_ERR_ARG, "blocks must be 1, 2, 4 or 8");
  if (!time_shape_ok(plan, blocks, &tx))
    return set_err(plan, PD_ERR_UNSUPPORTED, "no time tile of this many blocks for the plan's Nt");
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  else cudaDeviceSynchronize();
  if (plan->graph) {
    destroy_graph(plan->graph);
    plan->graph = nullptr;
  }
  plan->graph_state = 0;
  plan->CR = blocks;
  plan->TX = tx;
  return PD_OK;
}

pd_status pd_plan_set_xform_engine(pd_plan* plan, int engine) {
  if (!plan) return PD_ERR_ARG;
  if (engine != PD_XFORM_TENSOR && engine != PD_XFORM_FFT)
    return set_err(plan, PD_ERR_ARG, "engine must be PD_XFORM_TENSOR or PD_XFORM_FFT");
  if (!plan->xform) return set_err(plan, PD_ERR_UNSUPPORTED, "the plan has no x-eigentransform");
  if (engine == PD_XFORM_TENSOR && !plan->xform_tc)
    return set_err(plan, PD_ERR_UNSUPPORTED, "the plan has no tensor-core x-transform");
  if (engine == PD_XFORM_FFT && !plan->xq)
    return set_err(plan, PD_ERR_UNSUPPORTED, "the plan has no FFT x-transform");
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  else cudaDeviceSynchronize();
  if (plan->graph) {
    destroy_graph(plan->graph);
    plan->graph = nullptr;
  }
  plan->graph_state = 0;
  plan->xeng = engine;
  return PD_OK;
}

pd_status pd_plan_xform_engine(const pd_plan* plan, int* engine) {
  if (!plan || !engine) return PD_ERR_ARG;
  if (!plan->xform) *engine = -1;
  else if (plan->xform_tc && plan->xeng == PD_XFORM_TENSOR) *engine = PD_XFORM_TENSOR;
  else if (plan->xq) *engine = PD_XFORM_FFT;
  else *engine = PD_XFORM_DENSE;
  return PD_OK;
}

pd_status pd_plan_uses_graph(const pd_plan* plan, int* uses) {
  if (!plan || !uses) return PD_ERR_ARG;
  *uses = plan->graph_state == 1 ? 1 : 0;
  return PD_OK;
}

pd_status pd_profile_iteration(pd_plan* p, const double* b, const double* u, int reps,
                               float* ms) {
  if (!p || !b || !u || !ms || reps < 1) return set_err(p, PD_ERR_ARG, "bad argument");
  const size_t ns = NS(p);
  double* u64 = nullptr;
  if (p->fp64) {
    if (!p->w64b) CHK(dalloc(p, (void**)&p->w64b, ns * sizeof(double)));
    CU(cudaMemcpyAsync(p->w64b, u, ns * sizeof(double), cudaMemcpyDeviceToDevice, p->stream));
    u64 = p->w64b;
  } else {
    LK(launch_to_df(u, 1.0, p->Udf, ns, p->stream));
    LK(launch_to_df(b, p->s_scale, p->Bdf, ns, p->stream));
  }
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) CU(cudaEventCreate(&ev[i]));
  double acc[5] = {0, 0, 0, 0, 0};
  for (int r = 0; r < reps; ++r) {
    CU(cudaEventRecord(ev[0], p->stream));
    FwdArgs fa = fwd_base_impl(p);
    fa.mode = FWD_RESIDUAL;
    fa.norm2 = p->dsc + 1;
    if (p->fp64) { fa.U64 = u64; fa.B64 = b; }
    else { fa.Udf = p->Udf; fa.Bdf = p->Bdf; }
    LK(launch_time_fwd(fa, p->fp64, p->stream));
    CU(cudaEventRecord(ev[1], p->stream));
    void* data = p->spec;
    if (p->xform) {
      CHK(xform_dir(p, true));
      data = p->spec2;
    }
    CU(cudaEventRecord(ev[2], p->stream));
    LK(launch_tridiag(tri_args_impl(p, data), p->fp64, p->stream));
    CU(cudaEventRecord(ev[3], p->stream));
    if (p->xform) CHK(xform_dir(p, false));
    CU(cudaEventRecord(ev[4], p->stream));
    InvArgs ia = inv_base_impl(p);
    if (p->fp64) { ia.mode = INV_UPDATE64; ia.out64 = u64; }
    else { ia.mode = INV_UPDATE_DF; ia.Udf = p->Udf; ia.igam = p->igam_s; }
    LK(launch_time_inv(ia, p->fp64, p->stream));
    CU(cudaEventRecord(ev[5], p->stream));
    CU(cudaEventSynchronize(ev[5]));
    for (int i = 0; i < 5; ++i) {
      float t = 0.f;
      CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      acc[i] += t;
    }
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  for (int i = 0; i < 5; ++i) ms[i] = (float)(acc[i] / reps);
  if (!p->xform) { ms[1] = 0.f; ms[3] = 0.f; }
  return PD_OK;
}

pd_status pd_profile_precond(pd_plan* p, const double* r, double* z, int reps, float* ms) {
  if (!p || !r || !z || !ms || reps < 1) return set_err(p, PD_ERR_ARG, "bad argument");
  cudaEvent_t ev[6];
  for (int i = 0; i < 6; ++i) CU(cudaEventCreate(&ev[i]));
  double acc[5] = {0, 0, 0, 0, 0};
  for (int rep = 0; rep < reps; ++rep) {
    CU(cudaEventRecord(ev[0], p->stream));
    FwdArgs fa = fwd_base_impl(p);
    fa.mode = FWD_STANDALONE;
    fa.r64 = r;
    LK(launch_time_fwd(fa, p->fp64, p->stream));
    CU(cudaEventRecord(ev[1], p->stream));
    void* data = p->spec;
    if (p->xform) {
      CHK(xform_dir(p, true));
      data = p->spec2;
    }
    CU(cudaEventRecord(ev[2], p->stream));
    LK(launch_tridiag(tri_args_impl(p, data), p->fp64, p->stream));
    CU(cudaEventRecord(ev[3], p->stream));
    if (p->xform) CHK(xform_dir(p, false));
    CU(cudaEventRecord(ev[4], p->stream));
    InvArgs ia = inv_base_impl(p);
    ia.mode = INV_OUT64;
    ia.out64 = z;
    LK(launch_time_inv(ia, p->fp64, p->stream));
    CU(cudaEventRecord(ev[5], p->stream));
    CU(cudaEventSynchronize(ev[5]));
    for (int i = 0; i < 5; ++i) {
      float t = 0.f;
      CU(cudaEventElapsedTime(&t, ev[i], ev[i + 1]));
      acc[i] += t;
    }
  }
  for (int i = 0; i < 6; ++i) cudaEventDestroy(ev[i]);
  for (int i = 0; i < 5; ++i) ms[i] = (float)(acc[i] / reps);
  if (!p->xform) { ms[1] = 0.f; ms[3] = 0.f; }
  return PD_OK;
}

const char* pd_status_string(pd_status s) {
  switch (s) {
    case PD_OK: return "ok";
    case PD_ERR_ARG: return "invalid argument";
    case PD_ERR_CUDA: return "CUDA error";
    case PD_ERR_NOT_CONVERGED: return "not converged";
    case PD_ERR_NONFINITE: return "non-finite value";
    case PD_ERR_UNSUPPORTED: return "unsupported problem";
    case PD_ERR_NOMEM: return "out of device memory";
  }
  return "unknown status";
}

const char* pd_last_error(const pd_plan* plan) { return plan ? plan->msg : "null plan"; }

pd_status pd_plan_create(const pd_space* sp, int nt, double dt, double alpha, int scheme,
                         double theta, int precision, void* stream, pd_plan** out) {
  return plan_create_internal(sp, nt, dt, alpha, scheme, theta, precision, stream, true, out,
                              nullptr);
}

}  // extern "C"

// with_state = false skips the double-float iterate/right-hand side buffers
// (the batched solver keeps those packed for all problems)
pd_status plan_create_internal(const pd_space* sp, int nt, double dt, double alpha, int scheme,
                               double theta, int precision, void* stream, bool with_state,
                               pd_plan** out, const double* row_lam) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (!sp) return PD_ERR_ARG;
  if (sp->dim != 1 && sp->dim != 2) return PD_ERR_ARG;
  if (sp->nx < 1 || (sp->dim == 2 && sp->ny < 1)) return PD_ERR_ARG;
  if (!(sp->nu >= 0.0) || !(sp->lx > 0.0) || (sp->dim == 2 && !(sp->ly > 0.0))) return PD_ERR_ARG;
  if (!std::isfinite(sp->ax) || (sp->dim == 2 && !std::isfinite(sp->ay))) return PD_ERR_ARG;
  if (sp->bc_x != PD_DIRICHLET && sp->bc_x != PD_PERIODIC) return PD_ERR_ARG;
  if (sp->dim == 2 && sp->bc_y != PD_DIRICHLET && sp->bc_y != PD_PERIODIC) return PD_ERR_ARG;
  if (sp->bc_x == PD_PERIODIC && sp->nx < 2) return PD_ERR_ARG;
  if (!(dt > 0.0) || !std::isfinite(dt)) return PD_ERR_ARG;
  if (!(alpha > 0.0 && alpha <= 1.0)) return PD_ERR_ARG;
  if (scheme < PD_BE || scheme > PD_LEAPFROG) return PD_ERR_ARG;
  if (scheme == PD_THETA && !(theta >= 0.0 && theta <= 1.0)) return PD_ERR_ARG;
  if (precision != PD_FP64 && precision != PD_MIXED) return PD_ERR_ARG;
  if (nt < 1) return PD_ERR_ARG;
  // power-of-two Nt: Stockham FFT (tile rows = Nt); otherwise Bluestein with
  // M = 2^ceil(log2(2 Nt - 1)) rows; the tile must hold 2 columns at least
  // (a power-of-two Nt may be longer: the transform split over a cluster of up
  // to 8 blocks, each with two columns at least, takes Nt <= 4 x the budget)
  const int budget_rows = precision == PD_MIXED ? 4096 : 2048;
  const int max_split = 4 * time_budget(precision != PD_MIXED);
  int Mb = 0;
  if (!is_pow2(nt) && !row_lam) {
    Mb = 1;
    while (Mb < 2 * nt - 1) Mb <<= 1;
  }
  if ((Mb ? Mb : nt) > (Mb || row_lam ? budget_rows : std::max(budget_rows, max_split)))
    return PD_ERR_UNSUPPORTED;
  if (sp->dim == 2) {
    if (sp->bc_y != PD_DIRICHLET) return PD_ERR_UNSUPPORTED;
    if (sp->bc_x == PD_DIRICHLET && sp->ax != 0.0) return PD_ERR_UNSUPPORTED;
  }
  const long long S = (long long)sp->nx * (sp->dim == 2 ? sp->ny : 1);
  if (S > (1LL << 30) || S * nt > (1LL << 40)) return PD_ERR_ARG;
  // length of the tridiagonal direction of step (b)
  const int tri_len = sp->dim == 2 ? sp->ny : (sp->bc_x == PD_PERIODIC ? 1 : sp->nx);
  if (tri_len > TRI_NMAX) return PD_ERR_UNSUPPORTED;

  pd_plan* p = new (std::nothrow) pd_plan();
  if (!p) return PD_ERR_NOMEM;
  p->sp = *sp;
  if (sp->dim == 1) { p->sp.ny = 1; p->sp.ay = 0.0; p->sp.bc_y = PD_DIRICHLET; p->sp.ly = 1.0; }
  p->nt = nt;
  // ParaDiag-I plans (row_lam given) solve one shifted system per time row
  p->nh = row_lam ? nt : nt / 2 + 1;
  p->S = (int)S;
  p->logN = ilog2(nt);
  p->scheme = scheme;
  p->theta = scheme == PD_BE ? 1.0 : scheme == PD_CN ? 0.5 : theta;
  p->dt = dt;
  p->alpha = alpha;
  p->precision = precision;
  p->fp64 = precision == PD_FP64;
  p->stream = (cudaStream_t)stream;
  // tile of TX columns x Nt rows: 16 complex elements per thread in the mixed
  // path (one radix-16 butterfly per thread and pass, 32 KB of shared memory
  // for Nt >= 256), 4 in the FP64 path.  Where one block's tile would be
  // narrower than 8 columns, a power-of-two Nt is split over a cluster of
  // CR <= 8 blocks with 8 columns (or the narrowest that CR = 8 allows).
  p->xf.M = Mb;
  {
    int tx = 0;
    p->CR = 1;
    if (!time_shape_ok(p, 1, &tx) || tx < 8) {
      for (int cr : {2, 4, 8}) {
        int t = 0;
        if (!time_shape_ok(p, cr, &t)) continue;
        p->CR = cr;
        tx = t;
        if (t >= 8) break;
      }
    }
    p->TX = tx;
  }

  // spatial stencil
  Stencil& st = p->st;
  st.dim = sp->dim;
  st.nx = sp->nx;
  st.ny = p->sp.ny;
  st.S = (int)S;
  st.bcx = sp->bc_x;
  st.bcy = p->sp.bc_y;
  const double hx = hstep(sp->nx, sp->lx, sp->bc_x);
  const double kcx = 2.0 * sp->nu / (hx * hx);
  st.kxl = -sp->nu / (hx * hx) - sp->ax / (2.0 * hx);
  st.kxu = -sp->nu / (hx * hx) + sp->ax / (2.0 * hx);
  double kcy = 0.0;
  st.kyl = st.kyu = 0.0;
  if (sp->dim == 2) {
    const double hy = hstep(sp->ny, sp->ly, sp->bc_y);
    kcy = 2.0 * sp->nu / (hy * hy);
    st.kyl = -sp->nu / (hy * hy) - sp->ay / (2.0 * hy);
    st.kyu = -sp->nu / (hy * hy) + sp->ay / (2.0 * hy);
  }
  st.kc = kcx + kcy;

  // time band (first columns of B1, B2)
  TimeBand& tb = p->tb;
  memset(&tb, 0, sizeof(tb));
  if (scheme == PD_LEAPFROG) {
    tb.band = 2;
    tb.c1[0] = 1.0 / (dt * dt); tb.c1[1] = -2.0 / (dt * dt); tb.c1[2] = 1.0 / (dt * dt);
    tb.c2[0] = 0.5; tb.c2[1] = 0.0; tb.c2[2] = 0.5;
  } else {
    tb.band = 1;
    tb.c1[0] = 1.0 / dt; tb.c1[1] = -1.0 / dt;
    tb.c2[0] = p->theta; tb.c2[1] = 1.0 - p->theta;
  }
  p->s_scale = 1.0 / tb.c1[0];

  // step (b) layout
  std::vector<cd> mux;
  if (sp->dim == 2 || sp->bc_x == PD_PERIODIC) {
    p->xform = true;
    p->J = sp->nx;
    const int n = sp->nx;
    std::vector<cd> Qf((size_t)n * n), Qi((size_t)n * n);
    mux.resize(n);
    const double PI = 3.14159265358979323846;
    if (sp->bc_x == PD_PERIODIC) {
      // K_x v = mu_j v for v_x = exp(2 pi i j x / n); forward: exp(-2 pi i j x / n)
      for (int j = 0; j < n; ++j) {
        for (int x = 0; x < n; ++x) {
          const long long jx = ((long long)j * x) % n;
          const double th = 2.0 * PI * (double)jx / n;
          Qf[(size_t)j * n + x] = cd(std::cos(th), -std::sin(th));
          Qi[(size_t)x * n + j] = cd(std::cos(th), std::sin(th)) / (double)n;
        }
        const double th = 2.0 * PI * j / n;
        mux[j] = kcx + st.kxl * cd(std::cos(th), -std::sin(th)) + st.kxu * cd(std::cos(th), std::sin(th));
      }
    } else {
      // symmetric Dirichlet: sine eigenvectors sin(pi (j+1)(x+1)/(n+1)), Q^{-1} = 2/(n+1) Q
      for (int j = 0; j < n; ++j) {
        for (int x = 0; x < n; ++x) {
          const double v = std::sin(PI * (double)(j + 1) * (double)(x + 1) / (n + 1));
          Qf[(size_t)j * n + x] = cd(v, 0.0);
          Qi[(size_t)x * n + j] = cd(2.0 * v / (n + 1), 0.0);
        }
        mux[j] = kcx + 2.0 * st.kxl * std::cos(PI * (j + 1) / (n + 1));
      }
    }
    // grid lines padded to an even length: 16-byte aligned rows for TMA
    p->sg.nx = n;
    p->sg.nxp = n + (n & 1);
    p->sg.specS = (int)(S / n) * p->sg.nxp;
    pd_status s1 = upload_cplx(p, &p->Qf, Qf, p->fp64);
    if (s1 == PD_OK) s1 = upload_cplx(p, &p->Qi, Qi, p->fp64);
    if (s1 == PD_OK) s1 = upload_cplx(p, &p->mu, mux, p->fp64);
    if (s1 == PD_OK) {
      // the FFT form of the transform: DFT of length n (periodic x) or of the
      // odd extension, length 2 (n + 1) (Dirichlet x); the kernel's tile
      // holds up to 1024 transform points; tables in the plan's precision
      const int L = sp->bc_x == PD_PERIODIC ? n : 2 * (n + 1);
      DftTables t = dft_tables(L);
      if ((t.M ? t.M : L) <= 1024) {
        p->xq_L = L;
        p->xq_L1 = t.L1;
        p->xq_L2 = t.L2;
        p->xq_dst = sp->bc_x == PD_PERIODIC ? 0 : 1;
        s1 = upload_cplx(p, &p->xq_tw, t.tw, p->fp64);
        if (s1 == PD_OK && t.M) {
          void* c = nullptr;
          void* bh = nullptr;
          s1 = upload_cplx(p, &c, t.chirp, p->fp64);
          p->xq_xf.chirp = c;
          if (s1 == PD_OK) s1 = upload_cplx(p, &bh, t.bhat, p->fp64);
          p->xq_xf.bhat = bh;
          p->xq_xf.M = t.M;
          p->xq_xf.logM = ilog2(t.M);
        }
        p->xq = s1 == PD_OK;
      }
    }
    const int rows = p->nh * (int)(S / n);
    p->xform_tc = !p->fp64 && n >= 16 && rows >= 128;
    p->xeng = p->xform_tc ? PD_XFORM_TENSOR : PD_XFORM_FFT;
    if (s1 == PD_OK && p->xform_tc) {
      // real form of the complex operators, split into FP16 high and low parts:
      // G[2o][2i] = Re Q[o][i], G[2o][2i+1] = -Im, G[2o+1][2i] = Im, G[2o+1][2i+1] = Re
      const size_t P = xform_tc_bpad(n);
      for (int dir = 0; dir < 2; ++dir) {
        const std::vector<cd>& Qm = dir == 0 ? Qf : Qi;
        std::vector<float> G(P * P, 0.f);
        for (int o = 0; o < n; ++o)
          for (int i = 0; i < n; ++i) {
            const cd q = Qm[(size_t)o * n + i];
            const float v[2][2] = {{(float)q.real(), (float)-q.imag()},
                                   {(float)q.imag(), (float)q.real()}};
            for (int a = 0; a < 2; ++a)
              for (int b = 0; b < 2; ++b) G[(size_t)(2 * o + a) * P + (2 * i + b)] = v[a][b];
          }
        std::vector<uint16_t> hi, lo;
        const float ginv = xform_tc_split(G, hi, lo);
        (dir == 0 ? p->gf_inv : p->gi_inv) = ginv;
        if (s1 == PD_OK) s1 = upload(p, dir == 0 ? &p->Gf_hi : &p->Gi_hi, hi);
        if (s1 == PD_OK) s1 = upload(p, dir == 0 ? &p->Gf_lo : &p->Gi_lo, lo);
      }
      // max |value| words of the two transform inputs: [0] written by the
      // forward time kernel, [1] by the tridiagonal solver
      if (s1 == PD_OK) s1 = dalloc(p, (void**)&p->amax, 2 * sizeof(unsigned));
      if (s1 == PD_OK) {
        cudaError_t e = cudaMemset(p->amax, 0, 2 * sizeof(unsigned));
        if (e != cudaSuccess) s1 = fail_cuda(p, e, "cudaMemset");
      }
    }
    if (s1 != PD_OK) { free_plan(p); return s1; }
    if (sp->dim == 2) {
      p->tri_n = p->sp.ny; p->tri_stride = p->sg.nxp;
      p->tri_cl = st.kyl; p->tri_cd = kcy; p->tri_cu = st.kyu;
    } else {
      p->tri_n = 1; p->tri_stride = p->sg.nxp;
      p->tri_cl = 0; p->tri_cd = 0; p->tri_cu = 0;
    }
  } else {
    p->xform = false;
    p->J = 1;
    p->sg.nx = sp->nx;
    p->sg.nxp = sp->nx;
    p->sg.specS = (int)S;
    p->tri_n = sp->nx; p->tri_stride = 1;
    p->tri_cl = st.kxl; p->tri_cd = kcx; p->tri_cu = st.kxu;
  }

  // Lemma 1 eigenvalues (half spectrum) and the singularity check, or the
  // caller's per-row shifts (pairs lambda_1, lambda_2 as re, im)
  std::vector<cd> lam((size_t)2 * p->nh);
  if (row_lam) {
    for (int k = 0; k < 2 * p->nh; ++k) lam[k] = cd(row_lam[2 * k], row_lam[2 * k + 1]);
    pd_status s2 = upload_cplx(p, &p->lam, lam, p->fp64);
    const size_t specb = (size_t)p->nh * p->sg.specS * cbytes(p);
    if (s2 == PD_OK) s2 = dalloc(p, &p->spec, specb);
    if (s2 == PD_OK && p->xform) s2 = dalloc(p, &p->spec2, specb);
    if (s2 == PD_OK && p->xform_tc) {
      const int rows = p->nh * (int)(S / sp->nx);
      const int ldo = 2 * p->sg.nxp;
      cudaError_t e = xform_tc_prepare(&p->xtc_fwd, rows, sp->nx, ldo, (const float*)p->spec,
                                       (float*)p->spec2, p->Gf_hi, p->Gf_lo, p->gf_inv, p->amax);
      if (e == cudaSuccess)
        e = xform_tc_prepare(&p->xtc_inv, rows, sp->nx, ldo, (const float*)p->spec2,
                             (float*)p->spec, p->Gi_hi, p->Gi_lo, p->gi_inv, p->amax + 1);
      if (e != cudaSuccess) s2 = fail_cuda(p, e, "tensor map encoding");
    }
    if (s2 == PD_OK && !p->fp64 && with_state) s2 = dalloc(p, (void**)&p->Udf, NS(p) * sizeof(float2));
    if (s2 == PD_OK && !p->fp64 && with_state) s2 = dalloc(p, (void**)&p->Bdf, NS(p) * sizeof(float2));
    if (s2 == PD_OK) s2 = dalloc(p, (void**)&p->dsc, NSC * sizeof(double));
    if (s2 == PD_OK) s2 = dalloc(p, (void**)&p->dflag, sizeof(int));
    if (s2 == PD_OK) {
      cudaError_t e = cudaMallocHost((void**)&p->hsc, NSC * sizeof(double));
      if (e != cudaSuccess) s2 = fail_cuda(p, e, "cudaMallocHost");
    }
    if (s2 == PD_OK) {
      cudaError_t e = cudaMemset(p->dflag, 0, sizeof(int));
      if (e != cudaSuccess) s2 = fail_cuda(p, e, "cudaMemset");
    }
    if (s2 != PD_OK) {
      free_plan(p);
      return s2;
    }
    p->tuned = 1;
    *out = p;
    return PD_OK;
  }
  const double PI = 3.14159265358979323846;
  // lambda_{j,k} = sum_m c_j[m] w_k^m with w_k = e^{x + i y}, x = ln(alpha)/Nt,
  // y = -2 pi k/Nt.  For the slow modes w_k is close to 1 (|1 - w_0| is about
  // |ln alpha|/Nt), and summing the first columns as they stand would lose
  // the digits that cancel (a relative error of about eps Nt/|ln alpha| in
  // lambda_1).  The sums are therefore written with expm1 and half-angle
  // terms whose real parts add without cancellation:
  //   1 - w     = (2 sin^2(y/2) - expm1(x) cos y) - i e^x sin y,
  //   theta + (1 - theta) w: real part 2 theta cos^2(y/2) + (1 - 2 theta) cos y
  //                          + (1 - theta) expm1(x) cos y,
  //   (1 + w^2)/2: real part cos^2 y + expm1(2x) cos(2y)/2;
  // theta-schemes: lambda_1 = (1 - w)/dt, lambda_2 = theta + (1 - theta) w;
  // leap-frog: lambda_1 = (1 - w)^2/dt^2, lambda_2 = (1 + w^2)/2.
  const double lx = std::log(alpha) / nt;
  const double ex = std::exp(lx), em1 = std::expm1(lx);
  const double ex2 = std::exp(2.0 * lx), em2 = std::expm1(2.0 * lx);
  const double th_s = p->theta;
  for (int k = 0; k < p->nh; ++k) {
    const double y = -2.0 * PI * k / nt;
    const double cy = std::cos(y), sy = std::sin(y);
    const double sh = std::sin(0.5 * y), ch = std::cos(0.5 * y);
    const cd omw(2.0 * sh * sh - em1 * cy, -ex * sy);
    cd l1, l2;
    if (tb.band == 2) {
      l1 = omw * omw / (dt * dt);
      l2 = cd(cy * cy + 0.5 * em2 * std::cos(2.0 * y), 0.5 * ex2 * std::sin(2.0 * y));
    } else {
      l1 = omw / dt;
      l2 = cd(2.0 * th_s * ch * ch + (1.0 - 2.0 * th_s) * cy + (1.0 - th_s) * em1 * cy,
              (1.0 - th_s) * ex * sy);
    }
    if (nt <= tb.band) {
      // fewer levels than the band: only the first Nt entries of the first
      // columns exist (no cancellation to guard against at these sizes)
      const cd w = ex * cd(cy, sy);
      cd wm = 1;
      l1 = l2 = 0;
      for (int m = 0; m < nt; ++m) {
        l1 += tb.c1[m] * wm;
        l2 += tb.c2[m] * wm;
        wm *= w;
      }
    }
    lam[2 * k] = l1;
    lam[2 * k + 1] = l2;
  }
  if (alpha == 1.0) {
    // eigenvalues of the tridiagonal direction: cd + 2 sqrt(cl cu) cos(pi i/(n+1))
    std::vector<cd> mut;
    const int n = p->tri_n;
    for (int i = 1; i <= n; ++i)
      mut.push_back(p->tri_cd + 2.0 * std::sqrt(cd(p->tri_cl * p->tri_cu, 0.0)) * std::cos(PI * i / (n + 1)));
    if (p->xform && n == 1) mut.assign(1, cd(0.0, 0.0));
    const std::vector<cd> mx = p->xform ? mux : std::vector<cd>(1, cd(0.0, 0.0));
    for (int k = 0; k < p->nh; ++k)
      for (const cd& a : mx)
        for (const cd& b : mut) {
          const cd z = lam[2 * k] + lam[2 * k + 1] * (a + b);
          const double sc = std::abs(lam[2 * k]) + std::abs(lam[2 * k + 1]) * std::abs(a + b) + 1e-300;
          if (std::abs(z) <= 1e-12 * sc) {
            free_plan(p);
            return PD_ERR_ARG;
          }
        }
  }

  std::vector<double> gam(nt), igam(nt), igs(nt);
  for (int n = 0; n < nt; ++n) {
    gam[n] = std::pow(alpha, (double)n / nt);
    igam[n] = std::pow(alpha, -(double)n / nt) / nt;
    igs[n] = igam[n] / p->s_scale;
  }
  const int ntw = Mb ? Mb : nt;
  std::vector<cd> tw(ntw);
  for (int m = 0; m < ntw; ++m) {
    const double th = -2.0 * PI * m / ntw;
    tw[m] = cd(std::cos(th), std::sin(th));
  }
  std::vector<cd> chirp, bhat;
  if (Mb) {
    // w_n = exp(-i pi n^2 / Nt) with n^2 reduced mod 2 Nt for an accurate angle
    chirp.resize(nt);
    for (int n = 0; n < nt; ++n) {
      const long long q = ((long long)n * n) % (2LL * nt);
      const double th = -PI * (double)q / nt;
      chirp[n] = cd(std::cos(th), std::sin(th));
    }
    bhat.assign(Mb, cd(0.0, 0.0));
    bhat[0] = std::conj(chirp[0]);
    for (int m = 1; m < nt; ++m) bhat[m] = bhat[Mb - m] = std::conj(chirp[m]);
    host_fft(bhat);
    for (cd& v : bhat) v /= (double)Mb;
    p->xf.M = Mb;
    p->xf.logM = ilog2(Mb);
  }
  pd_status s2 = upload_cplx(p, &p->lam, lam, p->fp64);
  if (s2 == PD_OK) s2 = upload_real(p, &p->gam, gam, p->fp64);
  if (s2 == PD_OK) s2 = upload_real(p, &p->igam, igam, p->fp64);
  if (s2 == PD_OK) s2 = upload_real(p, &p->igam_s, igs, p->fp64);
  if (s2 == PD_OK) s2 = upload_cplx(p, &p->tw, tw, p->fp64);
  if (s2 == PD_OK && Mb) {
    void* c = nullptr;
    void* bh = nullptr;
    s2 = upload_cplx(p, &c, chirp, p->fp64);
    p->xf.chirp = c;
    if (s2 == PD_OK) s2 = upload_cplx(p, &bh, bhat, p->fp64);
    p->xf.bhat = bh;
  }
  const size_t specb = (size_t)p->nh * p->sg.specS * cbytes(p);
  if (s2 == PD_OK) s2 = dalloc(p, &p->spec, specb);
  if (s2 == PD_OK && p->xform) s2 = dalloc(p, &p->spec2, specb);
  if (s2 == PD_OK && p->xform_tc) {
    const int rows = p->nh * (int)(S / sp->nx);
    const int ldo = 2 * p->sg.nxp;
    cudaError_t e = xform_tc_prepare(&p->xtc_fwd, rows, sp->nx, ldo, (const float*)p->spec,
                                     (float*)p->spec2, p->Gf_hi, p->Gf_lo, p->gf_inv, p->amax);
    if (e == cudaSuccess)
      e = xform_tc_prepare(&p->xtc_inv, rows, sp->nx, ldo, (const float*)p->spec2,
                           (float*)p->spec, p->Gi_hi, p->Gi_lo, p->gi_inv, p->amax + 1);
    if (e != cudaSuccess) s2 = fail_cuda(p, e, "tensor map encoding");
  }
  if (s2 == PD_OK && !p->fp64 && with_state) s2 = dalloc(p, (void**)&p->Udf, NS(p) * sizeof(float2));
  if (s2 == PD_OK && !p->fp64 && with_state) s2 = dalloc(p, (void**)&p->Bdf, NS(p) * sizeof(float2));
  if (s2 == PD_OK) s2 = dalloc(p, (void**)&p->dsc, NSC * sizeof(double));
  if (s2 == PD_OK) s2 = dalloc(p, (void**)&p->dflag, sizeof(int));
  if (s2 == PD_OK) {
    cudaError_t e = cudaMallocHost((void**)&p->hsc, NSC * sizeof(double));
    if (e != cudaSuccess) s2 = fail_cuda(p, e, "cudaMallocHost");
  }
  if (s2 == PD_OK) s2 = autotune_plan(p);
  if (s2 != PD_OK) {
    free_plan(p);
    return s2;
  }
  *out = p;
  return PD_OK;
}

extern "C" {

pd_status pd_plan_destroy(pd_plan* plan) {
  if (!plan) return PD_ERR_ARG;
  if (plan->stream) cudaStreamSynchronize(plan->stream);
  else cudaDeviceSynchronize();
  free_plan(plan);
  return PD_OK;
}

pd_status pd_plan_workspace(const pd_plan* plan, unsigned long long* bytes) {
  if (!plan || !bytes) return PD_ERR_ARG;
  *bytes = plan->bytes + (plan->adj ? plan->adj->bytes : 0);
  return PD_OK;
}

pd_status pd_apply_precond(pd_plan* p, const double* r, double* z) {
  if (!p || !r || !z) return set_err(p, PD_ERR_ARG, "null argument");
  return precond_into(p, r, z);
}

pd_status pd_debug_xform_timeout(pd_plan* p, const double* r, double* z) {
  if (!p || !r || !z) return set_err(p, PD_ERR_ARG, "null argument");
  if (!p->xform || !p->xform_tc) return set_err(p, PD_ERR_UNSUPPORTED, "no tensor-core x-transform");
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  p->xtc_fwd.stall_chunk = 0;
  const pd_status s = precond_into(p, r, z);
  p->xtc_fwd.stall_chunk = -1;
  if (s != PD_OK) return s;
  CHK(sync_scalars(p, 0));
  CU(cudaMemsetAsync(p->dflag, 0, sizeof(int), p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return flag_value(p) != 0 ? flag_status(p) : PD_OK;
}

pd_status pd_residual(pd_plan* p, const double* b, const double* u, double* r) {
  if (!p || !b || !u || !r) return set_err(p, PD_ERR_ARG, "null argument");
  CU(launch_apply_A(p->st, p->tb, p->nt, u, b, r, nullptr, 0, p->stream));
  return PD_OK;
}

pd_status pd_apply_A(pd_plan* p, const double* u, double* y) {
  if (!p || !u || !y) return set_err(p, PD_ERR_ARG, "null argument");
  CU(launch_apply_A(p->st, p->tb, p->nt, u, nullptr, y, nullptr, 0, p->stream));
  return PD_OK;
}

pd_status pd_apply_AT(pd_plan* p, const double* u, double* y) {
  if (!p || !u || !y) return set_err(p, PD_ERR_ARG, "null argument");
  CU(launch_apply_A(p->st, p->tb, p->nt, u, nullptr, y, nullptr, 1, p->stream));
  return PD_OK;
}

pd_status pd_build_rhs(pd_plan* p, const double* u0, const double* u1, const double* f,
                       double* b) {
  if (!p || !u0 || !b) return set_err(p, PD_ERR_ARG, "null argument");
  LK(launch_build_rhs(p->st, p->tb, p->scheme, p->nt, p->dt, u0, u1, f, b, p->stream));
  return PD_OK;
}

pd_status pd_solve(pd_plan* p, const double* b, double* u, int mode, double tol, int maxit,
                   int restart, int* iters, double* relres) {
  return solve_any(p, b, u, mode, tol, maxit, restart, iters, relres);
}

pd_status pd_solve_windows(pd_plan* p, const double* u0, const double* f, int nwin, double* u,
                           int mode, double tol, int maxit, int restart, int* iters_total,
                           double* relres_max) {
  if (!p || !u0 || !u || nwin < 1) return set_err(p, PD_ERR_ARG, "bad argument");
  if (p->scheme == PD_LEAPFROG)
    return set_err(p, PD_ERR_UNSUPPORTED, "windowing needs a one-step scheme (theta-method)");
  const size_t ns = NS(p);
  const size_t S = (size_t)p->S;
  if (!p->w64a) CHK(dalloc(p, (void**)&p->w64a, ns * sizeof(double)));
  int total = 0;
  double worst = 0.0;
  for (int w = 0; w < nwin; ++w) {
    double* uw = u + (size_t)w * ns;
    const double* start = w == 0 ? u0 : uw - S;      // last time level of the previous window
    const double* fw = f ? f + (size_t)w * p->nt * S : nullptr;
    LK(launch_build_rhs(p->st, p->tb, p->scheme, p->nt, p->dt, start, nullptr, fw, p->w64a,
                        p->stream));
    CU(cudaMemsetAsync(uw, 0, ns * sizeof(double), p->stream));
    int it = 0;
    double rel = 0.0;
    const pd_status st = solve_any(p, p->w64a, uw, mode, tol, maxit, restart, &it, &rel);
    total += it;
    worst = std::max(worst, rel);
    if (st != PD_OK) {
      if (iters_total) *iters_total = total;
      if (relres_max) *relres_max = worst;
      return st;
    }
  }
  if (iters_total) *iters_total = total;
  if (relres_max) *relres_max = worst;
  return PD_OK;
}

pd_status pd_solve_async(pd_plan* p, const double* b, double* u, double tol, int maxit) {
  if (!p || !b || !u) return set_err(p, PD_ERR_ARG, "null argument");
  PdRange range("pd.solve.enqueue");
  if (!(tol >= 0.0) || maxit < 0) return set_err(p, PD_ERR_ARG, "tol must be >= 0 and maxit >= 0");
  if (!p->fp64) {
    SolveGraph* G = plan_graph(p);
    if (G) return enqueue_graph_solve(p, G, b, u, tol, maxit);
  }
  // no graph (FP64 plans): the synchronous host loop; its result is kept for
  // pd_solve_result
  p->async_status = solve_stationary(p, b, u, tol, maxit, &p->async_iters, &p->async_relres);
  return PD_OK;
}

pd_status pd_solve_result(pd_plan* p, int* iters, double* relres) {
  if (!p) return PD_ERR_ARG;
  if (p->graph && p->graph->pending > 0) return finish_graph_solves(p, p->graph, iters, relres);
  if (iters) *iters = p->async_iters;
  if (relres) *relres = p->async_relres;
  return p->async_status;
}

pd_status pd_solve_host(pd_plan* p, const double* b_host, double* u_host, int mode, double tol,
                        int maxit, int restart, int* iters, double* relres) {
  if (!p || !b_host || !u_host) return set_err(p, PD_ERR_ARG, "null argument");
  // Mixed stationary solves on pinned (device-mapped) host buffers read b and
  // the initial guess in the entry kernel and write u in the exit kernel
  // directly over the host link, with no staging copies.
  if (!p->fp64 && mode == PD_STATIONARY && tol >= 0.0 && maxit >= 0) {
    const double* bd = static_cast<const double*>(mapped_alias(b_host));
    double* ud = static_cast<double*>(mapped_alias(u_host));
    SolveGraph* G = (bd && ud) ? plan_graph(p) : nullptr;
    if (G) {
      CHK(enqueue_graph_solve(p, G, bd, ud, tol, maxit));
      return finish_graph_solves(p, G, iters, relres);
    }
  }
  const size_t bytes = NS(p) * sizeof(double);
  if (!p->w64a) CHK(dalloc(p, (void**)&p->w64a, bytes));
  if (!p->w64b) CHK(dalloc(p, (void**)&p->w64b, bytes));
  CU(cudaMemcpyAsync(p->w64a, b_host, bytes, cudaMemcpyHostToDevice, p->stream));
  CU(cudaMemcpyAsync(p->w64b, u_host, bytes, cudaMemcpyHostToDevice, p->stream));
  pd_status st = solve_any(p, p->w64a, p->w64b, mode, tol, maxit, restart, iters, relres);
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) return st;
  CU(cudaMemcpyAsync(u_host, p->w64b, bytes, cudaMemcpyDeviceToHost, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return st;
}

pd_status pd_adjoint_solve(pd_plan* p, const double* g, double* lam, int mode, double tol,
                           int maxit, int restart, int* iters, double* relres) {
  if (!p || !g || !lam) return set_err(p, PD_ERR_ARG, "null argument");
  PdRange range("pd.adjoint_solve");
  if (!p->adj) {
    pd_space sp2 = p->sp;
    sp2.ax = -sp2.ax;  // centred advection: K^T is K with the velocity reversed
    sp2.ay = -sp2.ay;
    pd_status s = pd_plan_create(&sp2, p->nt, p->dt, p->alpha, p->scheme, p->theta,
                                 p->precision, (void*)p->stream, &p->adj);
    if (s != PD_OK) return set_err(p, s, "creating the adjoint plan failed");
  }
  const size_t bytes = NS(p) * sizeof(double);
  if (!p->w64a) CHK(dalloc(p, (void**)&p->w64a, bytes));
  if (!p->w64b) CHK(dalloc(p, (void**)&p->w64b, bytes));
  LK(launch_flip_time(g, p->w64a, p->nt, p->S, p->stream));
  LK(launch_flip_time(lam, p->w64b, p->nt, p->S, p->stream));
  pd_status st = solve_any(p->adj, p->w64a, p->w64b, mode, tol, maxit, restart, iters, relres);
  if (st != PD_OK && st != PD_ERR_NOT_CONVERGED) {
    snprintf(p->msg, sizeof(p->msg), "adjoint: %.200s", p->adj->msg);
    return st;
  }
  LK(launch_flip_time(p->w64b, lam, p->nt, p->S, p->stream));
  CU(cudaStreamSynchronize(p->stream));
  return st;
}

}  // extern "C"
