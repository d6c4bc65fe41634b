// Batched ParaDiag-II: many independent 1D problems of uneven (nx, Nt, nu)
// solved together by the stationary iteration (eq. 5.1), every kernel type
// launched once per iteration over all problems.
//
// Problem i owns the slice [off_i, off_{i+1}) of the packed FP64 arrays b and
// u ([Nt_i][nx_i] each).  Its Lemma 1 tables and its half spectrum come from an
// internal per-problem plan; the double-float state is packed like b and u.
// The time kernels and the tridiagonal kernels read per-problem argument
// descriptors from device memory, and a work table maps every block (time
// kernels) or tile (tridiagonal) to (problem, tile).  Problems are grouped by
// the number of lanes per tridiagonal system (a power of two, chunks of at
// most 32 rows in FP32 and 16 in FP64), one launch per group.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <new>
#include <vector>

#include "pd_plan.h"

struct pd_batch {
  int np = 0;
  bool fp64 = false;
  int band = 1;
  cudaStream_t stream = nullptr;
  std::vector<pd_plan*> plans;
  std::vector<unsigned long long> off;
  unsigned long long total = 0;
  unsigned long long* d_off = nullptr;
  float2* d_bscale = nullptr;   // per problem: s_i (b is stored as s_i b)
  float2* d_one = nullptr;      // per problem: 1
  float2* Udf = nullptr;
  float2* Bdf = nullptr;
  std::vector<FwdArgs> h_fwd;
  std::vector<InvArgs> h_inv;
  std::vector<TriArgs> h_tri;
  FwdArgs* d_fwd = nullptr;
  InvArgs* d_inv = nullptr;
  TriArgs* d_tri = nullptr;
  // time-kernel work, one launch per class of tile footprint (complex
  // elements per thread: 4, 8 or 16), one block per tile of the work table
  struct TimeClass {
    int ept = 0;
    size_t smem_fwd = 0, smem_inv = 0;
    int nwork = 0;
    int2* d_work = nullptr;
  };
  static constexpr int NTC = 3;
  TimeClass tcls[NTC];
  int2* d_work_tri[TRI_NCLASS] = {};
  int ntiles_tri[TRI_NCLASS] = {};
  // work counters of the persistent tridiagonal launches, one per lane class
  static constexpr int NCTR = TRI_NCLASS;
  int* d_ctr = nullptr;
  int tuned = 0;                // 1 once the batch autotuner has run
  double* d_norms = nullptr;    // [0, np): ||b_i||^2, [np, 2np): ||r_i||^2
  double* h_norms = nullptr;    // pinned, 2np doubles + flag
  int* d_flag = nullptr;
  size_t bytes = 0;
  unsigned long long launches = 0;
  std::vector<double> relres;   // per problem, from the last residual evaluation
  char msg[256] = {0};
  // the mixed sweep as one CUDA graph (built on first use; graph_state 0
  // untried, 1 ready, -1 unavailable: the host loop runs)
  struct BatchGraph* graph = nullptr;
  int graph_state = 0;
};

// Loop state of the batched sweep graph (device copy and pinned host copy).
struct BLoop {
  double tol, rmax, prev;
  int maxit, it, status, norm_only, n_body, n_update, kmode;
};
struct BatchGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  cudaStream_t cs = nullptr;
  BLoop* dst = nullptr;
  BLoop* hst = nullptr;
  double* d_rel = nullptr;   // per-problem relative residual of the last check
  int update_kernels = 0;
  int fwd_kernels = 0;
};
void destroy_batch_graph(BatchGraph* G) {
  if (!G) return;
  if (G->ge) cudaGraphExecDestroy(G->ge);
  if (G->g) cudaGraphDestroy(G->g);
  if (G->cs) cudaStreamDestroy(G->cs);
  if (G->dst) cudaFree(G->dst);
  if (G->d_rel) cudaFree(G->d_rel);
  if (G->hst) cudaFreeHost(G->hst);
  delete G;
}

namespace {

constexpr int TB = 256;

__device__ __forceinline__ int find_problem(const unsigned long long* off, int np,
                                            unsigned long long e) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// y = df(x) * scale[problem of the element]; block b converts the contiguous
// range [b chunk, (b+1) chunk), each thread tracking its problem incrementally
__global__ void k_batch_to_df(const double* __restrict__ x, float2* __restrict__ y,
                              const unsigned long long* __restrict__ off,
                              const float2* __restrict__ scale, int np, unsigned long long total) {
  const unsigned long long chunk = ((total + gridDim.x - 1) / gridDim.x + TB - 1) / TB * TB;
  const unsigned long long e0 = blockIdx.x * chunk;
  const unsigned long long e1 = min(total, e0 + chunk);
  int p = -1;
  float2 sc = make_float2(1.f, 0.f);
  for (unsigned long long e = e0 + threadIdx.x; e < e1; e += TB) {
    if (p < 0 || (p + 1 < np && off[p + 1] <= e)) {
      p = p < 0 ? find_problem(off, np, e) : p;
      while (p + 1 < np && off[p + 1] <= e) ++p;
      sc = scale[p];
    }
    const df v = df_mul(df_from_double(x[e]), df_make(sc.x, sc.y));
    y[e] = make_float2(v.hi, v.lo);
  }
}

// out[p] += ||x_p||^2.  Block b sums the contiguous range [b chunk, (b+1) chunk)
// with coalesced loads; each thread keeps its running sum in a register and
// tracks its problem incrementally (its elements only increase), adding the
// sum into the block's shared slot of that problem when the problem changes,
// so the shared atomics are per problem boundary, not per element.
__global__ void k_batch_norm2(const double* __restrict__ x, const unsigned long long* __restrict__ off,
                              int np, unsigned long long total, double* out) {
  extern __shared__ double acc[];
  for (int i = threadIdx.x; i < np; i += TB) acc[i] = 0.0;
  __syncthreads();
  const unsigned long long chunk = ((total + gridDim.x - 1) / gridDim.x + TB - 1) / TB * TB;
  const unsigned long long e0 = blockIdx.x * chunk;
  const unsigned long long e1 = min(total, e0 + chunk);
  int p = -1;
  double sum = 0.0;
  for (unsigned long long e = e0 + threadIdx.x; e < e1; e += TB) {
    if (p < 0) {
      p = find_problem(off, np, e);
    } else if (p + 1 < np && off[p + 1] <= e) {
      atomicAdd(&acc[p], sum);
      sum = 0.0;
      while (p + 1 < np && off[p + 1] <= e) ++p;
    }
    const double v = x[e];
    sum = fma(v, v, sum);
  }
  if (p >= 0) atomicAdd(&acc[p], sum);
  __syncthreads();
  for (int i = threadIdx.x; i < np; i += TB)
    if (acc[i] != 0.0) atomicAdd(&out[i], acc[i]);
}

int grid_for(unsigned long long n) {
  unsigned long long g = (n + TB - 1) / TB;
  if (g > 152ull * 8) g = 152ull * 8;
  return g == 0 ? 1 : (int)g;
}

pd_status berr(pd_batch* b, pd_status s, const char* what) {
  if (b) snprintf(b->msg, sizeof(b->msg), "%s", what);
  return s;
}

pd_status bcuda(pd_batch* b, cudaError_t e, const char* what) {
  if (b) snprintf(b->msg, sizeof(b->msg), "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? PD_ERR_NOMEM : PD_ERR_CUDA;
}

#define BCU(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);     \
  } while (0)
#define BCHK(call)                                         \
  do {                                                     \
    pd_status s_ = (call);                                 \
    if (s_ != PD_OK) return s_;                            \
  } while (0)
#define BLK(call)                                          \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    ++b->launches;                                         \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call);     \
  } while (0)

template <typename T>
pd_status balloc(pd_batch* b, T** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    return bcuda(b, e, "cudaMalloc");
  }
  b->bytes += bytes;
  return PD_OK;
}

void free_batch(pd_batch* b) {
  if (!b) return;
  for (pd_plan* p : b->plans)
    if (p) pd_plan_destroy(p);
  void* ptrs[] = {b->d_off, b->d_bscale, b->d_one, b->Udf,     b->Bdf,
                  b->d_fwd, b->d_inv,    b->d_tri, b->d_norms, b->d_flag, b->d_ctr};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& c : b->tcls)
    if (c.d_work) cudaFree(c.d_work);
  for (int w = 0; w < TRI_NCLASS; ++w)
    if (b->d_work_tri[w]) cudaFree(b->d_work_tri[w]);
  if (b->h_norms) cudaFreeHost(b->h_norms);
  if (b->graph) destroy_batch_graph(b->graph);
  delete b;
}

// time-kernel class of a tile footprint (complex elements per thread)
int time_class(int ept) { return ept <= 4 ? 0 : ept <= 8 ? 1 : 2; }
int class_ept(int c) { return c == 0 ? 4 : c == 1 ? 8 : 16; }

// Descriptors and work tables from the members' current kernel shapes (tile
// width p->TX, tridiagonal lane class p->tri_cls): time-kernel tiles grouped
// by footprint class, tridiagonal tiles by lane class; uploaded to the device
// (replacing any earlier tables).  Per-call fields of the descriptors (state
// pointers, norms, flag) are filled by set_call_descs.
pd_status batch_tables(pd_batch* b) {
  const int np = b->np;
  const bool fp64 = b->fp64;
  std::vector<int2> wt[pd_batch::NTC];
  std::vector<int2> wtri[TRI_NCLASS];
  for (auto& c : b->tcls) {
    c.smem_fwd = c.smem_inv = 0;
    c.nwork = 0;
  }
  for (int i = 0; i < np; ++i) {
    pd_plan* p = b->plans[i];
    b->h_fwd[i] = plan_fwd_args(p);
    b->h_fwd[i].mode = FWD_RESIDUAL;
    b->h_inv[i] = plan_inv_args(p);
    b->h_tri[i] = plan_tri_args(p, p->spec);
    const int rows = p->xf.M ? p->xf.M : p->nt;
    const int c = time_class(time_tile_ept(rows, p->TX));
    pd_batch::TimeClass& tc = b->tcls[c];
    tc.ept = class_ept(c);
    const int tiles = ceil_div(p->S, p->TX);
    for (int t = 0; t < tiles; ++t) wt[c].push_back(make_int2(i, t));
    tc.smem_fwd = std::max(tc.smem_fwd, time_inv_smem(p->nt, rows, p->TX, fp64, false));
    tc.smem_inv = std::max(tc.smem_inv, time_inv_smem(p->nt, rows, p->TX, fp64, true));
    const int c0 = tridiag_class(p->tri_n, fp64);
    const int wc = p->tri_cls > c0 ? p->tri_cls : c0;
    const int SB = tridiag_batch_sb(wc, fp64);
    const long long systems = (long long)p->nh * p->J;
    const int ttiles = (int)((systems + SB - 1) / SB);
    for (int t = 0; t < ttiles; ++t) wtri[wc].push_back(make_int2(i, t));
  }
  // the costliest tiles first (Bluestein members, then longer transforms), so
  // the dynamically assigned tail of a launch is made of short tiles
  auto cost = [&](const int2& w) {
    const pd_plan* p = b->plans[w.x];
    return (p->xf.M ? 2LL : 1LL) * (p->xf.M ? p->xf.M : p->nt);
  };
  for (auto& v : wt)
    std::stable_sort(v.begin(), v.end(),
                     [&](const int2& x, const int2& y) { return cost(x) > cost(y); });
  for (int c = 0; c < pd_batch::NTC; ++c) {
    pd_batch::TimeClass& tc = b->tcls[c];
    if (tc.d_work) { cudaFree(tc.d_work); tc.d_work = nullptr; }
    tc.nwork = (int)wt[c].size();
    if (tc.nwork == 0) continue;
    BCU(cudaMalloc(&tc.d_work, wt[c].size() * sizeof(int2)));
    BCU(cudaMemcpy(tc.d_work, wt[c].data(), wt[c].size() * sizeof(int2), cudaMemcpyHostToDevice));
  }
  for (int w = 0; w < TRI_NCLASS; ++w) {
    if (b->d_work_tri[w]) { cudaFree(b->d_work_tri[w]); b->d_work_tri[w] = nullptr; }
    b->ntiles_tri[w] = (int)wtri[w].size();
    if (wtri[w].empty()) continue;
    BCU(cudaMalloc(&b->d_work_tri[w], wtri[w].size() * sizeof(int2)));
    BCU(cudaMemcpy(b->d_work_tri[w], wtri[w].data(), wtri[w].size() * sizeof(int2),
                   cudaMemcpyHostToDevice));
  }
  return PD_OK;
}

// per-call descriptor fields: the state the kernels read and write (FP64:
// the caller's arrays; mixed: the batch's double-float state), the norm
// accumulators and the flag; uploaded on the batch's stream
pd_status set_call_descs(pd_batch* b, const double* bvec, double* u) {
  const int np = b->np;
  cudaStream_t st = b->stream;
  for (int i = 0; i < np; ++i) {
    FwdArgs& fa = b->h_fwd[i];
    InvArgs& ia = b->h_inv[i];
    fa.norm2 = b->d_norms + np + i;
    if (b->fp64) {
      fa.U64 = u + b->off[i];
      fa.B64 = bvec + b->off[i];
      ia.mode = INV_UPDATE64;
      ia.out64 = u + b->off[i];
    } else {
      fa.Udf = b->Udf + b->off[i];
      fa.Bdf = b->Bdf + b->off[i];
      ia.mode = INV_UPDATE_DF;
      ia.Udf = b->Udf + b->off[i];
      ia.igam = b->plans[i]->igam_s;
    }
    ia.flag = b->d_flag;
    b->h_tri[i].flag = b->d_flag;
  }
  BCU(cudaMemcpyAsync(b->d_fwd, b->h_fwd.data(), np * sizeof(FwdArgs), cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->d_inv, b->h_inv.data(), np * sizeof(InvArgs), cudaMemcpyHostToDevice, st));
  BCU(cudaMemcpyAsync(b->d_tri, b->h_tri.data(), np * sizeof(TriArgs), cudaMemcpyHostToDevice, st));
  return PD_OK;
}

// the three kernel types of one sweep over all classes (each kernel launch
// counted; the tridiagonal work counters are zeroed first)
cudaError_t launch_fwd_all(pd_batch* b, cudaStream_t st, int* nk) {
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < pd_batch::NTC && e == cudaSuccess; ++c) {
    const auto& tc = b->tcls[c];
    if (tc.nwork == 0) continue;
    e = launch_time_fwd_batch(b->d_fwd, tc.d_work, tc.nwork, b->band, tc.smem_fwd, tc.ept,
                              b->fp64, st);
    ++*nk;
  }
  return e;
}
cudaError_t launch_tri_all(pd_batch* b, cudaStream_t st, int* nk) {
  cudaError_t e = cudaMemsetAsync(b->d_ctr, 0, TRI_NCLASS * sizeof(int), st);
  for (int w = 0; w < TRI_NCLASS && e == cudaSuccess; ++w) {
    if (b->ntiles_tri[w] == 0) continue;
    e = launch_tridiag_batch(b->d_tri, b->d_work_tri[w], b->ntiles_tri[w], w, b->fp64,
                             b->d_ctr + w, st);
    ++*nk;
  }
  return e;
}
cudaError_t launch_inv_all(pd_batch* b, cudaStream_t st, int* nk) {
  cudaError_t e = cudaSuccess;
  for (int c = 0; c < pd_batch::NTC && e == cudaSuccess; ++c) {
    const auto& tc = b->tcls[c];
    if (tc.nwork == 0) continue;
    e = launch_time_inv_batch(b->d_inv, tc.d_work, tc.nwork, tc.smem_inv, tc.ept, b->fp64, st);
    ++*nk;
  }
  return e;
}

// milliseconds per call of `body` on the batch's stream (one warm-up call,
// then `reps` timed with CUDA events)
pd_status batch_time_ms(pd_batch* b, int reps, float* ms, const std::function<cudaError_t()>& body) {
  cudaEvent_t e0, e1;
  BCU(cudaEventCreate(&e0));
  BCU(cudaEventCreate(&e1));
  cudaError_t e = body();
  if (e == cudaSuccess) {
    cudaEventRecord(e0, b->stream);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = body();
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= (float)reps;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return bcuda(b, e, "batch autotuner launch");
  return PD_OK;
}

// The batch autotuner (mixed batches): on the batch's own zeroed state, for
// every group of members sharing a transform length it times the forward and
// inverse time kernels of the whole sweep with the group's tile width at the
// default (8192 reals per tile) and at half of it, and for every group sharing
// a default tridiagonal lane class the tridiagonal launches with the default
// lane count and with twice it; each group keeps its faster choice.  Every
// candidate computes the same preconditioner up to FP32 rounding.
pd_status batch_autotune(pd_batch* b) {
  if (b->fp64) return PD_OK;
  cudaStream_t st = b->stream;
  BCU(cudaMemsetAsync(b->Udf, 0, b->total * sizeof(float2), st));
  BCU(cudaMemsetAsync(b->Bdf, 0, b->total * sizeof(float2), st));
  BCU(cudaMemsetAsync(b->d_norms, 0, 2 * b->np * sizeof(double), st));
  BCU(cudaMemsetAsync(b->d_flag, 0, sizeof(int), st));
  const unsigned long long launches = b->launches;
  int nk = 0;
  std::map<int, std::vector<int>> by_rows, by_cls;
  for (int i = 0; i < b->np; ++i) {
    pd_plan* p = b->plans[i];
    by_rows[p->xf.M ? p->xf.M : p->nt].push_back(i);
    by_cls[tridiag_class(p->tri_n, false)].push_back(i);
  }
  for (const auto& g : by_rows) {
    const int rows = g.first;
    const int tx_a = std::max(2, std::min(32, 8192 / rows)), tx_b = std::max(2, std::min(32, 4096 / rows));
    if (tx_a == tx_b) continue;
    float best = -1.f;  // no candidate timed yet
    int best_tx = tx_a;
    for (int tx : {tx_a, tx_b}) {
      for (int i : g.second) b->plans[i]->TX = tx;
      BCHK(batch_tables(b));
      BCHK(set_call_descs(b, nullptr, nullptr));
      float ms = 0.f;
      BCHK(batch_time_ms(b, 3, &ms, [&]() -> cudaError_t {
        cudaError_t e = launch_fwd_all(b, st, &nk);
        return e == cudaSuccess ? launch_inv_all(b, st, &nk) : e;
      }));
      if (best < 0.f || ms < best) { best = ms; best_tx = tx; }
    }
    for (int i : g.second) b->plans[i]->TX = best_tx;
  }
  BCHK(batch_tables(b));
  BCHK(set_call_descs(b, nullptr, nullptr));
  for (const auto& g : by_cls) {
    const int c0 = g.first;
    if (c0 < 0 || c0 + 1 >= TRI_NCLASS) continue;
    bool ok = true;
    for (int i : g.second) ok = ok && (2 << c0) * 2 <= b->plans[i]->tri_n;
    if (!ok) continue;
    float best = -1.f;  // no candidate timed yet
    int best_c = c0;
    for (int c : {c0, c0 + 1}) {
      for (int i : g.second) b->plans[i]->tri_cls = c;
      BCHK(batch_tables(b));
      BCHK(set_call_descs(b, nullptr, nullptr));
      float ms = 0.f;
      BCHK(batch_time_ms(b, 3, &ms, [&]() -> cudaError_t { return launch_tri_all(b, st, &nk); }));
      if (best < 0.f || ms < best) { best = ms; best_c = c; }
    }
    for (int i : g.second) b->plans[i]->tri_cls = best_c == c0 ? -1 : best_c;
  }
  BCHK(batch_tables(b));
  BCU(cudaMemsetAsync(b->d_flag, 0, sizeof(int), st));
  BCU(cudaStreamSynchronize(st));
  b->launches = launches;
  b->tuned = 1;
  return PD_OK;
}

enum { BS_RUNNING = 0, BS_CONVERGED, BS_MAXIT, BS_NONFINITE };

// Decisions of one batched sweep on the device (one block): per-problem
// relative residuals, their maximum, the stopping test, the norm-only
// prediction for the next forward pass, and the two graph conditions.
__global__ void k_batch_check(BLoop* st, double* norms, int np, const int* flag, double* rel,
                              cudaGraphConditionalHandle hw, cudaGraphConditionalHandle hif) {
  __shared__ double smax[TB];
  __shared__ int sbad[TB];
  double mx = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < np; i += TB) {
    const double nb = sqrt(norms[i]), nr = sqrt(norms[np + i]);
    const double r = nb > 0.0 ? nr / nb : (nr > 0.0 ? INFINITY : 0.0);
    if (!isfinite(r)) bad = 1;
    else mx = fmax(mx, r);
    rel[i] = r;
    norms[np + i] = 0.0;  // accumulator of the next forward pass
  }
  smax[threadIdx.x] = mx;
  sbad[threadIdx.x] = bad;
  __syncthreads();
  for (int o = TB / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
      sbad[threadIdx.x] |= sbad[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  BLoop s = *st;
  ++s.n_body;
  const double rmax = smax[0];
  s.rmax = rmax;
  bool stop = true, update = false;
  if (*flag != 0 || sbad[0]) {
    s.status = BS_NONFINITE;
  } else if (rmax <= s.tol) {
    s.status = BS_CONVERGED;
  } else if (s.it >= s.maxit) {
    s.status = BS_MAXIT;
  } else if (s.norm_only) {  // predicted convergence missed: redo with the transform
    s.norm_only = 0;
    stop = false;
  } else {
    update = true;
    stop = false;
    ++s.it;
    ++s.n_update;
    if (s.prev > 0.0) {
      const double rho = rmax / s.prev;
      s.norm_only = (rho < 1.0 && rmax * rho <= 0.25 * s.tol) ? 1 : 0;
    }
    s.prev = rmax;
  }
  s.kmode = s.norm_only ? FWD_RESIDUAL_NORM : FWD_RESIDUAL;
  *st = s;
  cudaGraphSetConditional(hif, update ? 1u : 0u);
  cudaGraphSetConditional(hw, stop ? 0u : 1u);
}

// the leaf node of a graph built by one stream capture (a chain)
cudaGraphNode_t batch_graph_leaf(cudaGraph_t g) {
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

// WHILE [batched forward pass -> check -> IF [tridiagonal classes, batched
// inverse pass with the update]]; the descriptors (uploaded by every solve)
// point at the batch's own buffers, so the graph does not depend on the call.
pd_status build_batch_graph(pd_batch* b, BatchGraph* G) {
  BCU(cudaStreamCreateWithFlags(&G->cs, cudaStreamNonBlocking));
  BCU(cudaMalloc(&G->dst, sizeof(BLoop)));
  BCU(cudaMalloc(&G->d_rel, b->np * sizeof(double)));
  BCU(cudaMallocHost(&G->hst, sizeof(BLoop)));
  BCU(cudaGraphCreate(&G->g, 0));
  cudaGraphConditionalHandle hw, hif;
  BCU(cudaGraphConditionalHandleCreate(&hw, G->g, 1u, cudaGraphCondAssignDefault));
  alignas(cudaGraphNodeParams) unsigned char wbuf[sizeof(cudaGraphNodeParams)];
  memset(wbuf, 0, sizeof(wbuf));
  cudaGraphNodeParams& wp = *reinterpret_cast<cudaGraphNodeParams*>(wbuf);
  wp.type = cudaGraphNodeTypeConditional;
  wp.conditional.handle = hw;
  wp.conditional.type = cudaGraphCondTypeWhile;
  wp.conditional.size = 1;
  cudaGraphNode_t wnode;
  BCU(cudaGraphAddNode(&wnode, G->g, nullptr, nullptr, 0, &wp));
  cudaGraph_t body = wp.conditional.phGraph_out[0];
  BCU(cudaGraphConditionalHandleCreate(&hif, body, 0u, cudaGraphCondAssignDefault));
  const int np = b->np;
  BCU(cudaStreamBeginCaptureToGraph(G->cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int nf = 0;
  cudaError_t e = launch_fwd_all(b, G->cs, &nf);
  G->fwd_kernels = nf;
  if (e == cudaSuccess) {
    k_batch_check<<<1, TB, 0, G->cs>>>(G->dst, b->d_norms, np, b->d_flag, G->d_rel, hw, hif);
    e = cudaGetLastError();
  }
  cudaGraph_t out = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(G->cs, &out);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return bcuda(b, e, "batch graph capture");
  cudaGraphNode_t leaf = batch_graph_leaf(body);
  if (!leaf) return berr(b, PD_ERR_CUDA, "batch graph capture");
  alignas(cudaGraphNodeParams) unsigned char ibuf[sizeof(cudaGraphNodeParams)];
  memset(ibuf, 0, sizeof(ibuf));
  cudaGraphNodeParams& ip = *reinterpret_cast<cudaGraphNodeParams*>(ibuf);
  ip.type = cudaGraphNodeTypeConditional;
  ip.conditional.handle = hif;
  ip.conditional.type = cudaGraphCondTypeIf;
  ip.conditional.size = 1;
  cudaGraphNode_t inode;
  BCU(cudaGraphAddNode(&inode, body, &leaf, nullptr, 1, &ip));
  cudaGraph_t ubody = ip.conditional.phGraph_out[0];
  BCU(cudaStreamBeginCaptureToGraph(G->cs, ubody, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
  int nk = 0;
  e = launch_tri_all(b, G->cs, &nk);
  if (e == cudaSuccess) e = launch_inv_all(b, G->cs, &nk);
  const cudaError_t e3 = cudaStreamEndCapture(G->cs, &out);
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) return bcuda(b, e, "batch graph capture");
  G->update_kernels = nk;
  BCU(cudaGraphInstantiate(&G->ge, G->g, 0));
  return PD_OK;
}

BatchGraph* batch_graph(pd_batch* b) {
  if (b->graph_state == 1) return b->graph;
  if (b->graph_state < 0) return nullptr;
  BatchGraph* G = new (std::nothrow) BatchGraph();
  if (!G) {
    b->graph_state = -1;
    return nullptr;
  }
  if (build_batch_graph(b, G) != PD_OK) {
    destroy_batch_graph(G);
    cudaGetLastError();
    b->graph_state = -1;
    return nullptr;
  }
  b->graph = G;
  b->graph_state = 1;
  return G;
}

}  // namespace

extern "C" {

pd_status pd_batch_create(const pd_problem* probs, int nprob, int precision, void* stream,
                          pd_batch** out) {
  if (!out) return PD_ERR_ARG;
  *out = nullptr;
  if (!probs || nprob < 1 || nprob > 4096) return PD_ERR_ARG;
  if (precision != PD_FP64 && precision != PD_MIXED) return PD_ERR_ARG;
  const int band0 = probs[0].scheme == PD_LEAPFROG ? 2 : 1;
  for (int i = 0; i < nprob; ++i) {
    const pd_problem& q = probs[i];
    if (q.space.dim != 1 || q.space.bc_x != PD_DIRICHLET) return PD_ERR_UNSUPPORTED;
    if ((q.scheme == PD_LEAPFROG ? 2 : 1) != band0) return PD_ERR_UNSUPPORTED;
  }
  pd_batch* b = new (std::nothrow) pd_batch();
  if (!b) return PD_ERR_NOMEM;
  b->np = nprob;
  b->fp64 = precision == PD_FP64;
  b->band = band0;
  b->stream = (cudaStream_t)stream;
  b->off.assign(nprob + 1, 0);
  for (int i = 0; i < nprob; ++i) {
    const pd_problem& q = probs[i];
    pd_plan* p = nullptr;
    pd_status s = plan_create_internal(&q.space, q.nt, q.dt, q.alpha, q.scheme, q.theta,
                                       precision, stream, false, &p);
    // the batched time kernels take one block per tile
    if (s == PD_OK && p->CR != 1) {
      int tx = 0;
      if (time_shape_ok(p, 1, &tx)) {
        p->CR = 1;
        p->TX = tx;
      } else {
        pd_plan_destroy(p);
        s = PD_ERR_UNSUPPORTED;
      }
    }
    if (s != PD_OK) {
      free_batch(b);
      return s;
    }
    b->plans.push_back(p);
    b->off[i + 1] = b->off[i] + (unsigned long long)q.nt * q.space.nx;
  }
  b->total = b->off[nprob];
  const bool fp64 = b->fp64;

  // descriptors (the work tables follow the members' kernel shapes)
  std::vector<float2> bscale(nprob), one(nprob, make_float2(1.f, 0.f));
  b->h_fwd.resize(nprob);
  b->h_inv.resize(nprob);
  b->h_tri.resize(nprob);
  for (int i = 0; i < nprob; ++i) {
    const dfc sc = dfc_from(b->plans[i]->s_scale);
    bscale[i] = make_float2(sc.hi, sc.lo);
  }
  pd_status s = PD_OK;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (s != PD_OK) return;
    s = balloc(b, (char**)dst, bytes);
    if (s == PD_OK) {
      cudaError_t e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
      if (e != cudaSuccess) s = bcuda(b, e, "cudaMemcpy");
    }
  };
  up((void**)&b->d_off, b->off.data(), b->off.size() * sizeof(unsigned long long));
  up((void**)&b->d_bscale, bscale.data(), nprob * sizeof(float2));
  up((void**)&b->d_one, one.data(), nprob * sizeof(float2));
  if (s == PD_OK) s = balloc(b, &b->d_tri, nprob * sizeof(TriArgs));
  if (s == PD_OK) s = balloc(b, &b->d_fwd, nprob * sizeof(FwdArgs));
  if (s == PD_OK) s = balloc(b, &b->d_inv, nprob * sizeof(InvArgs));
  if (s == PD_OK) s = balloc(b, &b->d_norms, 2 * nprob * sizeof(double));
  if (s == PD_OK) s = balloc(b, &b->d_flag, sizeof(int));
  if (s == PD_OK) s = balloc(b, &b->d_ctr, pd_batch::NCTR * sizeof(int));
  if (s == PD_OK && !fp64) s = balloc(b, &b->Udf, b->total * sizeof(float2));
  if (s == PD_OK && !fp64) s = balloc(b, &b->Bdf, b->total * sizeof(float2));
  if (s == PD_OK) {
    cudaError_t e = cudaMallocHost((void**)&b->h_norms, (2 * nprob + 1) * sizeof(double));
    if (e != cudaSuccess) s = bcuda(b, e, "cudaMallocHost");
  }
  if (s == PD_OK) s = batch_tables(b);
  // mixed batches of at least 2^18 unknowns: tile widths and lane counts by timing
  if (s == PD_OK && !fp64 && b->total >= (1ull << 18)) s = batch_autotune(b);
  if (s != PD_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return PD_OK;
}

pd_status pd_batch_destroy(pd_batch* b) {
  if (!b) return PD_ERR_ARG;
  if (b->stream) cudaStreamSynchronize(b->stream);
  else cudaDeviceSynchronize();
  free_batch(b);
  return PD_OK;
}

pd_status pd_batch_offsets(const pd_batch* b, unsigned long long* offsets) {
  if (!b || !offsets) return PD_ERR_ARG;
  for (int i = 0; i <= b->np; ++i) offsets[i] = b->off[i];
  return PD_OK;
}

pd_status pd_batch_uses_graph(const pd_batch* b, int* uses) {
  if (!b || !uses) return PD_ERR_ARG;
  *uses = b->graph_state == 1 ? 1 : 0;
  return PD_OK;
}

pd_status pd_batch_launches(const pd_batch* b, unsigned long long* count) {
  if (!b || !count) return PD_ERR_ARG;
  unsigned long long c = b->launches;
  for (pd_plan* p : b->plans) c += p->launches;
  *count = c;
  return PD_OK;
}

const char* pd_batch_last_error(const pd_batch* b) { return b ? b->msg : "null batch"; }

pd_status pd_batch_relres(const pd_batch* b, double* relres) {
  if (!b || !relres) return PD_ERR_ARG;
  for (int i = 0; i < b->np; ++i) relres[i] = i < (int)b->relres.size() ? b->relres[i] : 0.0;
  return PD_OK;
}

pd_status pd_batch_build_rhs(pd_batch* b, const double* u0, const double* f, double* rhs) {
  if (!b || !u0 || !rhs) return berr(b, PD_ERR_ARG, "null argument");
  unsigned long long ou = 0, of = 0;
  for (int i = 0; i < b->np; ++i) {
    pd_plan* p = b->plans[i];
    pd_status s = pd_build_rhs(p, u0 + ou, nullptr, f ? f + of : nullptr, rhs + b->off[i]);
    if (s != PD_OK) return berr(b, s, "pd_build_rhs failed for a batch member");
    ou += (unsigned long long)p->S;
    of += (unsigned long long)(p->nt + 1) * p->S;
  }
  return PD_OK;
}

pd_status pd_batch_tuned(const pd_batch* b, int* tuned) {
  if (!b || !tuned) return PD_ERR_ARG;
  *tuned = b->tuned;
  return PD_OK;
}

pd_status pd_batch_profile_sweep(pd_batch* b, const double* bvec, double* u, int reps, float* ms) {
  if (!b || !bvec || !u || !ms || reps < 1) return berr(b, PD_ERR_ARG, "bad argument");
  const int np = b->np;
  cudaStream_t st = b->stream;
  BCHK(set_call_descs(b, bvec, u));
  BCU(cudaMemsetAsync(b->d_norms, 0, 2 * np * sizeof(double), st));
  BCU(cudaMemsetAsync(b->d_flag, 0, sizeof(int), st));
  if (!b->fp64) {
    k_batch_to_df<<<grid_for(b->total), TB, 0, st>>>(u, b->Udf, b->d_off, b->d_one, np, b->total);
    BCU(cudaGetLastError());
    k_batch_to_df<<<grid_for(b->total), TB, 0, st>>>(bvec, b->Bdf, b->d_off, b->d_bscale, np,
                                                     b->total);
    BCU(cudaGetLastError());
  }
  const unsigned long long launches = b->launches;
  int nk = 0;
  BCHK(batch_time_ms(b, reps, &ms[0], [&]() -> cudaError_t { return launch_fwd_all(b, st, &nk); }));
  BCHK(batch_time_ms(b, reps, &ms[1], [&]() -> cudaError_t { return launch_tri_all(b, st, &nk); }));
  BCHK(batch_time_ms(b, reps, &ms[2], [&]() -> cudaError_t { return launch_inv_all(b, st, &nk); }));
  if (!b->fp64) BCU(launch_from_df(b->Udf, u, b->total, st));
  BCU(cudaStreamSynchronize(st));
  b->launches = launches;
  return PD_OK;
}

pd_status pd_batch_solve(pd_batch* b, const double* bvec, double* u, double tol, int maxit,
                         int* iters, double* relres_max) {
  PdRange range("pd.batch_solve");
  if (!b || !bvec || !u) return berr(b, PD_ERR_ARG, "null argument");
  if (!(tol >= 0.0) || maxit < 0) return berr(b, PD_ERR_ARG, "tol must be >= 0 and maxit >= 0");
  const int np = b->np;
  const bool fp64 = b->fp64;
  cudaStream_t st = b->stream;
  // descriptors for this call (FP64: they point into the caller's arrays)
  BCHK(set_call_descs(b, bvec, u));
  BCU(cudaMemsetAsync(b->d_norms, 0, 2 * np * sizeof(double), st));
  BCU(cudaMemsetAsync(b->d_flag, 0, sizeof(int), st));
  k_batch_norm2<<<grid_for(b->total), TB, np * sizeof(double), st>>>(bvec, b->d_off, np, b->total,
                                                                      b->d_norms);
  BLK(cudaGetLastError());
  if (!fp64) {
    k_batch_to_df<<<grid_for(b->total), TB, 0, st>>>(u, b->Udf, b->d_off, b->d_one, np, b->total);
    BLK(cudaGetLastError());
    k_batch_to_df<<<grid_for(b->total), TB, 0, st>>>(bvec, b->Bdf, b->d_off, b->d_bscale, np,
                                                     b->total);
    BLK(cudaGetLastError());
  }
  BatchGraph* G = fp64 ? nullptr : batch_graph(b);
  if (G) {
    // the whole sweep loop as one graph launch; the forward passes read
    // their mode (with or without the transform) from the loop state
    for (int i = 0; i < np; ++i) b->h_fwd[i].mode_dev = &G->dst->kmode;
    BCU(cudaMemcpyAsync(b->d_fwd, b->h_fwd.data(), np * sizeof(FwdArgs), cudaMemcpyHostToDevice,
                        st));
    for (int i = 0; i < np; ++i) b->h_fwd[i].mode_dev = nullptr;
    BLoop* h = G->hst;
    memset(h, 0, sizeof(BLoop));
    h->tol = tol;
    h->prev = -1.0;
    h->maxit = maxit;
    h->kmode = FWD_RESIDUAL;
    BCU(cudaMemcpyAsync(G->dst, h, sizeof(BLoop), cudaMemcpyHostToDevice, st));
    BCU(cudaGraphLaunch(G->ge, st));
    BCU(cudaMemcpyAsync(h, G->dst, sizeof(BLoop), cudaMemcpyDeviceToHost, st));
    b->relres.assign(np, 0.0);
    BCU(cudaMemcpyAsync(b->relres.data(), G->d_rel, np * sizeof(double), cudaMemcpyDeviceToHost,
                        st));
    BLK(launch_from_df(b->Udf, u, b->total, st));
    BCU(cudaStreamSynchronize(st));
    b->launches += (unsigned long long)h->n_body * (G->fwd_kernels + 1) +
                   (unsigned long long)h->n_update * G->update_kernels;
    if (iters) *iters = h->it;
    if (relres_max) *relres_max = h->rmax;
    if (h->status == BS_CONVERGED) return PD_OK;
    if (h->status == BS_MAXIT) return berr(b, PD_ERR_NOT_CONVERGED, "batched iteration reached maxit");
    return berr(b, PD_ERR_NONFINITE, "non-finite value in the batched iteration");
  }
  int it = 0;
  double rmax = 0.0;
  pd_status status = PD_OK;
  for (;;) {
    BCU(cudaMemsetAsync(b->d_norms + np, 0, np * sizeof(double), st));
    int nk = 0;
    const cudaError_t ef = launch_fwd_all(b, st, &nk);
    b->launches += nk;
    if (ef != cudaSuccess) return bcuda(b, ef, "batched forward time kernels");
    BCU(cudaMemcpyAsync(b->h_norms, b->d_norms, 2 * np * sizeof(double), cudaMemcpyDeviceToHost, st));
    BCU(cudaMemcpyAsync(b->h_norms + 2 * np, b->d_flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    BCU(cudaStreamSynchronize(st));
    int flag;
    memcpy(&flag, b->h_norms + 2 * np, sizeof(int));
    rmax = 0.0;
    bool finite = true;
    b->relres.assign(np, 0.0);
    for (int i = 0; i < np; ++i) {
      const double nb = std::sqrt(b->h_norms[i]);
      const double nr = std::sqrt(b->h_norms[np + i]);
      const double rel = nb > 0 ? nr / nb : (nr > 0 ? INFINITY : 0.0);
      if (!std::isfinite(rel)) finite = false;
      b->relres[i] = rel;
      rmax = std::max(rmax, rel);
    }
    if (flag || !finite) {
      status = berr(b, PD_ERR_NONFINITE, "non-finite value in the batched iteration");
      break;
    }
    if (rmax <= tol) break;
    if (it >= maxit) {
      status = berr(b, PD_ERR_NOT_CONVERGED, "batched iteration reached maxit");
      break;
    }
    nk = 0;
    cudaError_t eu = launch_tri_all(b, st, &nk);
    if (eu == cudaSuccess) eu = launch_inv_all(b, st, &nk);
    b->launches += nk;
    if (eu != cudaSuccess) return bcuda(b, eu, "batched tridiagonal / inverse time kernels");
    ++it;
  }
  if (!fp64) BLK(launch_from_df(b->Udf, u, b->total, st));
  BCU(cudaStreamSynchronize(st));
  if (iters) *iters = it;
  if (relres_max) *relres_max = rmax;
  return status;
}

}  // extern "C"
