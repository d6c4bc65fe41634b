// Internal plan structure (shared by pd_api.cu and pd_batch.cu).
#pragma once
#include "pd_internal.h"

struct pd_plan {
  pd_space sp;
  int nt = 0, nh = 0, S = 0, logN = 0, TX = 0;
  // blocks per time tile: CR > 1 splits each tile's transform over a cluster
  // of CR blocks (power-of-two Nt), with N TX = CR x the one-block budget
  int CR = 1;
  int scheme = 0;
  double theta = 1.0, dt = 0.0, alpha = 0.0;
  int precision = 0;
  bool fp64 = false;
  Stencil st;
  TimeBand tb;
  double s_scale = 1.0;
  cudaStream_t stream = nullptr;
  // spectrum layout (padded grid lines for x-transformed problems)
  SpecGeom sg;
  // step (b) layout
  bool xform = false;
  bool xform_tc = false;          // mixed path: tcgen05 x-transform
  XformTc xtc_fwd, xtc_inv;
  void* Gf_hi = nullptr;
  void* Gf_lo = nullptr;
  void* Gi_hi = nullptr;
  void* Gi_lo = nullptr;
  float gf_inv = 1.f, gi_inv = 1.f;   // scales of the FP16 operator splits
  unsigned* amax = nullptr;           // max |input| of the forward / inverse transform
  int J = 1, tri_n = 0, tri_stride = 1;
  int tri_cls = -1;                   // tridiagonal lane class (autotuned, -1: default)
  int tri_rows = 0;                   // rows per lane in registers (autotuned, 0: default)
  int tuned = 0;                      // 1 once the plan-time autotuner has run
  double tri_cl = 0, tri_cd = 0, tri_cu = 0;
  // device tables
  void* lam = nullptr;
  void* gam = nullptr;
  void* igam = nullptr;
  void* igam_s = nullptr;
  void* tw = nullptr;
  TimeXf xf = {0, 0, nullptr, nullptr};   // Bluestein tables for non-power-of-two Nt
  void* Qf = nullptr;
  void* Qi = nullptr;
  // the x-eigentransform by FFT (length xq_L DFT per row; sine transform for
  // a Dirichlet x direction), with its twiddle / Bluestein tables in the
  // plan's precision; mixed plans with the tensor-core transform too pick one
  // engine (xeng: PD_XFORM_TENSOR or PD_XFORM_FFT, autotuned)
  bool xq = false;
  int xeng = 0;
  int xq_L = 0, xq_dst = 0;
  int xq_L1 = 0, xq_L2 = 0;   // L = L1 L2: two direct DFTs (0: Stockham / Bluestein)
  TimeXf xq_xf = {0, 0, nullptr, nullptr};
  void* xq_tw = nullptr;
  void* mu = nullptr;
  // workspace
  void* spec = nullptr;
  void* spec2 = nullptr;
  float2* Udf = nullptr;
  float2* Bdf = nullptr;
  double* w64a = nullptr;
  double* w64b = nullptr;
  double* dsc = nullptr;   // device scalars
  int* dflag = nullptr;
  double* hsc = nullptr;   // pinned host scalars
  double* V = nullptr;
  double* Z = nullptr;
  double* dh = nullptr;
  int gm_cap = 0;
  // simplified Newton workspace (nonlinear problems), allocated on first use
  double* nl_r = nullptr;
  double* nl_z = nullptr;
  void* nl_lam0 = nullptr;   // copy of the plan's eigenvalue table
  double* nl_b = nullptr;    // right-hand side of one window (windowed solves)
  pd_plan* adj = nullptr;
  // the mixed stationary iteration as one CUDA graph (built on first use;
  // graph_state 0 untried, 1 ready, -1 unavailable: the host loop runs)
  struct SolveGraph* graph = nullptr;
  int graph_state = 0;
  // result of the last pd_solve_async that ran synchronously (no graph)
  pd_status async_status = PD_OK;
  int async_iters = 0;
  double async_relres = 0.0;
  size_t bytes = 0;
  unsigned long long launches = 0;
  char msg[256] = {0};
};

// helpers implemented in pd_api.cu
FwdArgs plan_fwd_args(const pd_plan* p);
InvArgs plan_inv_args(const pd_plan* p);
TriArgs plan_tri_args(const pd_plan* p, void* data);
// step (b) of the plan (x-eigentransform, shifted tridiagonal solves, inverse
// x-transform) on p->spec
pd_status plan_step_b(pd_plan* p);
// the x-eigentransform of the plan's spectrum: forward spec -> spec2, inverse
// spec2 -> spec (2D and periodic-x plans)
pd_status plan_xform(pd_plan* p, bool fwd);
pd_status plan_fail_cuda(pd_plan* p, cudaError_t e, const char* what);
// z = P_alpha^{-1} r (FP64 in and out) with the plan's current eigenvalue table
pd_status plan_precond(pd_plan* p, const double* r, double* z);
// Plan creation.  With row_lam (2 nt complex numbers as re, im pairs) the plan
// holds no time transform: its step (b) solves one system per time row n,
// (lambda_1n I + lambda_2n K) z_n = s_n, with lambda_1n = row_lam[4n] +
// i row_lam[4n+1] and lambda_2n = row_lam[4n+2] + i row_lam[4n+3].
// Time-tile shapes: one block holds at most time_budget reals (N TX); a tile
// split over CR blocks holds CR x that.  time_shape_ok says whether the plan
// can take cr blocks per tile and, if so, gives the tile's columns.
int time_budget(bool fp64);
bool time_shape_ok(const pd_plan* p, int cr, int* tx);
pd_status plan_create_internal(const pd_space* sp, int nt, double dt, double alpha, int scheme,
                               double theta, int precision, void* stream, bool with_state,
                               pd_plan** out, const double* row_lam = nullptr);
