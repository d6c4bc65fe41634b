/*
 * paradiag.h -- C ABI of the GB300 (sm_103a) ParaDiag-II library.
 *
 * Problem (Gander, Liu, Wu, Yue, Zhou, "ParaDiag: Parallel-in-Time Algorithms
 * Based on the Diagonalization Technique", arXiv:2005.09158):
 *   the all-at-once system A u = b,  A = B1 (x) M + B2 (x) K        (eq. 1.1)
 * of a linear multistep discretisation of M U' + K U = f with M = I (finite
 * differences), lower-triangular Toeplitz B1, B2 (theta-method, eq. 2.5b;
 * implicit leap-frog, eq. 3.2b), and its block alpha-circulant preconditioner
 *   P_alpha = C1^(alpha) (x) M + C2^(alpha) (x) K                   (eq. 1.2)
 * applied through the three steps of eq. 1.3 (Lemma 1): scale by Gamma_alpha
 * and FFT along time, Nt independent complex-shifted spatial solves, inverse
 * FFT and unscale.
 *
 * Conventions shared by every entry point
 *   Layout.   Space-time arrays are real FP64, time-major, [Nt][ny][nx] with x
 *             fastest: u = (U_1; ...; U_Nt) (eq. 2.5a), U_n = u at t_n.
 *   Memory.   Unless a function says otherwise, array arguments are DEVICE
 *             pointers owned by the caller; the plan owns its tables and
 *             workspace (allocated once in pd_plan_create).
 *   Streams.  All work is enqueued on the plan's stream.  Functions that need
 *             a scalar on the host (solvers) synchronise that stream.
 *   Aliasing. Inputs and outputs must not overlap, except where stated.
 *   Errors.   Every function returns a pd_status; nothing throws.  The text of
 *             the last error is available from pd_last_error(plan).
 *   Threads.  A plan must not be used by two host threads at once; distinct
 *             plans are independent.
 */
#ifndef PARADIAG_H
#define PARADIAG_H

#if defined(__GNUC__)
#define PD_API __attribute__((visibility("default")))
#else
#define PD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PD_OK = 0,
  PD_ERR_ARG = -1,            /* invalid argument (size, pointer, parameter) */
  PD_ERR_CUDA = -2,           /* a CUDA runtime call failed */
  PD_ERR_NOT_CONVERGED = -3,  /* the solver stopped at maxit above tol */
  PD_ERR_NONFINITE = -4,      /* a NaN or Inf appeared in a kernel */
  PD_ERR_UNSUPPORTED = -5,    /* valid problem that this library does not handle */
  PD_ERR_NOMEM = -6           /* device allocation failed */
} pd_status;

/* Time integrators: backward Euler and Crank-Nicolson are the theta-method of
 * eq. 2.4 with theta = 1 and 1/2; PD_THETA takes theta from the argument;
 * PD_LEAPFROG is the implicit leap-frog scheme of eq. 3.2b. */
typedef enum { PD_BE = 0, PD_CN = 1, PD_THETA = 2, PD_LEAPFROG = 3 } pd_scheme_kind;
typedef enum { PD_DIRICHLET = 0, PD_PERIODIC = 1 } pd_bc;
/* PD_MIXED: FP32 preconditioner (FFT, tridiagonal solves, x-transform) with the
 * outer residual b - A u and the update u += du kept in double-float (FP32
 * pairs, 48-bit significand).  PD_FP64: every step in FP64. */
typedef enum { PD_FP64 = 0, PD_MIXED = 1 } pd_precision;
typedef enum { PD_STATIONARY = 0, PD_GMRES = 1 } pd_mode;

/* Spatial operator K = -nu Lap_h + (ax, ay).grad_h (centred second-order
 * differences, eq. 2.2b in 1D; the 5-point stencil in 2D).  Dirichlet
 * directions hold n interior points with h = L/(n+1); periodic directions hold
 * n points with h = L/n.  dim = 2 requires bc_y = PD_DIRICHLET, and either
 * bc_x = PD_PERIODIC or (bc_x = PD_DIRICHLET and ax = 0).  The direction
 * solved by tridiagonal systems in step (b) (y in 2D, x for a Dirichlet 1D
 * problem) holds at most 4096 points (PD_ERR_UNSUPPORTED otherwise). */
typedef struct {
  int dim;        /* 1 or 2 */
  int nx, ny;     /* grid points per direction (ny ignored for dim = 1) */
  double nu;      /* diffusion coefficient */
  double ax, ay;  /* advection velocity */
  int bc_x, bc_y; /* pd_bc */
  double lx, ly;  /* domain lengths */
} pd_space;

typedef struct pd_plan pd_plan;

/* Create a plan for the all-at-once system on Nt uniform steps of size dt with
 * preconditioner parameter alpha in (0, 1] (Lemma 1).  Any Nt >= 1: powers of
 * two use a radix-16 Stockham FFT (one radix-2/4/8 pass when log2 Nt is not a
 * multiple of 4; Nt <= 32768 for PD_MIXED, <= 8192 for PD_FP64; from
 * Nt = 2048 (mixed) or 512 (FP64) on, each time tile's transform is split
 * over a thread-block cluster, pd_plan_time_cluster), other lengths
 * Bluestein's chirp-z transform of length M = 2^ceil(log2(2 Nt - 1)) with
 * M <= 4096 (mixed) or <= 2048 (FP64), i.e. Nt <= 2048 / 1024;
 * larger Nt gives PD_ERR_UNSUPPORTED.  alpha = 1 is
 * accepted only when no shifted system is singular (checked here).
 * stream: a cudaStream_t (NULL = legacy default stream).
 * Builds on the host, in FP64: the eigenvalues lambda_{j,k} of Lemma 1, the
 * Gamma tables, the FFT twiddles and (2D) the x-eigentransform; copies them to
 * the device and allocates the workspace.  *out receives the plan. */
PD_API pd_status pd_plan_create(const pd_space* sp, int nt, double dt, double alpha, int scheme,
                         double theta, int precision, void* stream, pd_plan** out);
PD_API pd_status pd_plan_destroy(pd_plan* plan);

/* Bytes of device memory the plan holds (tables + workspace). */
PD_API pd_status pd_plan_workspace(const pd_plan* plan, unsigned long long* bytes);

/* z = P_alpha^{-1} r (eq. 1.3, steps (a)-(c)); r, z: [Nt][S] device FP64. */
PD_API pd_status pd_apply_precond(pd_plan* plan, const double* r, double* z);

/* Testing aid (no paper counterpart): pd_apply_precond with the first thread
 * block of the forward tensor-core x-transform withholding all its operand
 * loads, so that its consumers' bounded waits run out (after 2^16 polls in
 * this launch).  That block then waits for the work it had issued, frees its
 * tensor memory and raises bit 1 of the plan's device flag; the call waits for
 * the stream and returns PD_ERR_CUDA ("... timed out") with z undefined, and
 * clears the flag, so that the plan stays usable.  PD_ERR_UNSUPPORTED on plans
 * without the tensor-core x-transform (1D, FP64, fewer than 16 x points or
 * 128 spectrum rows). */
PD_API pd_status pd_debug_xform_timeout(pd_plan* plan, const double* r, double* z);

/* r = b - A u (eq. 5.1); b, u, r: [Nt][S] device FP64, computed in FP64. */
PD_API pd_status pd_residual(pd_plan* plan, const double* b, const double* u, double* r);

/* y = A u (eq. 1.1) in FP64. */
PD_API pd_status pd_apply_A(pd_plan* plan, const double* u, double* y);

/* y = A^T u in FP64: the transpose of eq. 1.1, (B1^T (x) I + B2^T (x) K^T) u,
 * the operator of the adjoint system (Section 4 uses the transposed blocks
 * B1^T, B2^T in its optimality system). */
PD_API pd_status pd_apply_AT(pd_plan* plan, const double* u, double* y);

/* b of the all-at-once system from the initial data and the source:
 *   theta-method (eq. 2.4):  b_n = theta f(t_n) + (1-theta) f(t_{n-1}),
 *                            b_1 += (I/dt - (1-theta) K) u0;
 *   leap-frog (eq. 3.2b, ghost value U_{-1} = U_1 - 2 dt u1):
 *      b_1 = u0/dt^2 + u1/dt + (dt/2) K u1 + f(t_0)/2,
 *      b_2 = f(t_1) - u0/dt^2 - K u0/2,  b_n = f(t_{n-1}) for n >= 3.
 * u0: [S]; u1: [S] or NULL (zero; leap-frog only); f: [Nt+1][S] (values at
 * t_0..t_Nt) or NULL (zero source); b: [Nt][S].  All device FP64. */
PD_API pd_status pd_build_rhs(pd_plan* plan, const double* u0, const double* u1, const double* f,
                       double* b);

/* Solve A u = b.  mode PD_STATIONARY: the iteration of eq. 5.1,
 * u <- u + P_alpha^{-1}(b - A u); mode PD_GMRES: flexible GMRES(restart) on A
 * right-preconditioned by P_alpha^{-1} (the Krylov variant of Section 3),
 * FP64 Krylov vectors.  u holds the initial guess on entry and the solution
 * on exit (device FP64).  Stops when ||b - A u||_2 <= tol ||b||_2 or after maxit
 * preconditioner applications (PD_ERR_NOT_CONVERGED).  iters and relres may be
 * NULL.  Synchronises the plan's stream. */
PD_API pd_status pd_solve(pd_plan* plan, const double* b, double* u, int mode, double tol, int maxit,
                   int restart, int* iters, double* relres);

/* The stationary solve of pd_solve (mode PD_STATIONARY) without waiting for
 * it: on mixed plans the whole solve (entry split, the CUDA graph of the
 * iteration, exit) is enqueued on the plan's stream and the call returns at
 * once, so consecutive solves run back to back on the GPU; plans without a
 * graph (FP64) solve synchronously.  u must not be read, and b and u must not
 * be changed, before pd_solve_result returns.  No paper counterpart. */
PD_API pd_status pd_solve_async(pd_plan* plan, const double* b, double* u, double tol, int maxit);

/* Waits for the plan's queued asynchronous solves and returns the status,
 * iterations and relative residual of the last one (iters, relres may be
 * NULL); the launch counter adds the kernels of every queued solve, counted
 * as the last one's. */
PD_API pd_status pd_solve_result(pd_plan* plan, int* iters, double* relres);

/* The same solve with HOST buffers.  Mixed-precision stationary solves on
 * pinned (device-mapped) host buffers read b and the initial guess, and write
 * u, directly from the solver's entry and exit kernels over the host link;
 * otherwise b and the initial guess are copied to the device, the solve runs
 * and u is copied back (all on the plan's stream).  Returns when u_host holds
 * the result. */
PD_API pd_status pd_solve_host(pd_plan* plan, const double* b_host, double* u_host, int mode,
                        double tol, int maxit, int restart, int* iters, double* relres);

/* Windowing (Sections 2.1.1 and 2.2: long horizons as a sequence of time
 * windows, each solved by ParaDiag): nwin consecutive windows of the plan's
 * nt steps; window w starts from the last time level of window w-1 (u0 for
 * w = 0) and is solved by pd_solve from a zero initial guess.  u0: [S];
 * f: [nwin nt + 1][S] source values at t_0 .. t_{nwin nt}, or NULL for f = 0;
 * u: [nwin][nt][S] output (device FP64, caller-owned).  theta-method plans only
 * (leap-frog would need the velocity at every window start:
 * PD_ERR_UNSUPPORTED).  iters_total: iterations summed over the windows;
 * relres_max: the largest final relative residual (either may be NULL).  Stops
 * at the first window that fails, returning its status. */
PD_API pd_status pd_solve_windows(pd_plan* plan, const double* u0, const double* f, int nwin,
                                  double* u, int mode, double tol, int maxit, int restart,
                                  int* iters_total, double* relres_max);

/* Nonlinear problems U' + K U + phi(U) = f (Section 1, eq. 1.4 with M = I and
 * f(U) = K U + phi(U)) on a theta-method plan; phi(u) = a[0] u + a[1] u^2 +
 * a[2] u^3 acts pointwise.  a: 3 doubles in HOST memory (finite); every other
 * array is device FP64 in the time-major layout [Nt][S] (u0: [S], f: [Nt+1][S]
 * or NULL), caller-owned.  Leap-frog plans return PD_ERR_UNSUPPORTED.
 *
 * pd_nl_build_rhs: b of eq. 1.4, the linear right-hand side of
 * pd_build_rhs with -(1 - theta) phi(u0) added to the first row.
 *
 * pd_nl_residual: r = b - (B1 (x) I) u - (B2 (x) I) F(u), F(u)_n = K U_n +
 * phi(U_n), in FP64 on FP64 plans and in double-float (FP32 pairs, 48-bit
 * significand) on mixed plans.  sigma (host, may be NULL) receives the mean of phi'(U)
 * over all time levels and grid points, rnorm2 (host, may be NULL) ||r||^2;
 * asking for either synchronises the plan's stream.
 *
 * pd_nl_solve: the simplified Newton iteration of eq. 1.5 from the initial
 * guess in u (overwritten by the iterate): r as above, z = P_alpha(u)^{-1} r
 * with P_alpha(u) = C1 (x) I + C2 (x) (K + sigma I), sigma the mean of
 * phi'(U) (the averaged Jacobian), u += z; until ||r|| <= tol ||b|| or maxit
 * corrections.  The plan's preconditioner precision applies (FP32 on mixed
 * plans), and the residual is FP64 on FP64 plans, double-float on mixed plans
 * (the iterate then also lives in double-float inside the solve).  iters:
 * corrections applied; relres:
 * the last ||r|| / ||b|| (either may be NULL).  Returns PD_ERR_NOT_CONVERGED
 * after maxit corrections, PD_ERR_NONFINITE on a NaN or Inf (a diverging
 * iteration).  Allocates two [Nt][S] FP64 work arrays in the plan on first
 * use; synchronises the plan's stream once per correction; the plan's own
 * eigenvalue table is restored before it returns. */
PD_API pd_status pd_nl_build_rhs(pd_plan* plan, const double* a, const double* u0,
                                 const double* f, double* b);
PD_API pd_status pd_nl_residual(pd_plan* plan, const double* a, const double* b, const double* u,
                                double* r, double* sigma, double* rnorm2);
PD_API pd_status pd_nl_solve(pd_plan* plan, const double* a, const double* b, double* u,
                             double tol, int maxit, int* iters, double* relres);

/* Windowing with simplified Newton (Section 1): nwin consecutive windows of the
 * plan's nt steps, window w starting from the last time level of window w-1
 * (u0 for w = 0), each built by pd_nl_build_rhs and solved by pd_nl_solve from
 * a zero guess.  f: [nwin nt + 1][S] source values at t_0 .. t_{nwin nt}, or
 * NULL; u: [nwin][nt][S] output.  iters_total: corrections summed over the
 * windows; relres_max: the largest final relative residual (either may be
 * NULL).  Stops at the first window that fails and returns its status.  Short
 * windows keep the averaged-Jacobian iteration contracting where one long
 * window diverges. */
PD_API pd_status pd_nl_solve_windows(pd_plan* plan, const double* a, const double* u0,
                                     const double* f, int nwin, double* u, double tol,
                                     int maxit, int* iters_total, double* relres_max);

/* Solve A^T lambda = g (the transposed all-at-once system, backward in time).
 * Uses J A^T J = B1 (x) I + B2 (x) K^T (J = time reversal, B1, B2 Toeplitz):
 * a forward ParaDiag solve with K^T on time-reversed data.  lambda: initial
 * guess on entry (device FP64), solution on exit. */
PD_API pd_status pd_adjoint_solve(pd_plan* plan, const double* g, double* lam, int mode, double tol,
                           int maxit, int restart, int* iters, double* relres);

/* Time the kernels of one preconditioned iteration of the stationary solver
 * (residual + Gamma + FFT, x-transform forward, shifted tridiagonal solves,
 * x-transform inverse, inverse FFT + update) with CUDA events on the plan's
 * stream, averaged over reps >= 1 iterations started from the guess u with
 * right-hand side b (device FP64; u is not modified).  ms[0..4] receive the
 * average milliseconds per launch of these five kernels (0 where a kernel
 * does not occur).  Synchronises the plan's stream. */
PD_API pd_status pd_profile_iteration(pd_plan* plan, const double* b, const double* u, int reps,
                                      float* ms);

/* Measurement aid (no paper counterpart): reps applications of z = P^{-1} r
 * (pd_apply_precond), each kernel timed with CUDA events on the plan's
 * stream; ms[0..4] = forward time kernel (Gamma + FFT, FP64 input), forward
 * x-transform, tridiagonal solves, inverse x-transform, inverse time kernel
 * (IFFT + Gamma^{-1}, FP64 output); averages in milliseconds. */
PD_API pd_status pd_profile_precond(pd_plan* plan, const double* r, double* z, int reps,
                                    float* ms);

/* Number of kernels this plan (and its adjoint plan) has launched so far. */
PD_API pd_status pd_plan_launches(const pd_plan* plan, unsigned long long* count);

/* *uses = 1 if this plan's stationary solves run as one CUDA graph (mixed
 * precision: the whole iteration, convergence test included, is a graph
 * with a device-side WHILE loop; the first stationary solve builds it), else
 * 0 (FP64 plans, plans not yet solved, or a graph that could not be built:
 * the solver then loops on the host).  No paper counterpart; introspection. */
PD_API pd_status pd_plan_uses_graph(const pd_plan* plan, int* uses);

/* The kernel shapes of this plan: *tile_columns = spatial columns per block of
 * the time kernels, *tri_lanes = lanes per shifted tridiagonal system.  Mixed
 * plans with at least 2^18 unknowns choose them at creation by timing
 * candidates on the GPU (8 or 16 complex elements per thread for the time
 * kernels; for the tridiagonal solves the default lane count, twice it, and
 * the 16-rows-per-lane form; the x-transform engine, pd_plan_xform_engine);
 * others use the default rules.  No paper counterpart; introspection. */
PD_API pd_status pd_plan_tuning(const pd_plan* plan, int* tile_columns, int* tri_lanes);

/* The same shapes with the rows per lane that the tridiagonal solver keeps in
 * registers (*tri_rows: 32 or 16 on mixed plans, 16 on FP64 plans). */
PD_API pd_status pd_plan_get_tuning(const pd_plan* plan, int* tile_columns, int* tri_lanes,
                                    int* tri_rows);

/* Pin the kernel shapes of a mixed plan instead of the autotuner's choice:
 * tile_columns a power of two with 2 <= tile_columns <= 32 and tile_columns
 * times the transform length (Nt, or Bluestein's M) at most 8192 (plans whose
 * time tiles span a cluster, pd_plan_time_cluster, keep their width: only
 * the current tile_columns is accepted); tri_rows 32
 * or 16; tri_lanes a power of two at least the default for that row count
 * (ceil(n / tri_rows) rounded up to a power of two, n the tridiagonal
 * length) and at most 256.  Invalid shapes return PD_ERR_ARG and change
 * nothing; FP64 plans return PD_ERR_UNSUPPORTED.  Any CUDA graph the plan
 * holds is rebuilt at the next solve.  Every shape computes the same
 * preconditioner up to FP32 rounding.  No paper counterpart. */
PD_API pd_status pd_plan_set_tuning(pd_plan* plan, int tile_columns, int tri_lanes, int tri_rows);

/* Engines of the x-eigentransform of 2D (and periodic 1D) plans (step (b)'s
 * diagonalisation of K_x, Section 2.2's periodic 2D experiment):
 *   PD_XFORM_TENSOR  dense product with the eigenvector matrix on the tensor
 *                    cores (tcgen05, FP16 two-term split, FP32 accumulation);
 *                    mixed plans with nx >= 16 and >= 128 spectrum rows;
 *   PD_XFORM_FFT     FFT along x in the plan's precision: the DFT (periodic x)
 *                    or the sine transform through the odd extension
 *                    (Dirichlet x); a radix-16 Stockham FFT for powers of
 *                    two, one Cooley-Tukey step of two direct DFTs for
 *                    lengths L1 L2 with L1 <= L2 <= 32 (nx = 255 = 15 x 17),
 *                    Bluestein's form otherwise; transform lengths up to 1024;
 *   PD_XFORM_DENSE   dense product on the CUDA cores (the remaining cases).
 * Mixed plans with both of the first two and at least 2^18 unknowns pick the
 * faster at creation (timed on the GPU); otherwise the tensor cores where
 * available, else the FFT, else the dense form.  pd_plan_xform_engine: *engine
 * = the engine in use (-1: no x-transform).  pd_plan_set_xform_engine pins
 * PD_XFORM_TENSOR or PD_XFORM_FFT (PD_ERR_UNSUPPORTED where the plan lacks it,
 * PD_ERR_ARG for other values); it waits for the plan's stream, and any CUDA
 * graph the plan holds is rebuilt at the next solve.  No paper counterpart. */
#define PD_XFORM_TENSOR 0
#define PD_XFORM_FFT 1
#define PD_XFORM_DENSE 2
PD_API pd_status pd_plan_xform_engine(const pd_plan* plan, int* engine);
PD_API pd_status pd_plan_set_xform_engine(pd_plan* plan, int engine);

/* Blocks per time tile of the time kernels (steps (a) and (c) of eq. 1.3:
 * the FFT along t of TX spatial columns).  One block holds a tile of at most
 * 8192 (mixed) or 2048 (FP64) reals, N TX.  With *blocks = CR in {2, 4, 8}
 * a tile of CR times that is split over a thread-block cluster: block c forms
 * the time rows [c N/CR, (c+1) N/CR), one radix-CR step of the FFT exchanges
 * values through distributed shared memory, and each block finishes a
 * length-N/CR FFT and writes the spectrum rows k = CR k' + c (decimation in
 * frequency; the inverse runs the steps in reverse).  Power-of-two Nt only,
 * with 2 <= TX = CR budget / N <= 32.  Plans where one block's tile would be
 * narrower than 8 columns take the smallest CR giving 8 (the largest, 8,
 * beyond); mixed plans with at least 2^18 unknowns time the candidates at
 * creation with the tile widths of pd_plan_tuning.  pd_plan_set_time_cluster
 * pins CR (1, 2, 4 or 8; PD_ERR_UNSUPPORTED where the plan's Nt allows no
 * such tile, PD_ERR_ARG for other values) and sets TX to the budget's width;
 * it waits for the plan's stream, and any CUDA graph the plan holds is
 * rebuilt at the next solve.  Every CR computes the same transform up to
 * rounding.  No paper counterpart (the paper's FFT runs on one processor
 * per time step or sequentially). */
PD_API pd_status pd_plan_time_cluster(const pd_plan* plan, int* blocks);
PD_API pd_status pd_plan_set_time_cluster(pd_plan* plan, int blocks);

/* ---- batched solves: many independent problems of uneven size ----------
 * One problem of a batch (1D, Dirichlet, any scheme; all members of one batch
 * must share the time band: theta-method or leap-frog). */
typedef struct {
  pd_space space;
  int nt;
  double dt;
  double alpha;
  int scheme;
  double theta;
} pd_problem;

typedef struct pd_batch pd_batch;

/* Create a batch of nprob problems (1 <= nprob <= 4096).  Each problem gets
 * its own Lemma 1 tables and half spectrum; the iterate is packed.  Problem i
 * occupies elements [off_i, off_{i+1}) of the packed arrays, laid out
 * [Nt_i][nx_i] (see pd_batch_offsets).  The kernels of one iteration run as one
 * launch per kernel type over all problems (the tridiagonal solve: one launch
 * per class of system length), driven by per-problem descriptors and a
 * block-to-(problem, tile) work table in device memory.  Every member's time
 * tile must fit one block (pd_plan_time_cluster 1: Nt <= 4096 mixed, 2048
 * FP64 for powers of two; Bluestein lengths half that); a member beyond it
 * returns PD_ERR_UNSUPPORTED. */
PD_API pd_status pd_batch_create(const pd_problem* probs, int nprob, int precision, void* stream,
                                 pd_batch** out);
PD_API pd_status pd_batch_destroy(pd_batch* batch);
/* offsets[0..nprob]: element offsets of the problems in the packed arrays. */
PD_API pd_status pd_batch_offsets(const pd_batch* batch, unsigned long long* offsets);
/* Right-hand sides of all problems (pd_build_rhs per member): u0 packed with
 * problem i at sum_{j<i} nx_j; f packed ([Nt_i+1][nx_i] each) or NULL; b packed. */
PD_API pd_status pd_batch_build_rhs(pd_batch* batch, const double* u0, const double* f,
                                    double* b);
/* Stationary iteration (eq. 5.1) on all problems together until every
 * problem has ||b_i - A_i u_i|| <= tol ||b_i|| (relres_max receives the largest
 * relative residual) or maxit sweeps.  u: packed initial guess / solution. */
PD_API pd_status pd_batch_solve(pd_batch* batch, const double* b, double* u, double tol,
                                int maxit, int* iters, double* relres_max);
/* relres[0..nprob): relative residual of every problem at the last check. */
PD_API pd_status pd_batch_relres(const pd_batch* batch, double* relres);
PD_API pd_status pd_batch_launches(const pd_batch* batch, unsigned long long* count);

/* *uses = 1 if this batch's solves run as one CUDA graph (mixed precision:
 * the sweep loop with its convergence test is a graph with a device-side
 * WHILE loop; the first solve builds it), else 0.  No paper counterpart. */
PD_API pd_status pd_batch_uses_graph(const pd_batch* batch, int* uses);
PD_API const char* pd_batch_last_error(const pd_batch* batch);

/* *tuned = 1 when the batch's kernel shapes were chosen by timing at
 * creation (mixed batches of at least 2^18 unknowns: per group of members
 * with one transform length, the time-kernel tile width at the default or at
 * half of it; per group with one default tridiagonal lane class, that lane
 * count or twice it), else 0.  No paper counterpart; introspection. */
PD_API pd_status pd_batch_tuned(const pd_batch* batch, int* tuned);

/* Per-kernel timing of one sweep of the batched iteration on the batch's
 * stream (CUDA events, `reps` launches each after one warm-up): ms[0] the
 * forward time kernels (residual, Gamma, FFT) over all members, ms[1] the
 * tridiagonal solves, ms[2] the inverse time kernels with the update.  b and
 * u as for pd_batch_solve; u is overwritten by iterates that carry no
 * meaning.  No paper counterpart; measurement. */
PD_API pd_status pd_batch_profile_sweep(pd_batch* batch, const double* b, double* u, int reps,
                                        float* ms);

/* ---- the preconditioner in parts, for a solve spread over several GPUs ----
 * Steps (a) and (c) of eq. 1.3 act on every spatial point independently and
 * step (b) on every time frequency k independently (the discussion after
 * Lemma 1: the Nt shifted systems are "completely independent"), so a
 * distributed solve gives each rank a slab of grid lines for the residual and
 * the time transforms, and a slab of frequencies for step (b), with an
 * all-to-all transpose of the spectrum between them (the caller's: the
 * Python binding does it with torch.distributed).  A rank's slab plan is an
 * ordinary plan for its lines plus one halo line on each side (grid spacing
 * kept by scaling ly, or lx in 1D); the frequency-slab solves use a plan of
 * the whole grid.  2D problems slab y, 1D Dirichlet problems slab x; 1D
 * periodic plans return PD_ERR_UNSUPPORTED.  All arrays are device memory;
 * work goes on the plan's stream.  No paper counterpart for the split. */

/* Step (a) of P_alpha^{-1} r: Gamma scaling and FFT along t, then (2D) the
 * forward x-eigentransform.  r: [Nt][S] FP64.  The result is the plan's
 * step-(b) spectrum (pd_plan_spectrum). */
PD_API pd_status pd_precond_forward(pd_plan* plan, const double* r);

/* The step-(b) spectrum of the plan: *data -> complex [nh][lines][pitch]
 * (FP32 pairs on mixed plans, FP64 pairs on FP64 plans: *elem_bytes 8 or
 * 16), nh = Nt/2 + 1 frequencies, lines = ny (2D) or nx (1D), pitch = the
 * padded nx (2D) or 1 (1D). */
PD_API pd_status pd_plan_spectrum(pd_plan* plan, void** data, int* nh, int* lines, int* pitch,
                                  int* elem_bytes);

/* Copy the block k0 <= k < k1, l0 <= line < l1 of the plan's step-(b)
 * spectrum to (get) or from (put) a contiguous device buffer laid out
 * [k1-k0][l1-l0][pitch]; put with src NULL writes zeros. */
PD_API pd_status pd_spectrum_get(pd_plan* plan, int k0, int k1, int l0, int l1, void* dst);
PD_API pd_status pd_spectrum_put(pd_plan* plan, int k0, int k1, int l0, int l1, const void* src);

/* Step (b) for the frequencies k0 <= k < k1 on a caller-owned slab laid out
 * like the plan's spectrum with k1 - k0 frequencies ([k1-k0][lines][pitch]),
 * in place: the shifted systems (lambda_1k I + lambda_2k K) z = s of eq. 1.3
 * (2D: after the x-eigentransform, tridiagonal in y). */
PD_API pd_status pd_precond_solve_rows(pd_plan* plan, int k0, int k1, void* data);

/* Step (c): (2D) the inverse x-eigentransform of the plan's step-(b)
 * spectrum, the inverse FFT along t and Gamma^{-1}: z [Nt][S] FP64. */
PD_API pd_status pd_precond_backward(pd_plan* plan, double* z);

/* *out (host) = sum over time levels and the grid lines first_line ..
 * first_line + nlines - 1 of x^2 (x: [Nt][S]); synchronises the stream. */
PD_API pd_status pd_shard_norm2(pd_plan* plan, const double* x, int first_line, int nlines,
                                double* out);

/* u += z on the grid lines first_line .. first_line + nlines - 1 of every
 * time level (u, z: [Nt][S]). */
PD_API pd_status pd_shard_update(pd_plan* plan, const double* z, double* u, int first_line,
                                 int nlines);

/* Size of the device array used by pd_apply_precond_noalloc (8 MiB). */
#define PD_NOALLOC_SCRATCH_BYTES (8u << 20)

/* z = P_alpha^{-1} r for a 1D Dirichlet problem (sp->dim == 1, bc_x Dirichlet),
 * mixed precision, WITHOUT any device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc -- code running while an application's memory pool is frozen,
 * plug-ins whose host application owns every device allocation, or code in a
 * region where allocation is not allowed.  Such callers cannot create a plan
 * (pd_plan_create allocates its tables and workspace).
 *   Sizes.    Nt a power of two, 1 <= Nt <= 4096, and 1 <= nx <= 4096 (one
 *             block per time tile: the one-block limits of the plan path's
 *             mixed-precision kernels); other sizes return PD_ERR_UNSUPPORTED.  alpha = 1 is rejected with
 *             PD_ERR_ARG when a shifted system is singular (as pd_plan_create).
 *   Scratch.  The half spectrum and the eigenvalue, Gamma and twiddle tables
 *             live in one file-scope __device__ array of
 *             PD_NOALLOC_SCRATCH_BYTES that every GPU loading this library
 *             holds until the process exits.  Problems needing more (about
 *             8 (Nt/2+1) nx bytes plus small tables) are rejected with
 *             PD_ERR_ARG; *scratch_needed (if not NULL) receives the bytes the
 *             problem needs whenever the sizes are supported.
 *   Set-up.   The first call on a device looks up the array's device address
 *             (cudaGetSymbolAddress) with that device current; make that first
 *             call before any stream capture.
 *   Sharing.  All calls share the one array and leave their data in it; calls
 *             whose work overlaps on the GPU (other streams or host threads)
 *             race and must be serialised by the caller.
 *   Status.   The tables are copied from host memory onto the stream, the
 *             kernels enqueued, and a status word read back: the call returns
 *             after its work has finished, with PD_ERR_NONFINITE when r, the
 *             spectrum or z held a non-finite value.
 * r, z: [Nt][nx] device FP64 (caller-owned); stream: cudaStream_t. */
PD_API pd_status pd_apply_precond_noalloc(const pd_space* sp, int nt, double dt, double alpha,
                                          int scheme, double theta, const double* r, double* z,
                                          void* stream, unsigned long long* scratch_needed);

/* ---------------------------------------------------------------------------
 * ParaDiag-I with geometrically increasing time steps (Section 2.1.1): a
 * direct solver of the theta-method all-at-once system eq. 2.5a,
 *   (B1 (x) I + B2 (x) K) u = b,
 * B1, B2 the lower-bidiagonal matrices of eq. 2.5b for the steps of eq. 2.8,
 *   dt_n = dt_last * tau^(n - nt), n = 1..nt,
 * by the three steps of eq. 2.7 with the closed-form eigenvector matrix V of
 * B2^{-1} B1 (theorem of Section 2.1.1; for theta = 1/2 the printed factor
 * q^{-n} of q_n is read as tau^{-n}, the reading that makes V V^{-1} = I).
 * Layout of u and b as for pd_plan: [nt][S] device FP64, caller-owned.
 * --------------------------------------------------------------------------- */
typedef struct pd1_plan pd1_plan;

/* Plan for one window.  scheme: PD_BE (theta = 1) or PD_CN (theta = 1/2,
 * the trapezoidal rule); column_scaling: 1 uses V D~ with
 * D~ = diag((1 + sum_{j<=nt-n} p_j^2)^{-1/2}) (Section 2.1.1), 0 uses V.
 * precision PD_FP64: steps (a)-(c) and the residual in FP64; PD_MIXED: steps
 * (a)-(c) in FP32 (the tensor-core x-transform in 2D) and the residual of the
 * refinement sweeps in double-float.  sp: as for pd_plan_create (2D: x
 * Dirichlet needs ax = 0, y Dirichlet).  1 <= nt <= 32 (PD_ERR_UNSUPPORTED
 * above: the windows of Section 2.1.1 hold 20 to 32 steps, and Cond_2(V)
 * passes 1e9 beyond), dt_last > 0, tau > 1.  stream: cudaStream_t (NULL: the
 * default stream).  Allocates all device memory the solves need. */
PD_API pd_status pd1_plan_create(const pd_space* sp, int nt, double dt_last, double tau,
                                 int scheme, int column_scaling, int precision, void* stream,
                                 pd1_plan** out);
PD_API pd_status pd1_plan_destroy(pd1_plan* plan);

/* dts[0..nt): the step sizes dt_1..dt_nt of eq. 2.8 (host array). */
PD_API pd_status pd1_step_sizes(const pd1_plan* plan, double* dts);

/* *cond: ||V D~||_F ||(V D~)^{-1}||_F (an upper bound of Cond_2 of the
 * eigenvector matrix the plan uses; the roundoff of the direct solve grows
 * with it). */
PD_API pd_status pd1_condition(const pd1_plan* plan, double* cond);

/* y = A u (eq. 2.5a), FP64. */
PD_API pd_status pd1_apply_A(pd1_plan* plan, const double* u, double* y);

/* b of eq. 2.5a: b_n = theta f(t_n) + (1-theta) f(t_{n-1}), plus
 * (I/dt_1 - (1-theta) K) u0 in the first row.  u0: [S]; f: [nt+1][S] values
 * at t_0..t_nt, or NULL for f = 0; b: [nt][S]. */
PD_API pd_status pd1_build_rhs(pd1_plan* plan, const double* u0, const double* f, double* b);

/* u = A^{-1} b: the direct solve of eq. 2.7 (u on entry is ignored), then up
 * to max_refine sweeps u <- u + P^{-1}(b - A u) with the same solve P^{-1}
 * (residual in FP64 / double-float), stopping early once
 * ||b - A u||_2 <= tol ||b||_2.  max_refine = 0 is the paper's direct solver.
 * relres (may be NULL) receives ||b - A u||_2 / ||b||_2 of the returned u;
 * it costs one residual pass, skipped when relres is NULL and max_refine = 0.
 * refinements (may be NULL) receives the sweeps taken.  Returns
 * PD_ERR_NOT_CONVERGED when max_refine > 0, tol > 0 and the tolerance was not
 * reached, PD_ERR_NONFINITE on a NaN or Inf.  Synchronises the plan's stream
 * when a residual is formed. */
PD_API pd_status pd1_solve(pd1_plan* plan, const double* b, double* u, double tol,
                           int max_refine, int* refinements, double* relres);

/* Windowing (Section 2.1.1: the windows of 20-30 steps that keep ParaDiag-I's
 * roundoff bounded): nwin consecutive windows, each with the plan's geometric
 * steps; window w starts from the last time level of window w-1 (u0 for
 * w = 0) and is solved by pd1_solve.  f: [nwin nt + 1][S] values at the time
 * points of all windows, or NULL; u: [nwin][nt][S] output.  refinements_total
 * and relres_max as for pd_solve_windows. */
PD_API pd_status pd1_solve_windows(pd1_plan* plan, const double* u0, const double* f, int nwin,
                                   double* u, double tol, int max_refine, int* refinements_total,
                                   double* relres_max);

/* Measurement aid (no paper counterpart): from the direct solve of b, reps
 * refinement sweeps, each timed with CUDA events on the plan's stream;
 * ms[0] = step (a) fused with the residual, ms[1] = step (b) (with the
 * x-eigentransforms in 2D), ms[2] = step (c) fused with the update, averages
 * in milliseconds.  u receives the last iterate. */
PD_API pd_status pd1_profile_sweep(pd1_plan* plan, const double* b, double* u, int reps,
                                   float* ms);

/* Kernel launches made through the plan so far; device bytes it holds. */
PD_API pd_status pd1_launches(const pd1_plan* plan, unsigned long long* count);
PD_API pd_status pd1_workspace(const pd1_plan* plan, unsigned long long* bytes);
PD_API const char* pd1_last_error(const pd1_plan* plan);

/* ---------------------------------------------------------------------------
 * ParaDiag-I with the hybrid time discretisation (Section 2.1.2): explicit
 * midpoint steps n = 1..nt-1 and one backward-Euler step at the end, uniform
 * step dt (eq. neq2.9a).  All-at-once system (eq. neq2.9b, neq2.9c):
 *   (B (x) I + I (x) K) u = b,  B = (1/dt) tridiag(-1/2, 0, 1/2), last row
 *   (..., -1, 1),
 * diagonalised by the theorem of Section 2.1.2: eigenvalues i x_n / dt (the
 * printed i dt x_n read with B's 1/dt factor), x_n the roots of
 * P2_{nt-1}(x) - i P1_{nt}(x), eigenvectors v_{n,l} = i^l P2_l(x_n).
 * Layout of u and b as for pd_plan: [nt][S] device FP64, caller-owned.
 * --------------------------------------------------------------------------- */
typedef struct pdh_plan pdh_plan;

/* Plan for nt uniform steps of size dt (1 <= nt <= 4096; PD_ERR_UNSUPPORTED
 * above).  precision PD_FP64: steps (a)-(c) and the residual in FP64;
 * PD_MIXED: steps (a)-(c) at FP32 level (the tensor-core x-transform in 2D),
 * the residual of the refinement sweeps in double-float.  On mixed first-order
 * plans with nt a multiple of 16, 32 <= nt, and at least 128 spatial points, the
 * dense time contractions of steps (a) and (c) (the real forms of V^{-1} and V)
 * run on the tensor cores as GEMMs over the spatial points, with FP16 operands
 * split in two terms and FP32 accumulation (pdh_set_tensor_cores); otherwise
 * on the CUDA cores.  sp: as for pd_plan_create.  stream: cudaStream_t (NULL:
 * the default stream).  Finds the eigenvalues and the eigenvector matrices on
 * the host (O(nt^2) work) and allocates all device memory the solves need. */
PD_API pd_status pdh_plan_create(const pd_space* sp, int nt, double dt, int precision,
                                 void* stream, pdh_plan** out);
PD_API pd_status pdh_plan_destroy(pdh_plan* plan);

/* Second-order problems U'' + K U = f, U(0) = u0, U'(0) = v0 (eq. neq2.14a):
 * the hybrid scheme applied to the first-order form with the velocity
 * eliminated, (B^2 (x) I + I (x) K) u = F_v + B F_u (B_2nd = B^2, eq. neq2.15),
 * solved with the same eigenvectors and the eigenvalues (i x_n / dt)^2.  The
 * plan works with pdh_solve, pdh_apply_A (then B^2), pdh_eigenvalues (the
 * eigenvalues of B) and pdh_wave_build_rhs; arguments as pdh_plan_create. */
PD_API pd_status pdh_wave_plan_create(const pd_space* sp, int nt, double dt, int precision,
                                      void* stream, pdh_plan** out);

/* b = F_v + B F_u: b_n = f(t_n) + v0/(2 dt) [n = 1] + (B)_{n,1} u0/(2 dt)
 * (rows n = 1..nt); u0, v0: [S]; f: [nt+1][S] values at t_0..t_nt or NULL. */
PD_API pd_status pdh_wave_build_rhs(pdh_plan* plan, const double* u0, const double* v0,
                                    const double* f, double* b);

/* lam[2n], lam[2n+1]: real and imaginary part of the eigenvalue i x_n / dt of
 * B, n = 0..nt-1 (host array of 2 nt doubles). */
PD_API pd_status pdh_eigenvalues(const pdh_plan* plan, double* lam);

/* *cond: ||V||_F ||V^{-1}||_F for the eigenvector matrix the plan uses. */
PD_API pd_status pdh_condition(const pdh_plan* plan, double* cond);

/* y = A u (eq. neq2.9b), FP64. */
PD_API pd_status pdh_apply_A(pdh_plan* plan, const double* u, double* y);

/* b_n = f(t_n), n = 1..nt, plus u0 / (2 dt) in the first row (eq. neq2.9c).
 * u0: [S]; f: [nt+1][S] values at t_0..t_nt, or NULL for f = 0. */
PD_API pd_status pdh_build_rhs(pdh_plan* plan, const double* u0, const double* f, double* b);

/* u = A^{-1} b: the direct solve of eq. 2.7 with the eigendecomposition above
 * (u on entry is ignored), then up to max_refine sweeps
 * u <- u + P^{-1}(b - A u), stopping early once ||b - A u||_2 <= tol ||b||_2.
 * Arguments, return values and synchronisation as for pd1_solve. */
PD_API pd_status pdh_solve(pdh_plan* plan, const double* b, double* u, double tol,
                           int max_refine, int* refinements, double* relres);

/* Measurement aid (no paper counterpart): from the direct solve of b, reps
 * refinement sweeps timed with CUDA events on the plan's stream; ms[0] = the
 * residual, ms[1] = step (a) (dense time transform), ms[2] = step (b),
 * ms[3] = step (c) with the update (averages in milliseconds). */
PD_API pd_status pdh_profile_sweep(pdh_plan* plan, const double* b, double* u, int reps,
                                   float* ms);
PD_API pd_status pdh_launches(const pdh_plan* plan, unsigned long long* count);
PD_API const char* pdh_last_error(const pdh_plan* plan);

/* Engine of the time contractions of steps (a) and (c): on = 1 the tcgen05
 * GEMMs (the default where the plan allows them), on = 0 the CUDA-core GEMMs.
 * on = 1 on a plan that does not allow them (FP64, second-order, nt not a
 * multiple of 16 or below 32, fewer than 128 spatial points): PD_ERR_UNSUPPORTED.
 * Waits for the plan's stream.  pdh_tensor_cores: *on = the engine in use. */
PD_API pd_status pdh_set_tensor_cores(pdh_plan* plan, int on);
PD_API pd_status pdh_tensor_cores(const pdh_plan* plan, int* on);

/* ---------------------------------------------------------------------------
 * ParaDiag-II for the optimal control of the wave equation (Section 4): the
 * saddle-point all-at-once system of the implicit leap-frog scheme (state u,
 * adjoint p), scaled by dt^2 as in the section,
 *   A^ = [[T1, -dt^2 Ih / gamma], [dt^2 Ic, T1^T]] (x) I + blockdiag(T2, T2^T) (x) K,
 * T1 = lower Toeplitz (1, -2, 1), T2 = lower Toeplitz (1, 0, 1) dt^2/2 (dt^2
 * times B1, B2 of eq. 3.2b), Ih = diag(1/2, 1, ..., 1), Ic = diag(1, ..., 1, 1/2),
 * K the spatial operator of sp (the negative Laplacian for nu = 1, no
 * advection).  Solved by flexible GMRES on the gamma-balanced system
 * (unknowns (gamma^{1/2} u, p)) with the block circulant preconditioner P of
 * the section, applied through Theorem 4 (per frequency a 2 x 2 block with
 * orthogonal eigenvectors: Cond_2(V) = 1).  Vectors are [2][nt][S] device FP64:
 * the state field, then the adjoint field.
 * --------------------------------------------------------------------------- */
typedef struct pdc_plan pdc_plan;

/* Plan for nt steps of dt = T/nt (nt >= 3; nt divisible by 4 makes the
 * circulant of T2 singular: PD_ERR_UNSUPPORTED) and regularisation gamma > 0.
 * precision PD_FP64: the preconditioner in FP64; PD_MIXED: in FP32 (the
 * tensor-core x-transform in 2D); the Krylov vectors and A are FP64 in both. */
PD_API pd_status pdc_plan_create(const pd_space* sp, int nt, double T, double gamma,
                                 int precision, void* stream, pdc_plan** out);
PD_API pd_status pdc_plan_destroy(pdc_plan* plan);

/* y = A x for the balanced system A = S A^ S^{-1}, S = diag(gamma^{1/2} I, I). */
PD_API pd_status pdc_apply_A(pdc_plan* plan, const double* x, double* y);

/* z = P^{-1} r (the balanced preconditioner, Theorem 4). */
PD_API pd_status pdc_apply_precond(pdc_plan* plan, const double* r, double* z);

/* Solve A^ (u, p) = (f, g): FGMRES(restart) on the balanced system from a zero
 * guess, stopping when the balanced relative residual is <= tol or after maxit
 * iterations (PD_ERR_NOT_CONVERGED, x still written).  b = (f, g), x = (u, p);
 * restart in [0, 64] (0: 30). */
PD_API pd_status pdc_solve(pdc_plan* plan, const double* b, double* x, double tol, int maxit,
                           int restart, int* iters, double* relres);

/* The same solve with left preconditioning: GMRES(restart) on
 * P^{-1} A x = P^{-1} b from a zero guess, stopping when the preconditioned
 * relative residual ||P^{-1}(b - A x)|| / ||P^{-1} b|| is <= tol (relres
 * receives that ratio).  With this stopping test the iteration counts of
 * Table T2A are reproduced on the (16,16,17) to (64,64,65) meshes.
 * Arguments as pdc_solve. */
PD_API pd_status pdc_solve_left(pdc_plan* plan, const double* b, double* x, double tol,
                                int maxit, int restart, int* iters, double* relres);
PD_API pd_status pdc_launches(const pdc_plan* plan, unsigned long long* count);
PD_API const char* pdc_last_error(const pdc_plan* plan);

PD_API const char* pd_status_string(pd_status s);
PD_API const char* pd_last_error(const pd_plan* plan);

#ifdef __cplusplus
}
#endif
#endif /* PARADIAG_H */
