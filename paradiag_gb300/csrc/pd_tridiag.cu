// Step (b) of eq. 1.3: the Nt independent complex-shifted spatial solves
// (lambda_1 I + lambda_2 K) z = s, here for the constant-coefficient
// tridiagonal K of one direction (1D problems, or y after the x-eigentransform
// of 2D problems, where the shift also carries the x-eigenvalue mu_j).
//
// Partitioned solver, no pivoting.  W warps cooperate on one system of length
// n; lane G (0 <= G < 32W) owns the m = max(2, ceil(n/32W)) <= 8 consecutive
// rows i0 = G m .. i0+m-1.  Each lane eliminates its interior rows in
// registers, expressing them as z_i = Y_i + P_i f_G + Q_i g_G in terms of its
// first (f_G) and last (g_G) unknown; the first and last rows then form a
// tridiagonal reduced system of 64W unknowns (f_0, g_0, f_1, g_1, ...), solved
// by parallel cyclic reduction in shared memory.  Rows are scaled by 1/d so
// the diagonal is one; padding rows (i >= n) are identity rows with z = 0.
#include <cstring>

#include "pd_internal.h"

namespace {

constexpr int MMAX = 8;

template <typename C>
struct Row4 { C a, b, c, d; };

template <typename C>
PD_D C shfl_up_c(C v, int d) {
  v.x = __shfl_up_sync(0xffffffffu, v.x, d);
  v.y = __shfl_up_sync(0xffffffffu, v.y, d);
  return v;
}
template <typename C>
PD_D C shfl_down_c(C v, int d) {
  v.x = __shfl_down_sync(0xffffffffu, v.x, d);
  v.y = __shfl_down_sync(0xffffffffu, v.y, d);
  return v;
}
template <typename C>
PD_D Row4<C> shfl_up_r(const Row4<C>& r, int d) {
  Row4<C> o;
  o.a = shfl_up_c(r.a, d); o.b = shfl_up_c(r.b, d); o.c = shfl_up_c(r.c, d); o.d = shfl_up_c(r.d, d);
  return o;
}
template <typename C>
PD_D Row4<C> shfl_down_r(const Row4<C>& r, int d) {
  Row4<C> o;
  o.a = shfl_down_c(r.a, d); o.b = shfl_down_c(r.b, d); o.c = shfl_down_c(r.c, d);
  o.d = shfl_down_c(r.d, d);
  return o;
}

// one PCR elimination of row x with its neighbours at distance s (absent
// neighbours lie outside the system and contribute nothing)
template <typename C>
PD_D Row4<C> pcr_step(const Row4<C>& x, const Row4<C>& m, bool hm, const Row4<C>& p, bool hp) {
  Row4<C> o;
  o.a = czero<C>(); o.c = czero<C>(); o.b = x.b; o.d = x.d;
  if (hm) {
    const C k1 = cmul(x.a, crcp(m.b));
    o.a = mk(-(m.a.x * k1.x - m.a.y * k1.y), -(m.a.x * k1.y + m.a.y * k1.x));
    o.b = csub(o.b, cmul(m.c, k1));
    o.d = csub(o.d, cmul(m.d, k1));
  }
  if (hp) {
    const C k2 = cmul(x.c, crcp(p.b));
    o.c = mk(-(p.c.x * k2.x - p.c.y * k2.y), -(p.c.x * k2.y + p.c.y * k2.x));
    o.b = csub(o.b, cmul(p.a, k2));
    o.d = csub(o.d, cmul(p.d, k2));
  }
  return o;
}

// element i of system q (q = k*J + j) in global memory
template <typename C>
PD_D C* sys_elem(const TriArgs& a, C* data, long long q, int i) {
  const long long k = q / a.J, j = q % a.J;
  return data + k * a.S + j + (long long)i * a.stride;
}

// Shared tile layout: system sb, row i at sb * rows_pad + i + i / m (chunks of
// m rows padded to m + 1).  i / m by a 16-bit reciprocal cm = ceil(2^16 / m),
// exact for m <= 8 and i < 8192.
PD_D int tile_slot(int i, unsigned cm) { return i + (int)(((unsigned)i * cm) >> 16); }

template <typename C, bool ASYNC>
PD_D void put_elem(C* dst, const C* src);

// Copy the SB systems q0 .. q0+SB-1 between global memory and the shared tile
// (IN: global -> shared, zeros for systems past the end; OUT: shared -> global).
// Contiguous 1D systems are copied as one run (e -> (system, row) by an exact
// 32-bit reciprocal of n); strided systems give each thread one system and a
// fixed row step (blockDim.x is a multiple of SB).
template <typename C, bool IN, bool ASYNC>
PD_D void tile_copy(const TriArgs& a, C* tile, int rows_pad, int m, long long q0, int SB) {
  C* data = reinterpret_cast<C*>(a.data);
  const int n = a.n;
  const long long total = (long long)a.nh * a.J;
  const unsigned cm = (65536u + (unsigned)m - 1u) / (unsigned)m;
  if (a.stride == 1 && a.J == 1 && a.S == n) {
    const int nsys = (int)min((long long)SB, total - q0);
    const int nel = SB * n;
    C* g = data + q0 * n;
    const unsigned mn = n > 1 ? (unsigned)((0x100000000ull + (unsigned long long)n - 1) / (unsigned long long)n) : 0u;
    for (int e = threadIdx.x; e < nel; e += blockDim.x) {
      const int sb = n > 1 ? (int)__umulhi((unsigned)e, mn) : e;
      const int i = e - sb * n;
      C* t = tile + (size_t)sb * rows_pad + tile_slot(i, cm);
      if (IN) {
        if (sb < nsys) put_elem<C, ASYNC>(t, g + e);
        else *t = czero<C>();
      } else if (sb < nsys) {
        g[e] = *t;
      }
    }
  } else {
    const int sb = threadIdx.x % SB;
    const long long q = q0 + sb;
    const bool ok = q < total;
    C* g = ok ? data + (q / a.J) * a.S + (q % a.J) : data;
    const int step = blockDim.x / SB;
    C* t0 = tile + (size_t)sb * rows_pad;
    for (int i = threadIdx.x / SB; i < n; i += step) {
      C* t = t0 + tile_slot(i, cm);
      if (IN) {
        if (ok) put_elem<C, ASYNC>(t, g + (long long)i * a.stride);
        else *t = czero<C>();
      } else if (ok) {
        g[(long long)i * a.stride] = *t;
      }
    }
  }
}

// Solve the SB systems q0 .. q0+SB-1 held in the padded shared tile (one
// system per 32W threads); the solutions overwrite the tile.  pa..pd: PCR
// scratch (W > 1 only).
template <typename R, int W>
PD_D void solve_tile(const TriArgs& a, int m, int SB, cplx_t<R>* tile, cplx_t<R>* pa,
                     cplx_t<R>* pb, cplx_t<R>* pc, cplx_t<R>* pd, long long q0) {
  using C = cplx_t<R>;
  const int rows_pad = 32 * W * (m + 1);
  const int R2 = 64 * W;
  const int n = a.n, J = a.J;
  const long long total = (long long)a.nh * J;
  const int sb = threadIdx.x / (32 * W);
  const int G = threadIdx.x % (32 * W);
  const long long q = q0 + sb;
  const bool active = q < total;

  // ---- system coefficients, normalised by the diagonal
  C ld = czero<C>(), ud = czero<C>(), invd = mk((R)1, (R)0);
  if (active) {
    const long long k = q / J, j = q % J;
    const C* lam = reinterpret_cast<const C*>(a.lam);
    const C l1 = lam[2 * k], l2 = lam[2 * k + 1];
    C mu = czero<C>();
    if (a.mu != nullptr) mu = reinterpret_cast<const C*>(a.mu)[j];
    const C l = cscale(l2, (R)a.cl);
    const C u = cscale(l2, (R)a.cu);
    const C d = cadd(l1, cmul(l2, cadd(mk((R)a.cd, (R)0), mu)));
    invd = crcp(d);
    ld = cmul(l, invd);
    ud = cmul(u, invd);
  }

  // ---- lane rows: right-hand sides scaled by 1/d; the coefficients of row i
  // are (ld, 1, ud) except at the ends (no z_{-1}, no z_n) and on padding rows
  C rhs[MMAX];
  const int i0 = G * m;
  C* my = tile + (size_t)sb * rows_pad + G * (m + 1);
#pragma unroll
  for (int t = 0; t < MMAX; ++t)
    if (t < m) rhs[t] = (i0 + t < n) ? cmul(my[t], invd) : czero<C>();
  auto lrow = [&](int t) -> C { const int i = i0 + t; return (i > 0 && i < n) ? ld : czero<C>(); };
  auto urow = [&](int t) -> C { const int i = i0 + t; return (i < n - 1) ? ud : czero<C>(); };

  // ---- interior elimination (rows 1..m-2 of the chunk)
  const int mi = m - 2;
  C cc[MMAX], Y[MMAX], P[MMAX], Q[MMAX];
#pragma unroll
  for (int t = 0; t < MMAX; ++t) { cc[t] = czero<C>(); Y[t] = P[t] = Q[t] = czero<C>(); }
#pragma unroll
  for (int t = 1; t < MMAX - 1; ++t) {
    if (t <= mi) {
      const C lt = lrow(t);
      const C den = csub(mk((R)1, (R)0), cmul(lt, cc[t - 1]));
      const C iden = crcp(den);
      cc[t] = cmul(urow(t), iden);
      Y[t] = cmul(csub(rhs[t], cmul(lt, Y[t - 1])), iden);
      const C pr = (t == 1) ? mk(-lt.x, -lt.y) : czero<C>();
      P[t] = cmul(csub(pr, cmul(lt, P[t - 1])), iden);
      const C ut = urow(t);
      const C qr = (t == mi) ? mk(-ut.x, -ut.y) : czero<C>();
      Q[t] = cmul(csub(qr, cmul(lt, Q[t - 1])), iden);
    }
  }
#pragma unroll
  for (int t = MMAX - 2; t >= 1; --t) {
    if (t < mi) {
      Y[t] = csub(Y[t], cmul(cc[t], Y[t + 1]));
      P[t] = csub(P[t], cmul(cc[t], P[t + 1]));
      Q[t] = csub(Q[t], cmul(cc[t], Q[t + 1]));
    }
  }

  // ---- reduced rows (f_G at 2G, g_G at 2G+1)
  Row4<C> rf, rg;
  const C one = mk((R)1, (R)0);
  const C u0 = urow(0), lm = lrow(m - 1), um = urow(m - 1);
  C rm = czero<C>();
#pragma unroll
  for (int t = 1; t < MMAX; ++t)
    if (t == m - 1) rm = rhs[t];
  if (mi >= 1) {
    C Y1 = Y[1], P1 = P[1], Q1 = Q[1], Ym = czero<C>(), Pm = czero<C>(), Qm = czero<C>();
#pragma unroll
    for (int t = 1; t < MMAX - 1; ++t)
      if (t == mi) { Ym = Y[t]; Pm = P[t]; Qm = Q[t]; }
    rf.a = lrow(0);
    rf.b = cadd(one, cmul(u0, P1));
    rf.c = cmul(u0, Q1);
    rf.d = csub(rhs[0], cmul(u0, Y1));
    rg.a = cmul(lm, Pm);
    rg.b = cadd(one, cmul(lm, Qm));
    rg.c = um;
    rg.d = csub(rm, cmul(lm, Ym));
  } else {
    rf.a = lrow(0); rf.b = one; rf.c = u0; rf.d = rhs[0];
    rg.a = lm; rg.b = one; rg.c = um; rg.d = rm;
  }

  // ---- PCR on the reduced system (64W rows per system)
  C f, g;
  if constexpr (W == 1) {
    // one warp per system: lane G holds rows 2G (f) and 2G+1 (g); the
    // neighbours come from warp shuffles, no shared memory or block barrier
    for (int s = 1; s < 64; s <<= 1) {
      Row4<C> mf, pf, mg, pg;
      bool hmf, hpf, hmg, hpg;
      if (s == 1) {
        const Row4<C> gm = shfl_up_r(rg, 1);    // row 2G-1
        const Row4<C> fp = shfl_down_r(rf, 1);  // row 2G+2
        mf = gm; hmf = G > 0;  pf = rg; hpf = true;
        mg = rf; hmg = true;   pg = fp; hpg = G < 31;
      } else {
        const int d = s >> 1;
        mf = shfl_up_r(rf, d); mg = shfl_up_r(rg, d);
        pf = shfl_down_r(rf, d); pg = shfl_down_r(rg, d);
        hmf = hmg = G >= d;
        hpf = hpg = G + d < 32;
      }
      const Row4<C> nf = pcr_step(rf, mf, hmf, pf, hpf);
      const Row4<C> ng = pcr_step(rg, mg, hmg, pg, hpg);
      rf = nf;
      rg = ng;
    }
    f = cmul(rf.d, crcp(rf.b));
    g = cmul(rg.d, crcp(rg.b));
  } else {
    C* A_ = pa + (size_t)sb * R2;
    C* B_ = pb + (size_t)sb * R2;
    C* C_ = pc + (size_t)sb * R2;
    C* D_ = pd + (size_t)sb * R2;
    const int rf_i = 2 * G, rg_i = 2 * G + 1;
    A_[rf_i] = rf.a; B_[rf_i] = rf.b; C_[rf_i] = rf.c; D_[rf_i] = rf.d;
    A_[rg_i] = rg.a; B_[rg_i] = rg.b; C_[rg_i] = rg.c; D_[rg_i] = rg.d;
    __syncthreads();
    for (int s = 1; s < R2; s <<= 1) {
      Row4<C> nw[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * G + h;
        const int im = i - s, ip = i + s;
        Row4<C> x, m, p;
        x.a = A_[i]; x.b = B_[i]; x.c = C_[i]; x.d = D_[i];
        m = x; p = x;
        if (im >= 0) { m.a = A_[im]; m.b = B_[im]; m.c = C_[im]; m.d = D_[im]; }
        if (ip < R2) { p.a = A_[ip]; p.b = B_[ip]; p.c = C_[ip]; p.d = D_[ip]; }
        nw[h] = pcr_step(x, m, im >= 0, p, ip < R2);
      }
      __syncthreads();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = 2 * G + h;
        A_[i] = nw[h].a; B_[i] = nw[h].b; C_[i] = nw[h].c; D_[i] = nw[h].d;
      }
      __syncthreads();
    }
    f = cmul(D_[rf_i], crcp(B_[rf_i]));
    g = cmul(D_[rg_i], crcp(B_[rg_i]));
  }

  // ---- back-substitute the interior and write the chunk
  bool bad = false;
#pragma unroll
  for (int t = 0; t < MMAX; ++t) {
    if (t < m) {
      C z;
      if (t == 0) z = f;
      else if (t == m - 1) z = g;
      else z = cadd(Y[t], cadd(cmul(P[t], f), cmul(Q[t], g)));
      if (!(isfinite(z.x) && isfinite(z.y))) bad = true;
      my[t] = z;
    }
  }
  if (bad && active && a.flag != nullptr) atomicOr(a.flag, 1);

}

// Non-persistent form (W > 1): load one tile of SB systems, solve, store.
// Batch: work[block] = (problem, tile) selects the descriptor.
template <typename R, int W, bool BATCH>
__global__ void __launch_bounds__(512) k_tridiag(TriArgs a1, const TriArgs* __restrict__ descs,
                                                 const int2* __restrict__ work, int SB) {
  using C = cplx_t<R>;
  const TriArgs& a = BATCH ? descs[work[blockIdx.x].x] : a1;
  const int tile_id = BATCH ? work[blockIdx.x].y : (int)blockIdx.x;
  const int m = max(2, (a.n + 32 * W - 1) / (32 * W));
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rows_pad = 32 * W * (m + 1);
  C* tile = reinterpret_cast<C*>(smraw);                       // [SB][rows_pad]
  C* pa = tile + (size_t)SB * rows_pad;                         // [SB][64W] x 4
  const int R2 = 64 * W;
  C* pb = pa + (size_t)SB * R2;
  C* pc = pb + (size_t)SB * R2;
  C* pd = pc + (size_t)SB * R2;
  const long long q0 = (long long)tile_id * SB;
  tile_copy<C, true, false>(a, tile, rows_pad, m, q0, SB);
  __syncthreads();
  solve_tile<R, W>(a, m, SB, tile, pa, pb, pc, pd, q0);
  __syncthreads();
  tile_copy<C, false, false>(a, tile, rows_pad, m, q0, SB);
}

// cp.async copy of one complex value (8 or 16 bytes) global -> shared
template <typename C>
PD_D void cp_async_c(C* dst, const C* src) {
  const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
  if constexpr (sizeof(C) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
template <typename C, bool ASYNC>
PD_D void put_elem(C* dst, const C* src) {
  if constexpr (ASYNC) cp_async_c(dst, src);
  else *dst = *src;
}
PD_D void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
PD_D void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Persistent, double-buffered form for one warp per system (n <= 256): every
// block walks over tiles of SB systems; the next tile is copied into the other
// shared buffer with cp.async while the current one is solved.  Batch: tile g
// is (problem, tile) = work[g] and may change problem from tile to tile.
template <typename R, bool BATCH>
__global__ void __launch_bounds__(256, 2) k_tridiag_pipe(TriArgs a1, const TriArgs* __restrict__ descs,
                                                         const int2* __restrict__ work, int SB,
                                                         int ntiles, int mmax) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  C* buf[2] = {reinterpret_cast<C*>(smraw),
               reinterpret_cast<C*>(smraw) + (size_t)SB * 32 * (mmax + 1)};
  auto args = [&](int g) -> const TriArgs& { return BATCH ? descs[work[g].x] : a1; };
  auto tid_of = [&](int g) -> int { return BATCH ? work[g].y : g; };
  auto issue = [&](int g, C* tile) {
    const TriArgs& a = args(g);
    const int m = max(2, (a.n + 31) / 32);
    tile_copy<C, true, true>(a, tile, 32 * (m + 1), m, (long long)tid_of(g) * SB, SB);
    cp_async_commit();
  };
  int g = blockIdx.x;
  if (g < ntiles) issue(g, buf[0]);
  for (int it = 0; g < ntiles; g += gridDim.x, ++it) {
    C* cur = buf[it & 1];
    const int gn = g + gridDim.x;
    if (gn < ntiles) {
      issue(gn, buf[(it + 1) & 1]);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const TriArgs& a = args(g);
    const int n = a.n, m = max(2, (n + 31) / 32), rows_pad = 32 * (m + 1);
    const long long q0 = (long long)tid_of(g) * SB;
    solve_tile<R, 1>(a, m, SB, cur, nullptr, nullptr, nullptr, nullptr, q0);
    __syncthreads();
    tile_copy<C, false, false>(a, cur, rows_pad, m, q0, SB);
    __syncthreads();
  }
}

constexpr int PIPE_SB = 8;  // one-warp systems per 256-thread block

template <typename R>
cudaError_t launch_pipe(const TriArgs& a1, const TriArgs* descs, const int2* work, int ntiles,
                        int mmax, cudaStream_t st) {
  using C = cplx_t<R>;
  const size_t smem = (size_t)2 * PIPE_SB * 32 * (mmax + 1) * sizeof(C);
  auto kern = descs ? k_tridiag_pipe<R, true> : k_tridiag_pipe<R, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, nsm = 152, per = 2;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 256, smem);
  const int grid = std::max(1, std::min(ntiles, nsm * std::max(per, 1)));
  kern<<<grid, 256, smem, st>>>(a1, descs, work, PIPE_SB, ntiles, mmax);
  return cudaGetLastError();
}

template <typename R, int W>
cudaError_t launch_w(const TriArgs& a, cudaStream_t st) {
  using C = cplx_t<R>;
  const int m = std::max(2, ceil_div(a.n, 32 * W));
  const long long total = (long long)a.nh * a.J;
  if (total == 0) return cudaSuccess;
  if constexpr (W == 1) {
    const int ntiles = (int)((total + PIPE_SB - 1) / PIPE_SB);
    return launch_pipe<R>(a, nullptr, nullptr, ntiles, m, st);
  } else {
    const int SB = std::max(1, (sizeof(R) == 4 ? 8 : 4) / W);
    const size_t smem = (size_t)SB * (32 * W * (m + 1) + 4 * 64 * W) * sizeof(C);
    auto kern = k_tridiag<R, W, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = (int)((total + SB - 1) / SB);
    kern<<<grid, SB * 32 * W, smem, st>>>(a, nullptr, nullptr, SB);
    return cudaGetLastError();
  }
}

// batched W-warp class (W > 1): tiles of SB systems, work[t] = (problem, tile)
template <typename R, int W>
cudaError_t launch_wb(const TriArgs* descs, const int2* work, int ntiles, int mmax,
                      cudaStream_t st) {
  using C = cplx_t<R>;
  const int SB = std::max(1, (sizeof(R) == 4 ? 8 : 4) / W);
  const size_t smem = (size_t)SB * (32 * W * (mmax + 1) + 4 * 64 * W) * sizeof(C);
  auto kern = k_tridiag<R, W, true>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  TriArgs dummy;
  memset(&dummy, 0, sizeof(dummy));
  kern<<<ntiles, SB * 32 * W, smem, st>>>(dummy, descs, work, SB);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_r(const TriArgs& a, cudaStream_t st) {
  if (a.n <= 256) return launch_w<R, 1>(a, st);
  if (a.n <= 512) return launch_w<R, 2>(a, st);
  if (a.n <= 1024) return launch_w<R, 4>(a, st);
  if (a.n <= 2048) return launch_w<R, 8>(a, st);
  if (a.n <= 4096) return launch_w<R, 16>(a, st);
  return cudaErrorInvalidValue;
}

}  // namespace

cudaError_t launch_tridiag(const TriArgs& a, bool fp64, cudaStream_t st) {
  return fp64 ? launch_r<double>(a, st) : launch_r<float>(a, st);
}

int tridiag_batch_sb(int W, bool fp64) {
  return W == 1 ? PIPE_SB : std::max(1, (fp64 ? 4 : 8) / W);
}

cudaError_t launch_tridiag_batch(const TriArgs* descs, const int2* work, int ntiles, int W,
                                 int mmax, bool fp64, cudaStream_t st) {
  if (ntiles == 0) return cudaSuccess;
  TriArgs dummy;
  memset(&dummy, 0, sizeof(dummy));
  if (fp64) {
    switch (W) {
      case 1: return launch_pipe<double>(dummy, descs, work, ntiles, mmax, st);
      case 2: return launch_wb<double, 2>(descs, work, ntiles, mmax, st);
      case 4: return launch_wb<double, 4>(descs, work, ntiles, mmax, st);
      case 8: return launch_wb<double, 8>(descs, work, ntiles, mmax, st);
      case 16: return launch_wb<double, 16>(descs, work, ntiles, mmax, st);
    }
  } else {
    switch (W) {
      case 1: return launch_pipe<float>(dummy, descs, work, ntiles, mmax, st);
      case 2: return launch_wb<float, 2>(descs, work, ntiles, mmax, st);
      case 4: return launch_wb<float, 4>(descs, work, ntiles, mmax, st);
      case 8: return launch_wb<float, 8>(descs, work, ntiles, mmax, st);
      case 16: return launch_wb<float, 16>(descs, work, ntiles, mmax, st);
    }
  }
  return cudaErrorInvalidValue;
}
