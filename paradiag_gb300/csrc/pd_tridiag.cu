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
#include "pd_internal.h"

namespace {

constexpr int MMAX = 8;

template <typename C>
struct Row4 { C a, b, c, d; };

template <typename R, int W>
__global__ void __launch_bounds__(512) k_tridiag(TriArgs a, int m, int SB) {
  using C = cplx_t<R>;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int rows_pad = 32 * W * (m + 1);
  C* tile = reinterpret_cast<C*>(smraw);                       // [SB][rows_pad]
  C* pa = tile + (size_t)SB * rows_pad;                         // [SB][64W] x 4
  const int R2 = 64 * W;
  C* pb = pa + (size_t)SB * R2;
  C* pc = pb + (size_t)SB * R2;
  C* pd = pc + (size_t)SB * R2;

  const int n = a.n, J = a.J;
  const long long total = (long long)a.nh * J;
  const long long q0 = (long long)blockIdx.x * SB;
  const int nthreads = blockDim.x;

  // ---- coalesced load of SB systems into the padded tile
  C* data = reinterpret_cast<C*>(a.data);
  const long long nel = (long long)SB * n;
  for (long long e = threadIdx.x; e < nel; e += nthreads) {
    int sb, i;
    if (a.stride == 1) { sb = (int)(e / n); i = (int)(e % n); }
    else { i = (int)(e / SB); sb = (int)(e % SB); }
    const long long q = q0 + sb;
    C v = czero<C>();
    if (q < total) {
      const long long k = q / J, j = q % J;
      v = data[k * a.S + j + (long long)i * a.stride];
    }
    tile[(size_t)sb * rows_pad + (i / m) * (m + 1) + (i % m)] = v;
  }
  __syncthreads();

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
      C ai = A_[i], bi = B_[i], ci = C_[i], di = D_[i];
      C na = czero<C>(), nc = czero<C>();
      if (im >= 0) {
        const C k1 = cmul(ai, crcp(B_[im]));
        na = mk(-(A_[im].x * k1.x - A_[im].y * k1.y), -(A_[im].x * k1.y + A_[im].y * k1.x));
        bi = csub(bi, cmul(C_[im], k1));
        di = csub(di, cmul(D_[im], k1));
      }
      if (ip < R2) {
        const C k2 = cmul(ci, crcp(B_[ip]));
        nc = mk(-(C_[ip].x * k2.x - C_[ip].y * k2.y), -(C_[ip].x * k2.y + C_[ip].y * k2.x));
        bi = csub(bi, cmul(A_[ip], k2));
        di = csub(di, cmul(D_[ip], k2));
      }
      nw[h].a = na; nw[h].b = bi; nw[h].c = nc; nw[h].d = di;
    }
    __syncthreads();
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 2 * G + h;
      A_[i] = nw[h].a; B_[i] = nw[h].b; C_[i] = nw[h].c; D_[i] = nw[h].d;
    }
    __syncthreads();
  }
  const C f = cmul(D_[rf_i], crcp(B_[rf_i]));
  const C g = cmul(D_[rg_i], crcp(B_[rg_i]));

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
  __syncthreads();

  for (long long e = threadIdx.x; e < nel; e += nthreads) {
    int sb2, i;
    if (a.stride == 1) { sb2 = (int)(e / n); i = (int)(e % n); }
    else { i = (int)(e / SB); sb2 = (int)(e % SB); }
    const long long qq = q0 + sb2;
    if (qq < total) {
      const long long k = qq / J, j = qq % J;
      data[k * a.S + j + (long long)i * a.stride] =
          tile[(size_t)sb2 * rows_pad + (i / m) * (m + 1) + (i % m)];
    }
  }
}

template <typename R, int W>
cudaError_t launch_w(const TriArgs& a, cudaStream_t st) {
  using C = cplx_t<R>;
  const int m = std::max(2, ceil_div(a.n, 32 * W));
  const int SB = std::max(1, (sizeof(R) == 4 ? 8 : 4) / W);
  const size_t smem = (size_t)SB * (32 * W * (m + 1) + 4 * 64 * W) * sizeof(C);
  auto kern = k_tridiag<R, W>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long total = (long long)a.nh * a.J;
  const int grid = (int)((total + SB - 1) / SB);
  if (grid == 0) return cudaSuccess;
  kern<<<grid, SB * 32 * W, smem, st>>>(a, m, SB);
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
